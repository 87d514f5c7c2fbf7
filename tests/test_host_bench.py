"""Host logic of bench.py (CPU only): the clock record that decides whether a run is kept, the
ncu traffic lookup that must go null once a kernel's source changes, and the peak denominator."""
import hashlib
import json
import os

import pytest

import bench

IDLE = "2070, 2070, 850.25, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"


def test_clock_summary_median_max_and_no_reasons():
    text = "\n".join([IDLE, IDLE.replace("2070, 2070", "1995, 2070"), IDLE.replace("2070, 2070", "2055, 2070")])
    s = bench.summarise_clocks(text + "\n")
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


@pytest.mark.parametrize("col,name", [(4, "hw_slowdown"), (5, "hw_thermal_slowdown"),
                                      (6, "sw_thermal_slowdown"), (7, "sw_power_cap")])
def test_clock_summary_reports_each_active_reason(col, name):
    fields = [x.strip() for x in IDLE.split(",")]
    fields[col] = "Active"
    s = bench.summarise_clocks("\n".join([IDLE, ", ".join(fields), IDLE]))
    assert s["reasons"] == [name] and s["samples"] == 3


def test_clock_summary_skips_unreadable_lines_and_reports_none_without_samples():
    assert bench.summarise_clocks("") is None
    assert bench.summarise_clocks("[N/A], [N/A], [N/A], 0x0, Not Active, Not Active, Not Active, Not Active") is None
    s = bench.summarise_clocks("garbage\n" + IDLE + "\n1, 2, 3\n")
    assert s["samples"] == 1 and s["sm_mhz"] == 2070.0


def _fake_tree(root, source_text, table_lines):
    csrc = root / "paper_2211_00805_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "cheb.cu").write_text(source_text)
    (root / "profiles").mkdir()
    (root / "profiles" / "ncu_traffic.txt").write_text("\n".join(table_lines) + "\n")
    return hashlib.sha256(source_text.encode()).hexdigest()[:16]


def test_ncu_traffic_only_while_the_source_hash_matches(tmp_path, monkeypatch):
    h = _fake_tree(tmp_path, "// kernel v1\n", [])
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text(
        f"# comment\norder_x  {h}  123456\norder_y  0000000000000000  99\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("order_x") == 123456.0
    assert bench.ncu_traffic("order_y") is None  # taken on another version of the file
    assert bench.ncu_traffic("order_z") is None  # never captured
    (tmp_path / "paper_2211_00805_gb300" / "csrc" / "cheb.cu").write_text("// kernel v2\n")
    assert bench.ncu_traffic("order_x") is None  # the kernel changed since the capture


def test_ncu_traffic_without_files_is_none(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("order_x") is None


def test_peak_is_the_measured_copy_bandwidth_else_the_fallback(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6786.2, "bf16_tflops": 1900}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6786.2, "measured")
    os.remove(tmp_path / "MEASURED_PEAKS.json")
    assert bench.measured_peaks() == (6800.0, "fallback")


@pytest.mark.parametrize("n,iters,S", [(100_000, 500, 1), (100_000, 500, 7), (100_000, 500, 20), (13, 5, 8)])
def test_reference_shares_cover_one_whole_step(n, iters, S):
    # the reference arm's timed shares add up to exactly one step: every query row once, and the
    # iteration counts summing to the workload's
    rows, its = bench.reference_shares(n, iters, S)
    allrows = [r for part in rows for r in part.tolist()]
    assert allrows == list(range(n))
    assert sum(its) == iters and len(its) == S and max(its) - min(its) <= 1


def test_both_arms_print_the_same_config():
    assert bench.static_config(1, 123) == bench.static_config(1, 123)
    c = bench.static_config(1, 2005410)
    assert c["n"] == bench.WORKLOAD["n"] and c["iters"] == bench.WORKLOAD["iters"] and c["nnz"] == 2005410
    assert not any(k.endswith("_ms") for k in c)  # no timings in the config


def test_loop_roofline_persistent_form_counts_every_order_and_its_floor():
    # 100k rows, 2,005,410 nonzeros, K = 30, 500 iterations in 61.5 ms: the byte model of the
    # 30,000 orders over the loop's time, against the peak; the floor fraction from the per-order time
    n, nnz, K, iters, s = 100_000, 2_005_410, 30, 500, 0.0615
    r = bench.loop_roofline(n, nnz, K, iters, s, {"loop_mode": 0, "persist_sync": 2}, 6800.3, "measured")
    per_apply = bench.apply_bytes(n, nnz, K, 1, last_streams=6)
    assert r["bytes_per_launch"] == 2 * iters * per_apply
    assert r["achieved"] == pytest.approx(2 * iters * per_apply / s / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.3)
    assert r["order_us"] == pytest.approx(s / (2 * K * iters) * 1e6)
    assert r["frac_of_exchange_floor"] == pytest.approx(bench.EXCHANGE_FLOOR_US / r["order_us"])
    assert 0 < r["frac_of_exchange_floor"] < 1  # a loop cannot beat its own exchange
    assert r["kernel"].startswith("sinkhorn_tagged") and r["unit"] == "GB/s" and r["bound"] == "hbm"


def test_loop_roofline_per_order_form_has_no_floor():
    r = bench.loop_roofline(100_000, 2_005_410, 30, 500, 0.3, {"loop_mode": 1, "persist_sync": 2}, 6800.3, "measured")
    assert "frac_of_exchange_floor" not in r
    assert r["launch_us"] == pytest.approx(r["order_us"])
