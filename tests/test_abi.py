"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every symbol the
header declares, the binding wraps each of them, and the host-only coefficient routine agrees
with scipy's exponentially scaled Bessel function.  Also checks that the product path and the
oracle stay independent of each other."""
import ast
import os
import re
import subprocess

import numpy as np
import pytest
import scipy.special as ss

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2211_00805_gb300 import build
    return build.build()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "geosink.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(gs_[a-z0-9_]+)$", out, flags=re.M))
    declared = header_symbols()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, f"declared but not exported: {missing}"


# Calls with no operation of the paper behind them: context, options, diagnostics, tuning, layout.
PLUMBING = {"gs_create", "gs_destroy", "gs_set_stream", "gs_last_error", "gs_sync", "gs_reserve",
            "gs_set_option", "gs_get_option", "gs_launch_count", "gs_sell_step_order", "gs_graph_info",
            "gs_graph_layout", "gs_autotune", "gs_autotune_choices", "gs_graph_destroy"}


def test_every_entry_point_is_documented_and_compute_calls_cite_their_passage():
    # the comment block(s) between one declaration and the next document the latter
    txt = open(os.path.join(ROOT, "include", "geosink.h")).read()
    decl = re.compile(r"^[a-z][^;(]*?\b(gs_[a-z0-9_]+)\s*\([^;]*\);", re.M | re.S)
    prev, docs = 0, {}
    for m in decl.finditer(txt):
        docs[m.group(1)] = " ".join(re.findall(r"/\*(.*?)\*/", txt[prev:m.start()], flags=re.S))
        prev = m.end()
    assert sorted(docs) == header_symbols()
    cite = re.compile(r"Sec\. \d|Algorithm \d|Definition \d|Table \d|Eq\. \d")
    for name, doc in docs.items():
        assert doc.strip(), f"{name}: no comment"
        if name not in PLUMBING:
            assert cite.search(doc), f"{name}: cites no passage of the paper"


def header_constants():
    """Every `GS_NAME = value` of the header's enums (status codes, option numbers)."""
    txt = open(os.path.join(ROOT, "include", "geosink.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(GS_[A-Z0-9_]+)\s*=\s*(\d+)", txt)}


def test_binding_constants_match_the_header_enums():
    # a caller reaching the library through the binding must pass the header's option numbers and
    # read its status codes: every status and option the header defines has the same value there
    from paper_2211_00805_gb300 import binding
    consts = header_constants()
    assert "GS_OK" in consts and "GS_OPT_LOOP_REGS" in consts
    for name, value in consts.items():
        if name.startswith(("GS_OPT_", "GS_OK", "GS_ERR_")):
            assert getattr(binding, name) == value, name
    assert {v: k for k, v in binding.STATUS.items()} == {k: v for k, v in consts.items()
                                                         if k == "GS_OK" or k.startswith("GS_ERR_")}


def test_binding_wraps_every_symbol(built):
    from paper_2211_00805_gb300 import binding
    assert sorted(binding.SIGNATURES) == header_symbols()
    for name in binding.SIGNATURES:
        assert callable(getattr(binding.lib(), name))


@pytest.mark.parametrize("t,K", [(0.5, 10), (1.0, 20), (5.0, 30), (10.0, 40), (8.0, 40), (60.0, 90)])
def test_host_coefficients_match_scipy(built, t, K):
    from paper_2211_00805_gb300 import binding
    c = np.array(binding.gs_cheb_coeffs(t, K))
    k = np.arange(K + 1)
    ref = np.where(k == 0, 1.0, 2.0) * ss.ive(k, t)
    np.testing.assert_allclose(c, ref, rtol=1e-12, atol=1e-300)


def test_host_coefficients_reject_bad_arguments(built):
    from paper_2211_00805_gb300 import binding
    with pytest.raises(binding.GeosinkError):
        binding.gs_cheb_coeffs(-1.0, 5)
    with pytest.raises(binding.GeosinkError):
        binding.gs_cheb_coeffs(1.0, -1)


def _imports(path):
    tree = ast.parse(open(path).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module:
            names.add(node.module.split(".")[0])
    return names


def test_product_never_imports_oracle_and_oracle_never_imports_product():
    pkg = os.path.join(ROOT, "paper_2211_00805_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            assert "oracle" not in _imports(os.path.join(pkg, f)), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            assert "paper_2211_00805_gb300" not in _imports(os.path.join(ROOT, "oracle", f)), f
    src = " ".join(open(os.path.join(pkg, "csrc", f)).read() for f in os.listdir(os.path.join(pkg, "csrc")))
    assert "oracle" not in src.lower()


def _wavefronts(idx, steps):
    """Shared-memory wavefronts of a slice summed in the given step order: per step, the largest
    number of distinct indices that share a bank (at least 1)."""
    W = idx.shape[0]
    order = np.empty_like(idx)
    for l in range(32):
        order[steps[:, l], l] = idx[:, l]
    tot = 0
    for j in range(W):
        per_bank = {}
        for v in set(order[j].tolist()):
            per_bank[v % 32] = per_bank.get(v % 32, 0) + 1
        tot += max(per_bank.values())
    return tot


def test_sell_step_order_is_a_per_row_permutation_without_conflicts_when_banks_balance(built):
    # every bank holds exactly W of the slice's entries: a proper edge colouring exists (Koenig),
    # so no step may put two different indices in one bank
    from paper_2211_00805_gb300 import binding
    rng = np.random.default_rng(5)
    for W in (1, 2, 7, 16, 20, 33, 64):
        banks = rng.permutation(np.repeat(np.arange(32), W))
        idx = (rng.integers(0, 250, W * 32) * 32 + banks).astype(np.uint16).reshape(W, 32)
        steps = binding.gs_sell_step_order(idx)
        for l in range(32):
            assert sorted(steps[:, l].tolist()) == list(range(W))
        assert _wavefronts(idx, steps) == W


def test_sell_step_order_on_unbalanced_banks_stays_a_permutation_and_beats_the_stored_order(built):
    from paper_2211_00805_gb300 import binding
    rng = np.random.default_rng(6)
    for W in (5, 20, 48):
        idx = rng.integers(0, 9000, (W, 32)).astype(np.uint16)
        idx[W // 2:, 3] = idx[0, 3]  # a row whose padding repeats one index
        steps = binding.gs_sell_step_order(idx)
        for l in range(32):
            assert sorted(steps[:, l].tolist()) == list(range(W))
        ident = np.repeat(np.arange(W, dtype=np.uint8)[:, None], 32, axis=1)
        deg = np.bincount((idx % 32).ravel(), minlength=32).max()
        assert max(W, deg) <= _wavefronts(idx, steps) < _wavefronts(idx, ident)


def test_sell_step_order_rejects_bad_widths(built):
    from paper_2211_00805_gb300 import binding
    with pytest.raises(binding.GeosinkError):
        binding.gs_sell_step_order(np.zeros((65, 32), np.uint16))
    with pytest.raises(binding.GeosinkError):
        binding.gs_sell_step_order(np.zeros((0, 32), np.uint16))
