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
