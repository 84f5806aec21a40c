"""C-ABI checks that need no GPU: the library loads, exports every declared symbol,
and its host planner (Chebyshev coefficients, degree rule, radial cores) matches the
oracle."""
import os
import re

import numpy as np
import pytest

from oracle import chebyshev, hdf as ohdf, radial
from paper_2202_03655_gb300 import hdf
from paper_2202_03655_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(hdf_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = hdf.lib()
    names = declared_symbols()
    assert "hdf_build" in names and "hdf_matvec" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(hdf.SIGNATURES) <= names


def test_status_strings():
    lib = hdf.lib()
    for s in range(9):
        assert lib.hdf_status_string(s)


@pytest.mark.parametrize("kname", ["gaussian", "cauchy", "matern32", "matern52"])
@pytest.mark.parametrize("two_r", [1.0, 4.0, 13.0])
def test_planner_cheb_coeffs_match_oracle(kname, two_r):
    M = hdf.cheb_nodes(64)
    assert M == ohdf.cheb_nodes_count(64)
    a_lib = hdf.cheb_coeffs(kname, 0.7, two_r, M)
    from oracle.kernels import kernel
    a_orc = chebyshev.cheb_coeffs(lambda r: kernel(kname, two_r * r, 0.7), M)
    assert np.abs(a_lib - a_orc).max() <= 1e-14
    for budget in (1e-3, 1e-6, 1e-9):
        assert hdf.choose_degree(a_lib, budget, 64)[0] == chebyshev.choose_degree(a_orc, budget, 64)[0]


@pytest.mark.parametrize("d", [3, 4, 5, 8])
@pytest.mark.parametrize("kname,ell", [("gaussian", 0.5), ("cauchy", 2.0), ("matern52", 1.0)])
def test_planner_radial_cores_match_oracle(d, kname, ell):
    x = W.points("ball3_gauss", n=200) if d == 3 else np.random.default_rng(d).standard_normal((200, d))
    _, pl = ohdf.plan(x, kname, ell, 1e-7, p_max=48)
    lib_cores = hdf.radial_cores(pl.a, pl.p, d)
    orc_cores = radial.stable_core(pl.a, pl.p, d)
    scale = max(np.abs(c).max() for c in orc_cores if c.size)
    for k, (cl, co) in enumerate(zip(lib_cores, orc_cores)):
        assert cl.shape == co.shape
        assert np.abs(cl - co).max() <= 1e-12 * scale, k


def test_missing_library_fails_loudly(tmp_path):
    """Without libhdf.so every call raises: the binding has no CPU fallback."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2202_03655_gb300 import hdf\n"
            "hdf.LIB_PATH = %r\n"
            "hdf._lib = None\n"
            "try:\n"
            "    hdf.cheb_nodes(16)\n"
            "except RuntimeError as e:\n"
            "    print('raised', 'missing' in str(e))\n"
            "else:\n"
            "    print('no error')\n") % (ROOT, str(tmp_path / "absent" / "libhdf.so"))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert out.stdout.strip() == "raised True", out.stdout + out.stderr
