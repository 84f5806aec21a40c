"""Parity of the CUDA path with the oracle on the inputs of the two sweeps of Sec. 4.1: the
time-vs-n points (Fig. 1: N(0, I) scaled to max norm 1, Cauchy l = 1, tol 1e-3, d = 3..6) and
the error-vs-rank points (Fig. 3: d = 5, four kernels with sigma = 1, a range of tolerances)."""
import numpy as np
import pytest

from gpu_common import rel, to_dev
from oracle import hdf as ohdf
from paper_2202_03655_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2202_03655_gb300 import hdf
    return hdf


@pytest.mark.parametrize("d", [3, 4, 5, 6])
def test_fig1_points_matvec_vs_oracle(d):
    import torch
    hdf = _lib()
    w = W.WORKLOADS["fig1_cauchy"]
    x = W.maxnorm1_points("fig1_cauchy", 3001, d)
    f = hdf.build(to_dev(x), w["kernel"], w["ell"], w["tol"], precision="fp32")
    fo = ohdf.build(x, w["kernel"], w["ell"], w["tol"])
    assert f.info.p == fo.plan.p and f.info.reached
    v = np.random.default_rng(d).standard_normal((3001, 2))
    y = f.matvec(to_dev(v, torch.float32)).double().cpu().numpy()
    assert rel(y, ohdf.matvec(fo, v)) <= 10 * w["tol"]
    assert rel(y, ohdf.dense_kernel(x, w["kernel"], w["ell"]) @ v) <= w["tol"]


# Matern-3/2 (coefficients decaying like i^-4) needs p > 64 below tol 1e-3 in d = 5, where the
# factor has far more columns than points; its finer tolerances are left to the sweep itself.
FIG3_CASES = [(k, l, t) for k, l in W.WORKLOADS["fig3_rank5"]["kernels"]
              for t in ((1e-2, 1e-3) if k == "matern32" else (1e-2, 1e-4))]


@pytest.mark.parametrize("kname,ell,tol", FIG3_CASES)
def test_fig3_error_and_rank_vs_oracle(kname, ell, tol):
    """FP64 factor on 1,200 points of the d = 5 sweep: same degree as the oracle, rank within
    5%, achieved |K - K~|_F / |K|_F within tol and within a factor of two of the oracle's own
    error."""
    hdf = _lib()
    x = W.maxnorm1_points("fig3_rank5", 5000, 5)[:1200]
    f = hdf.build(to_dev(x), kname, ell, tol, precision="fp64")
    fo = ohdf.build(x, kname, ell, tol)
    assert f.info.p == fo.plan.p and bool(f.info.reached) == bool(fo.plan.reached)
    assert abs(f.rank - fo.rank) <= 0.05 * fo.rank + 2
    U, S = f.export()
    K = ohdf.dense_kernel(x, kname, ell)
    err = np.linalg.norm(K - (U * S) @ U.T) / np.linalg.norm(K)
    err_o = ohdf.rel_fro_error(fo, x, kname, ell)
    if fo.plan.reached:
        assert err <= tol
    assert err <= 2 * err_o + 1e-12
    v = np.random.default_rng(3).standard_normal(1200)
    assert rel(f.matvec(to_dev(v)).cpu().numpy(), ohdf.matvec(fo, v)) <= 10 * max(tol, err_o)
