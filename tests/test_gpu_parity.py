"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same seeded inputs.

K~ is unique but U is not (eigenvector signs, rotations in degenerate eigenspaces), so
parity is checked on K~ V, on solves and on K~ entries, never on U itself.  The bar is
|K~_gpu V - K~_oracle V| / |K~_oracle V| <= 10 tol, the tolerance the factorization is
asked for (both sides are within tol of K in relative Frobenius norm).
"""
import numpy as np
import pytest

from gpu_common import dense_rows_matvec_torch, rel, to_dev
from oracle import hdf as ohdf
from paper_2202_03655_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2202_03655_gb300 import hdf
    return hdf


def _pair(x, kname, ell, tol, prec="fp64", **kw):
    import torch
    hdf = _lib()
    f = hdf.build(to_dev(x), kname, ell, tol, precision=prec, **kw)
    fo = ohdf.build(x, kname, ell, tol, **kw)
    return f, fo


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ball3_gauss_matvec_vs_oracle_and_dense(prec):
    """2,000 points uniform in the unit ball, Gaussian l = 0.5, tol 1e-6: K~ v against the
    oracle and against the dense 2000 x 2000 kernel matrix."""
    import torch
    x = W.points("ball3_gauss")
    tol = 1e-6
    f, fo = _pair(x, "gaussian", 0.5, tol, prec)
    assert f.info.p == fo.plan.p
    assert abs(f.rank - fo.rank) <= 0.05 * fo.rank
    v = W.rng(100).standard_normal(x.shape[0])
    dt = torch.float64 if prec == "fp64" else torch.float32
    y = f.matvec(to_dev(v, dt)).double().cpu().numpy()
    yo = ohdf.matvec(fo, v)
    assert rel(y, yo) <= 10 * tol
    K = ohdf.dense_kernel(x, "gaussian", 0.5)
    assert rel(y, K @ v) <= 10 * tol


@pytest.mark.parametrize("d,kname,ell,tol", [(3, "cauchy", 0.6, 1e-5), (4, "gaussian", 0.8, 1e-6),
                                             (5, "cauchy", 2.0, 1e-4), (5, "matern52", 1.5, 1e-3),
                                             (4, "matern32", 2.0, 1e-3)])
@pytest.mark.parametrize("n", [1, 7, 33, 1531])
def test_kernels_dims_ragged_sizes(d, kname, ell, tol, n):
    x = np.random.default_rng(1000 + n + d).standard_normal((n, d))
    f, fo = _pair(x, kname, ell, tol)
    v = np.random.default_rng(7).standard_normal((n, 3))
    y = f.matvec(to_dev(v)).cpu().numpy()
    yo = ohdf.matvec(fo, v)
    assert rel(y, yo) <= 10 * tol
    assert f.info.p == fo.plan.p


def test_many_columns_and_layout():
    """ncols = 37 spans three column groups; matvec of column j equals K~ v_j."""
    x = W.points("cube4_gauss", n=3000)
    f, fo = _pair(x, "gaussian", 0.8, 1e-6)
    V = np.random.default_rng(3).standard_normal((3000, 37))
    Y = f.matvec(to_dev(V)).cpu().numpy()
    Yo = ohdf.matvec(fo, V)
    for j in (0, 15, 16, 36):
        assert rel(Y[:, j], Yo[:, j]) <= 1e-5


def test_identical_points_and_single_point():
    import torch
    hdf = _lib()
    # K = k(0) 1 1^T exactly; the factor approximates it to tol like any other input
    x = np.ones((50, 3)) * 0.3
    f = hdf.build(to_dev(x), "gaussian", 1.0, 1e-6)
    v = np.arange(50, dtype=np.float64)
    y = f.matvec(to_dev(v)).cpu().numpy()
    assert rel(y, np.full(50, v.sum())) <= 1e-6
    f1 = hdf.build(to_dev(np.array([[1.0, 2.0, 3.0]])), "cauchy", 1.0, 1e-6)
    assert rel(f1.matvec(to_dev(np.array([2.5]))).cpu().numpy(), [2.5]) <= 1e-6


def test_entries_of_K_tilde_match_oracle():
    """Exported U S U^T equals the oracle's K~ entrywise (K~ is unique, U is not)."""
    x = W.points("ball3_gauss", n=600)
    f, fo = _pair(x, "gaussian", 0.5, 1e-7)
    U, S = f.export()
    Kt = (U * S) @ U.T
    Kto = (fo.U * fo.S) @ fo.U.T
    assert np.abs(Kt - Kto).max() <= 1e-6 * np.abs(Kto).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve_vs_oracle(prec):
    import torch
    x = W.points("ball3_gauss", n=1500)
    tol = 1e-7 if prec == "fp64" else 1e-5
    f, fo = _pair(x, "gaussian", 0.5, tol, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    B = np.random.default_rng(9).standard_normal((1500, 2))
    for lam in (1e-1, 1e-3):
        X = f.solve(lam, to_dev(B, dt), refine_steps=1).double().cpu().numpy()
        Xo = ohdf.solve(fo, lam, B)
        assert rel(X, Xo) <= (1e-6 if prec == "fp64" else 2e-3), lam


def test_error_falls_with_tol():
    """Relative error against the dense matrix falls as tol falls (abstract, Remark 3)."""
    import torch
    hdf = _lib()
    x = W.points("ball3_gauss")
    K = ohdf.dense_kernel(x, "gaussian", 0.5)
    v = W.rng(5).standard_normal(x.shape[0])
    errs = []
    for tol in (1e-2, 1e-4, 1e-6, 1e-8):
        f = hdf.build(to_dev(x), "gaussian", 0.5, tol)
        e = rel(f.matvec(to_dev(v)).cpu().numpy(), K @ v)
        assert e <= tol
        errs.append(e)
    assert errs == sorted(errs, reverse=True)


def test_cube4_full_size_sampled_rows():
    """500,000 points in [-1,1]^4, Gaussian l = 0.8, tol 1e-6, FP32 (the differentiation
    workload's size): sampled rows of K~ v against exact rows of K v."""
    import torch
    hdf = _lib()
    x = W.points("cube4_gauss")
    v = W.rng(103).standard_normal(x.shape[0])
    for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        f = hdf.build(to_dev(x), "gaussian", 0.8, 1e-6, precision=prec)
        y = f.matvec(to_dev(v, dt)).double().cpu().numpy()
        rows = np.sort(W.rng(7).choice(x.shape[0], 1024, replace=False))
        exact = dense_rows_matvec_torch(x, "gaussian", 0.8, v[:, None], rows)[:, 0]
        assert rel(y[rows], exact) <= 1e-5, prec
        del f
