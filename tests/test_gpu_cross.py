"""Parity of the cross factorization K(X, Y) ~= U S V^T (hdf_build_cross, hdf_matvec,
hdf_matvec_transpose) with the CPU oracle of Algorithm 1's general form, on the same seeded
inputs.  As for the symmetric factor, parity is checked on products and on entries of K~,
never on U or V (singular vectors are unique only up to sign and rotation)."""
import functools

import numpy as np
import pytest

from gpu_common import rel, to_dev
from oracle import cross as ocross
from paper_2202_03655_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2202_03655_gb300 import hdf
    return hdf


def _sets(seed, m, n, d, shift=0.6):
    g = np.random.default_rng(seed)
    x = W.uniform_ball(g, m, d, 1.0)
    y = g.standard_normal((n, d)) * 0.5 + shift
    return x, y


def _dt(prec):
    import torch
    return torch.float64 if prec == "fp64" else torch.float32


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("d,kname,ell,tol", [(3, "gaussian", 0.5, 1e-6), (4, "cauchy", 1.5, 1e-5),
                                             (5, "matern52", 2.0, 1e-3), (3, "matern32", 1.0, 1e-4)])
def test_cross_matvec_and_transpose_vs_oracle(prec, d, kname, ell, tol):
    """K~ V and K~^T W against the oracle's factor, and against the dense cross kernel."""
    hdf = _lib()
    x, y = _sets(40 + d, 1531, 1097, d)
    f = hdf.build_cross(to_dev(x), to_dev(y), kname, ell, tol, precision=prec)
    fo = ocross.build_xy(x, y, kname, ell, tol)
    assert f.info.p == fo.plan.p and f.n == 1531 and f.n_y == 1097
    assert abs(f.rank - fo.rank) <= 0.05 * fo.rank + 2
    g = np.random.default_rng(3)
    V, Wt = g.standard_normal((1097, 5)), g.standard_normal((1531, 3))
    Y = f.matvec(to_dev(V, _dt(prec))).double().cpu().numpy()
    Z = f.matvec_t(to_dev(Wt, _dt(prec))).double().cpu().numpy()
    assert f.device_errors() == 0
    assert rel(Y, ocross.matvec_xy(fo, V)) <= 10 * tol
    assert rel(Z, ocross.matvec_xy_t(fo, Wt)) <= 10 * tol
    K = ocross.dense_kernel_xy(x, y, kname, ell)
    assert rel(Y, K @ V) <= 10 * tol
    assert rel(Z, K.T @ Wt) <= 10 * tol


def test_cross_entries_vs_oracle():
    """Entries of K~ = U S V^T from the exported factors against the oracle's entries."""
    hdf = _lib()
    x, y = _sets(5, 700, 450, 4)
    tol = 1e-6
    f = hdf.build_cross(to_dev(x), to_dev(y), "gaussian", 0.8, tol)
    fo = ocross.build_xy(x, y, "gaussian", 0.8, tol)
    U, S = f.export()
    V = f.export_y()
    assert U.shape == (700, f.rank) and V.shape == (450, f.rank)
    Kt = (U * S) @ V.T
    Ko = (fo.U * fo.S) @ fo.V.T
    assert np.abs(Kt - Ko).max() <= 10 * tol * np.abs(Ko).max()
    K = ocross.dense_kernel_xy(x, y, "gaussian", 0.8)
    assert np.linalg.norm(K - Kt) <= tol * np.linalg.norm(K)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cross_with_x_equal_y_matches_symmetric(prec):
    """X = Y: the cross factor's product equals the symmetric factor's (Remark 1)."""
    hdf = _lib()
    x = W.points("ball3_gauss", n=1800)
    fc = hdf.build_cross(to_dev(x), to_dev(x), "gaussian", 0.5, 1e-6, precision=prec)
    fs = hdf.build(to_dev(x), "gaussian", 0.5, 1e-6, precision=prec)
    assert fc.info.p == fs.info.p and list(fc.s_k) == list(fs.s_k)
    v = np.random.default_rng(1).standard_normal((1800, 2))
    a = fc.matvec(to_dev(v, _dt(prec))).double().cpu().numpy()
    b = fs.matvec(to_dev(v, _dt(prec))).double().cpu().numpy()
    assert rel(a, b) <= (1e-11 if prec == "fp64" else 2e-6)


@pytest.mark.parametrize("m,n", [(1, 1), (1, 300), (300, 1), (5, 3), (2, 4099)])
def test_cross_degenerate_sizes(m, n):
    hdf = _lib()
    x, y = _sets(m * 7 + n, m, n, 3)
    tol = 1e-6
    f = hdf.build_cross(to_dev(x), to_dev(y), "gaussian", 0.9, tol)
    fo = ocross.build_xy(x, y, "gaussian", 0.9, tol)
    V = np.random.default_rng(2).standard_normal((n, 2))
    Y = f.matvec(to_dev(V)).cpu().numpy()
    K = ocross.dense_kernel_xy(x, y, "gaussian", 0.9)
    assert rel(Y, ocross.matvec_xy(fo, V)) <= 10 * tol
    assert rel(Y, K @ V) <= 10 * tol
    Z = f.matvec_t(to_dev(np.ones((m, 1)))).cpu().numpy()
    assert rel(Z, K.T @ np.ones((m, 1))) <= 10 * tol


@functools.lru_cache(maxsize=None)
def _fp32_cross(flags):
    hdf = _lib()
    x, y = _sets(9, 20011, 6007, 4)
    f = hdf.build_cross(to_dev(x), to_dev(y), "gaussian", 0.8, 1e-6, precision="fp32", flags=flags)
    U, S = f.export()
    return f, U.astype(np.float64), S, f.export_y().astype(np.float64)


@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("c", [1, 9, 16, 37, 64, 70])
def test_cross_fp32_column_counts(flags, c):
    """FP32 products on the tensor cores (flags 0, 9..64 columns per group) and on the CUDA
    cores against an FP64 product of the exported U, S, V."""
    f, U, S, V = _fp32_cross(flags)
    B = np.random.default_rng(c).standard_normal((6007, c)).astype(np.float32)
    Wt = np.random.default_rng(c + 1).standard_normal((20011, c)).astype(np.float32)
    Y = f.matvec(to_dev(B)).double().cpu().numpy()
    Z = f.matvec_t(to_dev(Wt)).double().cpu().numpy()
    assert f.device_errors() == 0
    assert rel(Y, U @ (S[:, None] * (V.T @ B.astype(np.float64)))) <= 1e-5
    assert rel(Z, V @ (S[:, None] * (U.T @ Wt.astype(np.float64)))) <= 1e-5


def test_cross_rejects_symmetric_only_calls():
    import torch
    hdf = _lib()
    x, y = _sets(11, 300, 200, 3)
    f = hdf.build_cross(to_dev(x), to_dev(y), "gaussian", 0.9, 1e-6)
    with pytest.raises(hdf.HdfError):
        f.solve(1.0, torch.zeros(300, dtype=torch.float64, device="cuda"))
    with pytest.raises(hdf.HdfError):
        f.adjoint(to_dev(x), torch.zeros(300, dtype=torch.float64, device="cuda"),
                  torch.zeros(300, dtype=torch.float64, device="cuda"))
    fs = hdf.build(to_dev(x), "gaussian", 0.9, 1e-6)
    with pytest.raises(hdf.HdfError):
        fs.export_y()
    # symmetric factor: the transposed product is the product
    v = to_dev(np.random.default_rng(0).standard_normal(300))
    assert rel(fs.matvec_t(v).cpu().numpy(), fs.matvec(v).cpu().numpy()) <= 1e-15


def test_cross_large_sampled_rows():
    """400,000 points of the 8-component mixture against 100,000 points of a wider Gaussian
    cloud (joint radius 6.9), Gaussian l = 1.5, tol 1e-6, FP32, 16 columns: sampled rows of
    K~ V and of K~^T W against the exact kernel."""
    import torch
    hdf = _lib()
    x = W.points("mixture3_matern", n=400000)
    y = np.random.default_rng(21).standard_normal((100000, 3)) * 1.2
    f = hdf.build_cross(to_dev(x), to_dev(y), "gaussian", 1.5, 1e-6, precision="fp32")
    assert f.info.reached
    g = np.random.default_rng(4)
    V = g.standard_normal((100000, 16)).astype(np.float32)
    Wt = g.standard_normal((400000, 16)).astype(np.float32)
    Y = f.matvec(to_dev(V))
    Z = f.matvec_t(to_dev(Wt))
    assert f.device_errors() == 0
    xt, yt = to_dev(x), to_dev(y)
    rows = torch.from_numpy(np.sort(g.choice(400000, 256, replace=False))).cuda()
    cols = torch.from_numpy(np.sort(g.choice(100000, 256, replace=False))).cuda()
    Kr = torch.exp(-0.5 * (torch.cdist(xt[rows], yt) / 1.5) ** 2)    # 256 x 100,000
    Kc = torch.exp(-0.5 * (torch.cdist(yt[cols], xt) / 1.5) ** 2)    # 256 x 400,000
    ey = rel(Y[rows].double().cpu().numpy(), (Kr @ to_dev(V).double()).cpu().numpy())
    ez = rel(Z[cols].double().cpu().numpy(), (Kc @ to_dev(Wt).double()).cpu().numpy())
    assert ey <= 1e-5 and ez <= 1e-5, (ey, ez)
