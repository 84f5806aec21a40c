"""The matrix-free form of the factor (U not stored; HDF_FLAG_MATRIX_FREE, chosen by hdf_build
by itself when U would not fit) through the C ABI.

* Against the stored form of the same factor (same points, same build): K~ V agrees to the
  rounding of the bulk precision -- the two forms multiply the same numbers in a different
  order -- for d = 4, 5, 6, several kernels, ragged sizes and 1 to 70 columns.
* Against the oracle on the d = 5 Cauchy recipe of the large workload (standardised rotated
  normal points, l = 2, tol 1e-4) at 3,000 points: within 10 tol, and within the tighter
  same-factor bound.
* The adjoint of a matrix-free factor (U^T [v w] from the Z rows, harmonics recomputed per
  point) equals the adjoint of the stored factor.
* All 4,000,000 points of that recipe: the build selects the matrix-free form by itself (U
  would be more than a terabyte), and sampled rows of K~ V (16 columns) agree with exact rows
  of K V within the build's a-priori bound.
"""
import numpy as np
import pytest

from gpu_common import dense_rows_matvec_torch, rel, to_dev
from oracle import hdf as ohdf
from paper_2202_03655_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _pair(x, kname, ell, tol, prec, p_max=None):
    from paper_2202_03655_gb300 import hdf
    xt = to_dev(x)
    fs = hdf.build(xt, kname, ell, tol, precision=prec, p_max=p_max)
    fm = hdf.build(xt, kname, ell, tol, precision=prec, p_max=p_max, flags=hdf.FLAG_MATRIX_FREE)
    return fs, fm


@pytest.mark.parametrize("d,kname,ell,tol", [(4, "gaussian", 0.8, 1e-6), (5, "cauchy", 2.0, 1e-4),
                                             (5, "matern52", 1.5, 1e-3), (6, "gaussian", 1.2, 1e-5)])
@pytest.mark.parametrize("n", [1, 7, 33, 1531])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_matrix_free_equals_stored(d, kname, ell, tol, n, prec):
    import torch
    x = np.random.default_rng(500 + n + d).standard_normal((n, d))
    fs, fm = _pair(x, kname, ell, tol, prec)
    if fs.rank > 0:
        assert fm.info.matrix_free == 1 and fs.info.matrix_free == 0
    assert fm.rank == fs.rank and fm.info.ldu == fs.info.ldu
    dt = torch.float64 if prec == "fp64" else torch.float32
    V = np.random.default_rng(9).standard_normal((n, 5))
    Ys = fs.matvec(to_dev(V, dt)).double().cpu().numpy()
    Ym = fm.matvec(to_dev(V, dt)).double().cpu().numpy()
    assert np.isfinite(Ym).all()
    if prec == "fp64":
        assert rel(Ym, Ys) <= 1e-11
    else:
        # FP32 rounding of the factor's entries, amplified by the cancellation in U S U^T V (rank
        # far above n here): both forms are held against the FP64 factor's product, the
        # matrix-free one to the order of the stored one's own error
        from paper_2202_03655_gb300 import hdf
        f64 = hdf.build(to_dev(x), kname, ell, tol, precision="fp64")
        Y64 = f64.matvec(to_dev(V)).cpu().numpy()
        assert rel(Ym, Y64) <= 2 * rel(Ys, Y64) + 2e-6
        assert rel(Ym, Ys) <= 1e-4


@pytest.mark.parametrize("c", [1, 3, 16, 37, 64, 70])
def test_matrix_free_column_counts(c):
    """FP32 matrix-free products on the tensor cores (the default) and on the CUDA cores
    (HDF_FLAG_CUDA_CORES) against the stored factor, column by column."""
    import torch
    from paper_2202_03655_gb300 import hdf
    x = W.points("normal5_cauchy", n=2003)
    fs, fm = _pair(x, "cauchy", 2.0, 1e-3, "fp32")
    fc = hdf.build(to_dev(x), "cauchy", 2.0, 1e-3, precision="fp32",
                   flags=hdf.FLAG_MATRIX_FREE | hdf.FLAG_CUDA_CORES)
    V = to_dev(np.random.default_rng(c).standard_normal((x.shape[0], c)), torch.float32)
    Ys = fs.matvec(V).double().cpu().numpy()
    Ym = fm.matvec(V).double().cpu().numpy()
    Yc = fc.matvec(V).double().cpu().numpy()
    assert fm.device_errors() == 0
    for j in range(c):
        assert rel(Ym[:, j], Ys[:, j]) <= 2e-5, j
        assert rel(Yc[:, j], Ys[:, j]) <= 2e-5, j


def test_matrix_free_padded_leading_dimension_ragged_n():
    """A point count that is not a multiple of 4 with V's leading dimension padded to one (rows of
    16-byte multiples), so the B generators of U^T V take their vector loads up to the last full
    group of four points and element loads after it.  The padding holds NaN: a read past the
    last point would reach the result."""
    import torch
    from paper_2202_03655_gb300 import hdf
    n, c, ld = 1533, 16, 1536
    x = W.points("normal5_cauchy", n=n)
    fs, fm = _pair(x, "cauchy", 2.0, 1e-3, "fp32")
    V = np.random.default_rng(77).standard_normal((n, c))
    Vp = torch.full((c, ld), float("nan"), dtype=torch.float32, device="cuda")
    Vp[:, :n] = torch.from_numpy(V.T.astype(np.float32)).cuda()
    Y = torch.zeros((c, ld), dtype=torch.float32, device="cuda")
    fm.matvec_ptr(Vp.data_ptr(), ld, c, Y.data_ptr(), ld)
    torch.cuda.synchronize()
    assert fm.device_errors() == 0
    Ym = Y[:, :n].t().double().cpu().numpy()
    Ys = fs.matvec(to_dev(V, torch.float32)).double().cpu().numpy()
    assert np.isfinite(Ym).all()
    for j in range(c):
        assert rel(Ym[:, j], Ys[:, j]) <= 2e-5, j


@pytest.fixture(scope="module")
def oracle_normal5():
    x = W.points("normal5_cauchy", n=3000)
    fo = ohdf.build(x, "cauchy", 2.0, 1e-4)
    V = W.rng(102).standard_normal((x.shape[0], 16))
    return x, fo, V, ohdf.matvec(fo, V)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_normal5_cauchy_matrix_free_vs_oracle(oracle_normal5, prec):
    """Both sides build the same degree and truncation; they differ by eigenpairs at the budget
    boundary (a relative change of order tol), the radial-basis factor and the bulk rounding."""
    import torch
    from paper_2202_03655_gb300 import hdf
    x, fo, V, Yo = oracle_normal5
    f = hdf.build(to_dev(x), "cauchy", 2.0, 1e-4, precision=prec, flags=hdf.FLAG_MATRIX_FREE)
    assert f.info.matrix_free == 1
    assert f.info.p == fo.plan.p
    assert abs(f.rank - fo.rank) <= 0.05 * fo.rank
    dt = torch.float64 if prec == "fp64" else torch.float32
    Y = f.matvec(to_dev(V, dt)).double().cpu().numpy()
    worst = max(rel(Y[:, j], Yo[:, j]) for j in range(V.shape[1]))
    print(f"normal5_cauchy 3000 matrix-free {prec}: rank {f.rank} (oracle {fo.rank}), worst column {worst:.3e}")
    assert worst <= 10 * 1e-4
    assert worst <= (1e-5 if prec == "fp64" else 1e-4)


def test_matrix_free_adjoint_equals_stored():
    import torch
    g = np.random.default_rng(12)
    x = W.uniform_cube(g, 2500, 4)
    fs, fm = _pair(x, "gaussian", 0.8, 1e-7, "fp64")
    V, Wm = g.standard_normal((2500, 2)), g.standard_normal((2500, 2))
    Gs, dls, vs = fs.adjoint(to_dev(x), to_dev(V), to_dev(Wm))
    Gm, dlm, vm = fm.adjoint(to_dev(x), to_dev(V), to_dev(Wm))
    assert rel(Gm.cpu().numpy(), Gs.cpu().numpy()) <= 1e-10
    assert abs(dlm - dls) <= 1e-10 * abs(dls)
    assert abs(vm - vs) <= 1e-10 * abs(vs)


def test_matrix_free_refuses_what_needs_U():
    import torch
    from paper_2202_03655_gb300 import hdf
    x = W.uniform_cube(np.random.default_rng(3), 500, 4)
    f = hdf.build(to_dev(x), "gaussian", 0.8, 1e-6, flags=hdf.FLAG_MATRIX_FREE)
    B = to_dev(np.ones(500))
    for call in (lambda: f.solve(1.0, B), lambda: f.export()):
        with pytest.raises(hdf.HdfError) as ei:
            call()
        assert ei.value.status == 1
    with pytest.raises(hdf.HdfError):
        hdf.build(to_dev(W.points("ball3_gauss", n=200)), "gaussian", 0.5, 1e-6, flags=hdf.FLAG_MATRIX_FREE)


def test_normal5_cauchy_full_size_sampled_rows():
    """n = 4,000,000, d = 5, Cauchy l = 2, tol 1e-4, FP32, 16 columns: U would take about 1.4 TB,
    so hdf_build stores the matrix-free rows; 256 sampled rows of K~ V against exact K V."""
    import torch
    from paper_2202_03655_gb300 import hdf
    x = W.points("normal5_cauchy")
    n = x.shape[0]
    f = hdf.build(to_dev(x), "cauchy", 2.0, 1e-4, precision="fp32")
    assert f.info.matrix_free == 1
    assert f.info.ldu * n * 4 > 1e12
    V = W.rng(102).standard_normal((n, 16))
    Y = f.matvec(to_dev(V, torch.float32))
    rows = np.sort(W.rng(13).choice(n, 256, replace=False))
    got = Y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    exact = dense_rows_matvec_torch(x, "cauchy", 2.0, V, rows)
    err = rel(got, exact)
    print(f"normal5_cauchy 4M matrix-free: rank {f.rank}, sampled-row error {err:.3e}, "
          f"a-priori bound {f.info.err_bound:.3e}")
    assert err <= f.info.err_bound
