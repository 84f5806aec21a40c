"""hdf_matvec_noalloc against hdf_matvec.

The no-allocation entry point exists for callers that cannot obtain device memory during
the call -- code under another allocator's pool, or loops that reserve everything at
start-up.  It must give the same K~ V as hdf_matvec (work space in the library's fixed
array), including on a second call that reuses the array left over from the first, and it
must refuse exactly the requests whose work space exceeds that array.  This file is named
to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-6), ("fp32", 1e-5)])
def test_noalloc_matches_matvec_twice(prec, tol):
    import torch
    from paper_2202_03655_gb300 import hdf, workloads as W
    x = W.points("ball3_gauss", n=3000)
    f = hdf.build(torch.from_numpy(x).cuda(), "gaussian", 0.5, 1e-6, precision=prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    n = x.shape[0]
    for ncols, seed in ((5, 1), (70, 2)):              # second call: new shapes, same array
        V = torch.from_numpy(np.random.default_rng(seed).standard_normal((ncols, n))).to("cuda", dt)
        Y_ref = torch.empty_like(V)
        Y_new = torch.full_like(V, float("nan"))
        f.matvec_ptr(V.data_ptr(), n, ncols, Y_ref.data_ptr(), n)
        f.matvec_noalloc_ptr(V.data_ptr(), n, ncols, Y_new.data_ptr(), n)
        torch.cuda.synchronize()
        a, b = Y_new.double().cpu().numpy(), Y_ref.double().cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= tol


def test_noalloc_size_limit_boundary():
    """The limit is ldu * min(ncols, 64) * (8 + element size) <= 32 MiB.  A factor with a padded
    width between 2^15 and 2^21 (FP64: 16 bytes per entry and column) has a largest admissible
    column count c_max in 1..63: c_max columns run and match hdf_matvec, c_max + 1 columns
    return HDF_ETOOBIG.  (5,000 points in d = 5 scaled to maximum norm 1, Matern-3/2 with l = 1 at
    tol 1e-4: the degree is capped and the rank is of order 10^5.)"""
    import torch
    from paper_2202_03655_gb300 import hdf, workloads as W
    x = W.maxnorm1_points("fig3_rank5", 5000, 5)
    f = hdf.build(torch.from_numpy(x).cuda(), "matern32", 1.0, 1e-4, precision="fp64")
    n, ldu = x.shape[0], f.info.ldu
    cmax = (32 << 20) // (ldu * 16)
    assert 1 <= cmax < 64, (ldu, cmax)      # the case must exercise the boundary, never skip it
    g = np.random.default_rng(5)
    V = torch.from_numpy(g.standard_normal((cmax + 1, n))).cuda()
    Y_ref = torch.empty_like(V)
    Y_new = torch.full_like(V, float("nan"))
    f.matvec_ptr(V.data_ptr(), n, cmax, Y_ref.data_ptr(), n)
    f.matvec_noalloc_ptr(V.data_ptr(), n, cmax, Y_new.data_ptr(), n)
    torch.cuda.synchronize()
    a, b = Y_new[:cmax].cpu().numpy(), Y_ref[:cmax].cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-10
    Y_keep = torch.full_like(V, 7.0)
    with pytest.raises(hdf.HdfError) as ei:
        f.matvec_noalloc_ptr(V.data_ptr(), n, cmax + 1, Y_keep.data_ptr(), n)
    assert ei.value.status == 8
    torch.cuda.synchronize()
    assert bool((Y_keep == 7.0).all())        # outputs untouched on error
