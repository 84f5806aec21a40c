"""hdf_matvec_noalloc against hdf_matvec.

The no-allocation entry point exists for callers that cannot obtain device memory during
the call -- inside a stream capture, under another allocator's pool, or in loops that
reserve everything at start-up.  It must give the same K~ V as hdf_matvec (same kernels,
work space in the library's fixed array), including on a second call that reuses the
array left over from the first.  This file is named to be collected last.
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


def test_noalloc_rejects_oversized_request():
    import torch
    from paper_2202_03655_gb300 import hdf, workloads as W
    x = W.points("cube4_gauss", n=4000)
    f = hdf.build(torch.from_numpy(x).cuda(), "gaussian", 0.3, 1e-8, precision="fp64")
    n = x.shape[0]
    if f.rank * 64 * 16 <= 32 << 20:
        pytest.skip("factor rank too small to exceed the fixed work space")
    V = torch.zeros(64, n, device="cuda", dtype=torch.float64)
    Y = torch.zeros_like(V)
    with pytest.raises(hdf.HdfError) as ei:
        f.matvec_noalloc_ptr(V.data_ptr(), n, 64, Y.data_ptr(), n)
    assert ei.value.status == 8
