"""Failure detection through the C ABI, without faulting the GPU.

* Non-finite points: every build entry point returns HDF_ENOTFINITE and no factor.
* A tolerance the degree cap cannot reach: HDF_ETOL_UNREACHABLE with a usable factor and
  info.reached == 0.
* Allocation failure, injected on the host (hdf_debug_fail_alloc): the call that meets it
  returns HDF_ENOMEM, hands back no factor and leaves its output buffers untouched; the library
  keeps working afterwards.
* A bounded device wait that runs out: the tensor-core kernels' work-wait limit is set to a few
  hundred clock cycles (hdf_set_wait_limit), far below the latency of a TMA copy, so their
  waits give up; each kernel then records the error, lets its own copies and MMAs finish, frees
  its tensor memory and returns.  The matvec reports it through hdf_device_errors, the solve
  returns HDF_ETIMEOUT, and with the default limit restored the same factor gives correct
  results again.
"""
import numpy as np
import pytest

from gpu_common import rel, to_dev
from paper_2202_03655_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ENOMEM, ENOTFINITE, ETOL_UNREACHABLE, ETIMEOUT = 2, 5, 4, 7


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_points(bad):
    import torch
    from paper_2202_03655_gb300 import hdf
    x = W.points("ball3_gauss", n=500).copy()
    x[137, 1] = bad
    with pytest.raises(hdf.HdfError) as ei:
        hdf.build(to_dev(x), "gaussian", 0.5, 1e-6)
    assert ei.value.status == ENOTFINITE
    y = W.points("ball3_gauss", n=300)
    with pytest.raises(hdf.HdfError) as ei:
        hdf.build_cross(to_dev(x), to_dev(y), "gaussian", 0.5, 1e-6)
    assert ei.value.status == ENOTFINITE
    with pytest.raises(hdf.HdfError) as ei:
        hdf.build_batched(to_dev(x), [0, 200, 500], "gaussian", [0.5, 0.7], 1e-6)
    assert ei.value.status == ENOTFINITE
    # the library still works
    f = hdf.build(to_dev(W.points("ball3_gauss", n=500)), "gaussian", 0.5, 1e-6)
    assert f.status == hdf.HDF_OK


def test_tolerance_unreachable_status():
    from paper_2202_03655_gb300 import hdf
    x = W.points("mixture3_matern", n=4000)
    f = hdf.build(to_dev(x), "matern32", 1.0, 1e-8, p_max=16)
    assert f.status == ETOL_UNREACHABLE
    assert f.info.reached == 0 and f.info.p == 16
    assert f.info.cheb_tail > f.info.tail_budget
    v = np.random.default_rng(1).standard_normal(4000)
    assert np.isfinite(f.matvec(to_dev(v)).cpu().numpy()).all()


def test_injected_allocation_failures():
    import torch
    from paper_2202_03655_gb300 import hdf
    x = W.points("cube4_gauss", n=3000)
    xt = to_dev(x)
    failed = 0
    try:
        # every allocation of the build in turn (a build makes a few dozen)
        for k in range(200):
            hdf.debug_fail_alloc(k)
            try:
                f = hdf.build(xt, "gaussian", 0.8, 1e-6, precision="fp32")
            except hdf.HdfError as e:
                assert e.status == ENOMEM, (k, str(e))
                failed += 1
                continue
            hdf.debug_fail_alloc(-1)
            break                           # k passed the build's last allocation
        else:
            pytest.fail("the build made more than 200 allocations")
        assert failed >= 5
        # the product: its first allocation fails, the output block keeps its contents
        V = to_dev(np.random.default_rng(2).standard_normal((3000, 16)), torch.float32)
        Vc = V.t().contiguous()
        Yc = torch.full_like(Vc, 3.0)
        hdf.debug_fail_alloc(0)
        with pytest.raises(hdf.HdfError) as ei:
            f.matvec_ptr(Vc.data_ptr(), 3000, 16, Yc.data_ptr(), 3000)
        assert ei.value.status == ENOMEM
        torch.cuda.synchronize()
        assert bool((Yc == 3.0).all())
    finally:
        hdf.debug_fail_alloc(-1)
    # afterwards everything works and agrees with a fresh factor
    g = hdf.build(xt, "gaussian", 0.8, 1e-6, precision="fp32")
    assert rel(f.matvec(V).double().cpu().numpy(), g.matvec(V).double().cpu().numpy()) <= 1e-6


def test_wait_timeout_is_reported_and_recoverable():
    import torch
    from paper_2202_03655_gb300 import hdf
    x = W.points("cube4_gauss", n=20011)
    f = hdf.build(to_dev(x), "gaussian", 0.8, 1e-6, precision="fp32")
    ref = hdf.build(to_dev(x), "gaussian", 0.8, 1e-6, precision="fp32", flags=hdf.FLAG_CUDA_CORES)
    V = to_dev(np.random.default_rng(3).standard_normal((x.shape[0], 16)), torch.float32)
    Y_ref = ref.matvec(V).double().cpu().numpy()
    assert f.device_errors() == 0
    prev = hdf.set_wait_limit(300)
    try:
        assert prev == 4000000000
        f.matvec(V)                                   # asynchronous: the error is in the flag
        assert f.device_errors() == 1
        assert f.device_errors() == 0                 # reading clears it
        B = to_dev(np.random.default_rng(4).standard_normal(x.shape[0]), torch.float32)
        with pytest.raises(hdf.HdfError) as ei:       # the solve's U^T U on the tensor cores
            f.solve(50.0, B, refine_steps=0)
        assert ei.value.status == ETIMEOUT
    finally:
        hdf.set_wait_limit(0)
    assert hdf.set_wait_limit(0) == 4000000000
    # the context and the factor are usable: the same product is right again
    Y = f.matvec(V).double().cpu().numpy()
    assert f.device_errors() == 0
    assert rel(Y, Y_ref) <= 1e-5
    X = f.solve(50.0, B, refine_steps=1)
    assert f.device_errors() == 0
    assert np.isfinite(X.cpu().numpy()).all()
