"""Tensor-core (tcgen05, 3xTF32) matvec of FP32 factors against the CUDA-core path of the
same factor, and against the oracle."""
import numpy as np
import pytest

from gpu_common import rel, to_dev
from oracle import hdf as ohdf
from paper_2202_03655_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,n,kname,ell", [("ball3_gauss", 2000, "gaussian", 0.5),
                                              ("cube4_gauss", 20011, "gaussian", 0.8),
                                              ("normal5_cauchy", 3001, "cauchy", 2.0)])
@pytest.mark.parametrize("c", [9, 16, 37, 64, 70])
def test_tensor_core_matvec_matches_cuda_cores(name, n, kname, ell, c):
    import torch
    from paper_2202_03655_gb300 import hdf
    x = W.points(name, n=n)
    f_tc = hdf.build(to_dev(x), kname, ell, 1e-6, precision="fp32")
    f_cc = hdf.build(to_dev(x), kname, ell, 1e-6, precision="fp32", flags=hdf.FLAG_CUDA_CORES)
    V = np.random.default_rng(c).standard_normal((n, c)).astype(np.float32)
    Y_tc = f_tc.matvec(to_dev(V)).double().cpu().numpy()
    Y_cc = f_cc.matvec(to_dev(V)).double().cpu().numpy()
    assert f_tc.device_errors() == 0
    assert rel(Y_tc, Y_cc) <= 2e-6
    if n <= 3001:
        fo = ohdf.build(x, kname, ell, 1e-6)
        assert rel(Y_tc, ohdf.matvec(fo, V.astype(np.float64))) <= 1e-5


def test_tensor_core_solve_refinement():
    """The solve's refinement runs the matvec with a beta term (alpha U W + beta B)."""
    import torch
    from paper_2202_03655_gb300 import hdf
    x = W.points("ball3_gauss", n=1500)
    f = hdf.build(to_dev(x), "gaussian", 0.5, 1e-5, precision="fp32")
    fo = ohdf.build(x, "gaussian", 0.5, 1e-5)
    B = np.random.default_rng(9).standard_normal((1500, 20))
    X = f.solve(1e-2, to_dev(B, torch.float32), refine_steps=1).double().cpu().numpy()
    assert f.device_errors() == 0
    assert rel(X, ohdf.solve(fo, 1e-2, B)) <= 2e-3
