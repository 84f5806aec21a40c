"""Tensor-core (tcgen05, 3xTF32 with per-stage promotion) matvec of FP32 factors against the
CUDA-core path of the same factor and against an FP64 product of the exported U and S."""
import functools

import numpy as np
import pytest

from gpu_common import rel, to_dev
from oracle import hdf as ohdf
from paper_2202_03655_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = {"ball3": ("ball3_gauss", 2000, "gaussian", 0.5),
         "cube4": ("cube4_gauss", 20011, "gaussian", 0.8),
         "normal5": ("normal5_cauchy", 3001, "cauchy", 2.0)}


@functools.lru_cache(maxsize=None)
def _factors(case):
    from paper_2202_03655_gb300 import hdf
    name, n, kname, ell = CASES[case]
    x = W.points(name, n=n)
    f_tc = hdf.build(to_dev(x), kname, ell, 1e-6, precision="fp32")
    f_cc = hdf.build(to_dev(x), kname, ell, 1e-6, precision="fp32", flags=hdf.FLAG_CUDA_CORES)
    U, S = f_tc.export()
    return x, f_tc, f_cc, U.astype(np.float64), S


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("c", [1, 2, 5, 8, 9, 16, 37, 64, 70])
def test_tensor_core_matvec(case, c):
    x, f_tc, f_cc, U, S = _factors(case)
    n = x.shape[0]
    V = np.random.default_rng(c).standard_normal((n, c)).astype(np.float32)
    Y_tc = f_tc.matvec(to_dev(V)).double().cpu().numpy()
    Y_cc = f_cc.matvec(to_dev(V)).double().cpu().numpy()
    assert f_tc.device_errors() == 0
    exact = U @ (S[:, None] * (U.T @ V.astype(np.float64)))       # same U, FP64 products
    # FP32 rounding of the two GEMMs, amplified by cancellation in U (S U^T V): a few 1e-7 to
    # a few 1e-6; both paths share the bound
    assert rel(Y_tc, exact) <= 1e-5
    assert rel(Y_cc, exact) <= 1e-5
    assert rel(Y_tc, exact) <= 2 * rel(Y_cc, exact) + 1e-6


def test_tensor_core_vs_oracle():
    x, f_tc, _, _, _ = _factors("ball3")
    fo = ohdf.build(x, "gaussian", 0.5, 1e-6)
    V = np.random.default_rng(1).standard_normal((x.shape[0], 24))
    Y = f_tc.matvec(to_dev(V.astype(np.float32))).double().cpu().numpy()
    assert rel(Y, ohdf.matvec(fo, V)) <= 1e-5


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


@pytest.mark.parametrize("case", ["ball3", "cube4"])
def test_tensor_core_gram_solve(case):
    """hdf_solve with U^T U on the tensor cores (FP32 factors) against the same solve with the
    CUDA-core Gram, and the residual of (lam I + K~) X = B through the factor."""
    import torch
    x, f_tc, f_cc, U, S = _factors(case)
    n = x.shape[0]
    lam = 1e-2
    B = np.random.default_rng(17).standard_normal((n, 3)).astype(np.float32)
    X_tc = f_tc.solve(lam, to_dev(B), refine_steps=1).double().cpu().numpy()
    X_cc = f_cc.solve(lam, to_dev(B), refine_steps=1).double().cpu().numpy()
    assert f_tc.device_errors() == 0
    assert rel(X_tc, X_cc) <= 1e-4
    # the FP32 residual is bounded by the conditioning of lam I + K~ (X is ~ B / lam in the
    # directions K~ does not reach); the tensor-core Gram must not make it worse
    Bd = B.astype(np.float64)
    res = lambda X: rel(lam * X + U @ (S[:, None] * (U.T @ X)), Bd)
    assert res(X_tc) <= 2 * res(X_cc) + 1e-6
    assert res(X_tc) <= 1e-2


def test_tf32_operand_rounding_matches_conversion_instruction():
    """The 3xTF32 split rounds each FP32 operand to TF32 (nearest, ties away from zero) with
    integer operations on its bit pattern; over all 2^32 bit patterns it must equal the device's
    cvt.rna.tf32.f32 on every finite value, including the top binade where rounding overflows."""
    from paper_2202_03655_gb300 import hdf
    assert hdf.check_tf32_rounding() == (0, 0)
