"""hdf_solve at the benchmark's rank (about 10,000 padded columns): the Woodbury core
lambda S^-1 + U^T U, indefinite because S has eigenvalues of both signs, factored by the
blocked LU with partial pivoting (host panels, device updates) and solved on the device.

The exact solution of (lambda I + K~) X = B is not available at this size, so the check is
the residual |lambda X + K~ X - B| / |B| (through the library's own product), FP64 against
FP32, and the repeat solve (cached factors) against the first.
"""
import numpy as np
import pytest

from gpu_common import rel, to_dev
from paper_2202_03655_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_solve_at_benchmark_rank():
    import torch
    from paper_2202_03655_gb300 import hdf
    n = 30000
    x = W.points("mixture3_matern", n=n)
    lam = 1e-4 * n
    B = np.random.default_rng(21).standard_normal((n, 2))
    out = {}
    for prec, dt, bound in (("fp64", torch.float64, 1e-9), ("fp32", torch.float32, 1e-4)):
        f = hdf.build(to_dev(x), "matern32", 1.0, 1e-8, precision=prec, p_max=64)
        assert f.info.ldu > 4096
        Bt = to_dev(B, dt)
        X = f.solve(lam, Bt, refine_steps=1)
        res = lam * X.double() + f.matvec(X).double() - Bt.double()
        r = float(torch.linalg.norm(res) / torch.linalg.norm(Bt.double()))
        print(f"solve {prec}: ldu {f.info.ldu}, U^T U {f.info.t_ms[6]:.1f} ms, LU {f.info.lu_ms:.1f} ms, "
              f"residual {r:.2e}")
        assert r <= bound
        X2 = f.solve(lam, Bt, refine_steps=1)
        assert rel(X2.double().cpu().numpy(), X.double().cpu().numpy()) <= (1e-12 if prec == "fp64" else 1e-5)
        out[prec] = X.double().cpu().numpy()
        del f
    assert rel(out["fp32"], out["fp64"]) <= 1e-3
