"""Adjoint of f = w^T K~ v (frozen-structure semantics) through the C ABI.

Checked against the oracle's central differences (Richardson-extrapolated, base step
h = 1e-4, FP64) of its own frozen-structure evaluator, against the gradient of the exact
kernel matrix, and through the torch.autograd wrapper.
"""
import numpy as np
import pytest

from gpu_common import rel, to_dev
from oracle import hdf as ohdf
from paper_2202_03655_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _build(x, kname, ell, tol, prec, p_max=None):
    from paper_2202_03655_gb300 import hdf
    return hdf.build(to_dev(x), kname, ell, tol, precision=prec, p_max=p_max)


@pytest.mark.parametrize("d,kname,ell,n,p_max", [(4, "gaussian", 0.8, 120, 64), (3, "cauchy", 0.7, 120, 64),
                                                (5, "gaussian", 2.0, 200, 64), (3, "matern52", 1.0, 400, 32)])
def test_adjoint_vs_oracle_fd(d, kname, ell, n, p_max):
    """The frozen radial functions agree between the two sides at the data points; between
    them (and so in their derivatives) they agree only where the radial basis is well
    conditioned on the data, so the cases keep n well above the basis size p/2 + 1.  At a
    loose tol the two sides may also keep different eigenpairs near the budget boundary; at
    1e-9 both keep the same set."""
    import torch
    g = np.random.default_rng(20 + d)
    x = W.uniform_cube(g, n, d)
    v, w = g.standard_normal(n), g.standard_normal(n)
    tol = 1e-9
    f = _build(x, kname, ell, tol, "fp64", p_max)
    G, dl, val = f.adjoint(to_dev(x), to_dev(v), to_dev(w))
    fo = ohdf.build(x, kname, ell, tol, p_max=p_max)
    assert f.info.p == fo.plan.p
    Go, dlo = ohdf.adjoint_fd(fo, x, v, w)
    vo = float(w @ ohdf.matvec(fo, v))
    # The value f = w^T K~ v: both sides build the same degree and apply the same truncation
    # rule, so their K~ differ only by eigenpairs kept on one side and dropped on the other at
    # the budget boundary.  The dropped pairs of either side cost at most eta tol |K|_F / 2 in
    # Frobenius norm (eta = 1), so |K~_gpu - K~_orc|_F <= tol |K|_F and
    # |w^T (K~_gpu - K~_orc) v| <= tol |K|_F |v| |w|, with |K|_F = n sqrt(mu2).
    normK = n * np.sqrt(fo.plan.mu2)
    assert abs(val - vo) <= tol * normK * np.linalg.norm(v) * np.linalg.norm(w) + 1e-12 * abs(vo)
    # the derivatives of the frozen function, by central differences on the oracle's side
    gtol = max(1e-5, 100 * tol)
    assert rel(G.cpu().numpy(), Go) <= gtol
    assert abs(dl - dlo) <= gtol * abs(dlo)


def test_adjoint_fp32_and_multicolumn():
    """FP32 bulk, and two columns = the sum of the single-column adjoints."""
    import torch
    g = np.random.default_rng(3)
    x = W.uniform_cube(g, 400, 4)
    V, Wm = g.standard_normal((400, 2)), g.standard_normal((400, 2))
    f64 = _build(x, "gaussian", 0.8, 1e-7, "fp64")
    f32 = _build(x, "gaussian", 0.8, 1e-7, "fp32")
    G2, dl2, v2 = f64.adjoint(to_dev(x), to_dev(V), to_dev(Wm))
    Ga, dla, va = f64.adjoint(to_dev(x), to_dev(V[:, 0]), to_dev(Wm[:, 0]))
    Gb, dlb, vb = f64.adjoint(to_dev(x), to_dev(V[:, 1]), to_dev(Wm[:, 1]))
    assert rel(G2.cpu().numpy(), (Ga + Gb).cpu().numpy()) <= 1e-12
    assert abs(dl2 - (dla + dlb)) <= 1e-10 * abs(dl2)
    G32, dl32, _ = f32.adjoint(to_dev(x), to_dev(V[:, 0], torch.float32), to_dev(Wm[:, 0], torch.float32))
    assert rel(G32.double().cpu().numpy(), Ga.cpu().numpy()) <= 1e-3
    assert abs(dl32 - dla) <= 1e-3 * abs(dla)


def test_autograd_function():
    import torch
    from paper_2202_03655_gb300.autograd import kernel_matvec
    g = np.random.default_rng(4)
    x = to_dev(W.uniform_cube(g, 300, 4)).requires_grad_(True)
    ell = torch.tensor(0.8, dtype=torch.float64, requires_grad=True)
    v = to_dev(g.standard_normal(300)).requires_grad_(True)
    w = to_dev(g.standard_normal(300))
    y = kernel_matvec(x, ell, v, "gaussian", 1e-8)
    (w * y).sum().backward()
    from paper_2202_03655_gb300 import hdf
    f = hdf.build(x.detach(), "gaussian", 0.8, 1e-8)
    G, dl, _ = f.adjoint(x.detach(), v.detach(), w)
    assert rel(x.grad.cpu().numpy(), G.cpu().numpy()) <= 1e-12
    assert abs(ell.grad.item() - dl) <= 1e-12 * abs(dl)
    assert rel(v.grad.cpu().numpy(), f.matvec(w).cpu().numpy()) <= 1e-12


def test_cube4_full_size_vs_dense_gradient():
    """500,000 points in [-1,1]^4, Gaussian l = 0.8, tol 1e-6, FP32: the adjoint against the
    exact kernel's gradient on 256 sampled points (plain torch FP64 rows), and d/dl against
    a 4,000-point dense check.  Derivatives amplify approximation error; the bound is loose."""
    import torch
    from paper_2202_03655_gb300 import hdf
    x = W.points("cube4_gauss")
    n = x.shape[0]
    v = W.rng(103).standard_normal(n)
    w = W.rng(104).standard_normal(n)
    xt = to_dev(x)
    f = hdf.build(xt, "gaussian", 0.8, 1e-6, precision="fp32")
    G, dl, val = f.adjoint(xt, to_dev(v, torch.float32), to_dev(w, torch.float32))
    G = G.double().cpu().numpy()
    rows = np.sort(W.rng(9).choice(n, 256, replace=False))
    vt, wt = to_dev(v), to_dev(w)
    ref = []
    for i in rows:
        diff = xt[i][None, :] - xt                         # (n, d)
        r = torch.sqrt((diff * diff).sum(1))
        kp = -(r / 0.8 ** 2) * torch.exp(-0.5 * (r / 0.8) ** 2)     # dk/dr
        coef = torch.where(r > 0, kp / torch.where(r > 0, r, torch.ones_like(r)), torch.zeros_like(r))
        m = coef * (wt[i] * vt + wt * vt[i])
        ref.append((m[:, None] * diff).sum(0).cpu().numpy())
    ref = np.array(ref)
    err = np.linalg.norm(G[rows] - ref) / np.linalg.norm(ref)
    assert err <= 5e-3, err
    del f
