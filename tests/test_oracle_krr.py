"""Pins of the kernel-ridge-regression oracle (Sec. 4.2: k-means blocks, HDF diagonal blocks,
block-preconditioned CG) against facts fixed by mathematics (no GPU)."""
import numpy as np
import pytest

from oracle import hdf as ohdf
from oracle import krr
from paper_2202_03655_gb300 import workloads as W


def _blobs(seed=0, q=5, per=60, d=4):
    g = np.random.default_rng(seed)
    centres = g.uniform(-10, 10, size=(q, d))
    x = np.concatenate([c + 0.3 * g.standard_normal((per, d)) for c in centres])
    truth = np.repeat(np.arange(q), per)
    return x, truth


def test_kmeans_recovers_separated_blobs():
    x, truth = _blobs()
    init = np.arange(5) * 60 + 7                      # one starting point in every blob
    labels, C, it = krr.kmeans(x, init)
    assert np.array_equal(labels, truth)
    for c in range(5):
        assert np.allclose(C[c], x[truth == c].mean(axis=0))


def test_kmeans_fixed_point():
    """At convergence every centre is the mean of its points and every point is nearest its
    own centre (Lloyd's two steps leave the state unchanged)."""
    xtr, _, _, _, init = W.krr_data(n=1500)
    labels, C, it = krr.kmeans(xtr, init)
    d2 = ((xtr[:, None, :] - C[None]) ** 2).sum(-1)
    assert np.all(d2[np.arange(len(xtr)), labels] <= d2.min(axis=1) + 1e-12)
    for c in np.unique(labels):
        assert np.allclose(C[c], xtr[labels == c].mean(axis=0), atol=1e-14)


def test_pcg_matches_direct_solve():
    g = np.random.default_rng(1)
    A = g.standard_normal((80, 80))
    A = A @ A.T + 0.5 * np.eye(80)
    b = g.standard_normal(80)
    D = np.diag(A).copy()
    x, it, res = krr.pcg(lambda v: A @ v, lambda r: r / D, b, rtol=1e-12, max_iter=500)
    assert res <= 1e-12
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-9 * np.abs(x).max())
    # the exact preconditioner converges in one step
    Ainv = np.linalg.inv(A)
    x1, it1, _ = krr.pcg(lambda v: A @ v, lambda r: Ainv @ r, b, rtol=1e-10)
    assert it1 == 1 and np.allclose(x1, np.linalg.solve(A, b))


def test_block_operator_and_preconditioner():
    """K^ differs from K only inside the diagonal blocks, there by at most each block's HDF
    error; the preconditioner inverts lambda I + K_{C_i C_i} exactly."""
    xtr, ytr, _, _, init = W.krr_data(n=900)
    labels, _, _ = krr.kmeans(xtr, init)
    op = krr.BlockOperator(xtr, labels, "gaussian", 0.5, 1e-6)
    Kh = op.dense()
    E = Kh - op.K
    for i in op.idx:
        blk = E[np.ix_(i, i)]
        assert np.linalg.norm(blk) <= 1e-6 * np.linalg.norm(op.K[np.ix_(i, i)]) + 1e-14
        E[np.ix_(i, i)] = 0.0
    assert np.abs(E).max() == 0.0
    v = np.random.default_rng(2).standard_normal(len(xtr))
    assert np.allclose(op.apply(v), Kh @ v, rtol=0, atol=1e-12 * np.abs(Kh @ v).max())
    M = krr.block_preconditioner(op, 0.1)
    for i in op.idx[:5]:
        r = np.zeros(len(xtr))
        r[i] = np.random.default_rng(3).standard_normal(len(i))
        z = M(r)
        assert np.allclose((0.1 * np.eye(len(i)) + op.K[np.ix_(i, i)]) @ z[i], r[i], atol=1e-10)


def test_krr_fit_tends_to_dense_krr():
    """As the block tolerance falls, the PCG solution tends to the dense KRR solution of Eq. (opt)."""
    xtr, ytr, xte, yte, init = W.krr_data(n=900)
    labels, _, _ = krr.kmeans(xtr, init)
    lam = 0.1
    wd = np.linalg.solve(lam * np.eye(len(ytr)) + ohdf.dense_kernel(xtr, "gaussian", 0.5), ytr)
    errs = []
    for tol in (1e-2, 1e-5, 1e-8):
        w, it, res, op = krr.krr_fit(xtr, ytr, labels, "gaussian", 0.5, lam, tol, rtol=1e-10)
        assert res <= 1e-10
        pr = krr.kernel_matvec(xte, xtr, "gaussian", 0.5, w)
        pd = krr.kernel_matvec(xte, xtr, "gaussian", 0.5, wd)
        errs.append(np.linalg.norm(pr - pd) / np.linalg.norm(pd))
    assert errs[0] > errs[1] > errs[2] and errs[2] <= 1e-5


def test_kernel_matvec_is_the_dense_product():
    g = np.random.default_rng(4)
    x, xq, w = g.standard_normal((50, 3)), g.standard_normal((7, 3)), g.standard_normal(50)
    K = np.array([[np.exp(-0.5 * np.sum((a - b) ** 2) / 0.7 ** 2) for b in x] for a in xq])
    assert np.allclose(krr.kernel_matvec(xq, x, "gaussian", 0.7, w), K @ w)


def test_single_cluster_exact_preconditioner_converges_in_one_step():
    """One cluster: K^ is that block's HDF factor and M^-1 = lambda I + K exactly; with the block
    tolerance near rounding, M is the inverse of the system and PCG stops after one step."""
    g = np.random.default_rng(8)
    xtr = W.uniform_ball(g, 300, 3, 1.0)
    ytr = np.sin(3.0 * xtr[:, 0]) + 0.1 * g.standard_normal(300)
    labels = np.zeros(len(xtr), dtype=int)
    op = krr.BlockOperator(xtr, labels, "gaussian", 0.5, 1e-12)
    M = krr.block_preconditioner(op, 1.0)
    w, it, res = krr.pcg(lambda v: 1.0 * v + op.apply(v), M, ytr, rtol=1e-9, max_iter=50)
    assert it == 1 and res <= 1e-9
