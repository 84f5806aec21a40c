"""Kernel ridge regression of Sec. 4.2 through the C ABI (hdf_kmeans, hdf_kernel_matvec,
hdf_krr_*) against the oracle of oracle/krr.py on the same seeded inputs."""
import numpy as np
import pytest

from gpu_common import rel, to_dev
from oracle import krr as okrr
from paper_2202_03655_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2202_03655_gb300 import hdf
    return hdf


def test_kmeans_matches_oracle():
    hdf = _lib()
    xtr, _, _, _, init = W.krr_data(n=3000)
    labels, C, it = hdf.kmeans(to_dev(xtr), init)
    lo, Co, ito = okrr.kmeans(xtr, init)
    assert it == ito
    assert np.array_equal(labels.cpu().numpy(), lo)
    assert np.allclose(C.cpu().numpy(), Co, rtol=0, atol=1e-13)


def test_kmeans_separated_blobs_and_single_cluster():
    hdf = _lib()
    g = np.random.default_rng(0)
    centres = g.uniform(-10, 10, size=(6, 5))
    x = np.concatenate([c + 0.3 * g.standard_normal((50, 5)) for c in centres])
    labels, _, _ = hdf.kmeans(to_dev(x), np.arange(6) * 50 + 3)
    assert np.array_equal(labels.cpu().numpy(), np.repeat(np.arange(6), 50))
    labels, C, it = hdf.kmeans(to_dev(x), [17])
    assert np.all(labels.cpu().numpy() == 0) and it == 2
    assert np.allclose(C.cpu().numpy()[0], x.mean(axis=0))


def test_kernel_matvec_vs_oracle():
    hdf = _lib()
    xtr, _, xte, _, _ = W.krr_data(n=3000)
    w = np.random.default_rng(1).standard_normal(len(xtr))
    for kname in ("gaussian", "cauchy", "matern32", "matern52"):
        out = hdf.kernel_matvec(to_dev(xte), to_dev(xtr), kname, 0.5, to_dev(w)).cpu().numpy()
        assert rel(out, okrr.kernel_matvec(xte, xtr, kname, 0.5, w)) <= 1e-5, kname


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_krr_operator_preconditioner_and_solve(prec):
    """(lambda I + K^) v and M r against the oracle's operator and preconditioner; PCG reaches
    rtol on the library's own operator; predictions agree with the oracle's PCG solution."""
    hdf = _lib()
    w_ = W.WORKLOADS["krr8_clusters"]
    ell, lam, tol = w_["ell"], w_["lam"], 1e-5
    xtr, ytr, xte, yte, init = W.krr_data(n=3000)
    lo, _, _ = okrr.kmeans(xtr, init)
    x = to_dev(xtr)
    labels, _, _ = hdf.kmeans(x, init)
    assert np.array_equal(labels.cpu().numpy(), lo)
    K = hdf.KRR(x, labels, "gaussian", ell, lam, tol, precision=prec)
    nc, rank, _ = K.info()
    op = okrr.BlockOperator(xtr, lo, "gaussian", ell, tol)
    assert nc == len(op.idx)
    assert abs(rank - sum(op.ranks)) <= 0.05 * sum(op.ranks) + 2 * nc
    v = np.random.default_rng(2).standard_normal(len(xtr))
    Av = K.apply(to_dev(v)).cpu().numpy()
    assert rel(Av, lam * v + op.apply(v)) <= (10 * tol if prec == "fp64" else 2e-5)
    M = okrr.block_preconditioner(op, lam)
    assert rel(K.precond(to_dev(v)).cpu().numpy(), M(v)) <= 1e-10
    w, it, res = K.solve(to_dev(ytr), rtol=1e-8, max_iter=3000)
    assert res <= 1e-8
    # the true residual follows the recurrence when the operator is linear to working
    # precision: FP64 blocks and the double-float direct product; FP32 blocks round their
    # input to FP32 (relative 6e-8, amplified by the condition number ~1e4)
    true_res = rel(K.apply(w).cpu().numpy(), ytr)
    assert true_res <= (1e-7 if prec == "fp64" else 1e-3)
    wo, ito, reso = okrr.pcg(lambda u: lam * u + op.apply(u), M, ytr, 1e-8, 3000)
    pr = hdf.kernel_matvec(to_dev(xte), x, "gaussian", ell, w).cpu().numpy()
    po = okrr.kernel_matvec(xte, xtr, "gaussian", ell, wo)
    assert rel(pr, po) <= 1e-3
    mse, mse_o = np.mean((pr - yte) ** 2), np.mean((po - yte) ** 2)
    assert abs(mse - mse_o) <= 1e-3 * mse_o


def test_krr_labels_with_gaps():
    """Unused labels are skipped: labels 0, 2, 4, ... give the operator of labels 0, 1, 2, ..."""
    import torch
    hdf = _lib()
    xtr, ytr, _, _, init = W.krr_data(n=1200)
    x = to_dev(xtr)
    labels, _, _ = hdf.kmeans(x, init)
    K1 = hdf.KRR(x, labels, "gaussian", 0.5, 0.1, 1e-4)
    K2 = hdf.KRR(x, labels * 2 + 1, "gaussian", 0.5, 0.1, 1e-4)
    v = to_dev(np.random.default_rng(3).standard_normal(len(xtr)))
    assert torch.equal(K1.apply(v), K2.apply(v))
