"""Batched factorization (hdf_build_batched / hdf_batch_matvec) against per-set oracle builds
and against hdf_build on the same sets."""
import numpy as np
import pytest

from gpu_common import dense_rows_matvec_torch, rel, to_dev
from oracle import hdf as ohdf
from paper_2202_03655_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ragged(seed, sizes):
    g = np.random.default_rng(seed)
    xs = [W.uniform_ball(g, m, 3, r) for m, r in zip(sizes, g.uniform(0.5, 2.0, len(sizes)))]
    ells = g.uniform(0.3, 1.5, len(sizes))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(xs, axis=0), off, ells


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_oracle_and_single_builds(prec):
    import torch
    from paper_2202_03655_gb300 import hdf
    sizes = [1, 33, 700, 2500, 64, 1800, 7]
    x, off, ells = _ragged(11, sizes)
    tol = 1e-6
    b = hdf.build_batched(to_dev(x), off, "gaussian", ells, tol, precision=prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    V = np.random.default_rng(2).standard_normal((off[-1], 3))
    Y = b.matvec(to_dev(V, dt)).double().cpu().numpy()
    Y2 = b.matvec(to_dev(V, dt)).double().cpu().numpy()          # graph replay path
    assert np.array_equal(Y.shape, Y2.shape)
    for s in range(len(sizes)):
        xs, Vs = x[off[s]:off[s + 1]], V[off[s]:off[s + 1]]
        fo = ohdf.build(xs, "gaussian", ells[s], tol)
        assert b.info(s).p == fo.plan.p
        Yo = ohdf.matvec(fo, Vs)
        assert rel(Y[off[s]:off[s + 1]], Yo) <= 10 * tol, s
        f1 = hdf.build(to_dev(xs), "gaussian", ells[s], tol, precision=prec)
        Y1 = f1.matvec(to_dev(Vs, dt)).double().cpu().numpy()
        assert rel(Y[off[s]:off[s + 1]], Y1) <= (1e-9 if prec == "fp64" else 1e-5), s


def test_batch512_full_size_sampled():
    """512 sets, n log-uniform in [1000, 65536], uniform balls of radius U[0.5, 2], Gaussian
    l ~ U[0.3, 1.5], tol 1e-6, FP32, 8 columns: sampled rows of sampled sets against the
    exact kernel."""
    import torch
    from paper_2202_03655_gb300 import hdf
    x, off, ells = W.batch_sets(W.rng(4))
    b = hdf.build_batched(to_dev(x), off, "gaussian", ells, 1e-6, precision="fp32")
    V = np.random.default_rng(8).standard_normal((off[-1], 8)).astype(np.float32)
    Y = b.matvec(to_dev(V)).double().cpu().numpy()
    g = np.random.default_rng(5)
    for s in g.choice(len(ells), 12, replace=False):
        I = b.info(s)
        xs, Vs = x[off[s]:off[s + 1]], V[off[s]:off[s + 1]].astype(np.float64)
        rows = np.sort(g.choice(I.n, min(64, I.n), replace=False))
        exact = dense_rows_matvec_torch(xs, "gaussian", ells[s], Vs, rows)
        err = rel(Y[off[s]:off[s + 1]][rows], exact)
        assert err <= (1e-5 if I.reached else 10 * I.err_bound + 1e-5), (s, err, I.p, I.reached)


@pytest.mark.parametrize("c", [1, 2, 5, 8, 13, 16, 20])
def test_batch_matvec_column_counts(c):
    """FP32 batched K~V for every column-tile width (the streaming kernels for c <= 16, U W with
    bulk copies of 32-row tiles and ragged last tiles of 3, 900 - 896 and 131 - 128 rows; the
    register-tiled ones above) against hdf_build + hdf_matvec on the same sets."""
    import torch
    from paper_2202_03655_gb300 import hdf
    sizes = [3, 900, 131, 2049]
    x, off, ells = _ragged(23, sizes)
    tol = 1e-6
    b = hdf.build_batched(to_dev(x), off, "gaussian", ells, tol, precision="fp32")
    V = np.random.default_rng(c).standard_normal((off[-1], c)).astype(np.float32)
    Y = b.matvec(to_dev(V, torch.float32)).double().cpu().numpy().reshape(off[-1], c)
    Y2 = b.matvec(to_dev(V, torch.float32)).double().cpu().numpy().reshape(off[-1], c)
    assert np.array_equal(Y, Y2)                                   # deterministic replay
    assert b.device_errors() == 0                                  # no bounded wait ran out
    for s in range(len(sizes)):
        xs, Vs = x[off[s]:off[s + 1]], V[off[s]:off[s + 1]]
        f1 = hdf.build(to_dev(xs), "gaussian", ells[s], tol, precision="fp32")
        Y1 = f1.matvec(to_dev(Vs, torch.float32)).double().cpu().numpy().reshape(-1, c)
        assert rel(Y[off[s]:off[s + 1]], Y1) <= 1e-5, (s, c)
