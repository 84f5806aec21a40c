"""Kernel ridge regression with HDF-compressed diagonal blocks and preconditioned CG (Sec. 4.2
of Ryan & Damle), plain FP64 numpy.

Test infrastructure (like the rest of ``oracle``): only the tests, the smoke check and the
CPU-baseline leg of the benchmark use it.

The system is Eq. (opt): (lambda I + K) w = y, predictions y* = K(x*, x) w.  Sec. 4.2 builds the
operator from k-means clusters C_1..C_q of the training points: the diagonal blocks K_{C_i C_i}
are replaced by their HDF factors, the off-diagonal blocks are kept exact, and the system with
that operator K^ is solved by conjugate gradients, preconditioned by the block-diagonal matrix
whose blocks are the inverses of the exact blocks (lambda I + K_{C_i C_i}).

Steps here, in that order:
1. ``kmeans``: Lloyd's iteration from given initial centres (the random choice of the centres is
   an input): assign every point to its nearest centre (lowest index on ties), move each centre
   to the mean of its points (a centre with no points stays), until no assignment changes.
2. ``BlockOperator``: K^ v = sum_i K~_i v_{C_i} + sum_{i != j} K_{C_i C_j} v_{C_j}, K~_i the
   symmetric HDF factor of cluster i (``oracle.hdf.build``).
3. ``block_preconditioner``: the inverses of lambda I + K_{C_i C_i} (exact kernel).
4. ``pcg``: textbook preconditioned conjugate gradients (Hestenes-Stiefel), x_0 = 0, stopped when
   |y - (lambda I + K^) x| <= rtol |y| or after max_iter steps.
"""
import numpy as np

from . import hdf as ohdf


def kmeans(x, init_idx, max_iter=100):
    """(labels, centres, iterations) of Lloyd's iteration from the centres x[init_idx]."""
    x = np.asarray(x, dtype=np.float64)
    C = x[np.asarray(init_idx)].copy()
    labels = None
    it = 0
    for it in range(1, max_iter + 1):
        d2 = ((x[:, None, :] - C[None, :, :]) ** 2).sum(axis=-1)
        new = np.argmin(d2, axis=1)                  # first minimum: lowest index on ties
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        for c in range(C.shape[0]):
            m = labels == c
            if m.any():
                C[c] = x[m].mean(axis=0)
    return labels, C, it


class BlockOperator:
    """K^ = block-diagonal HDF factors + exact off-diagonal blocks, over clusters of x."""

    def __init__(self, x, labels, kname, ell, tol, p_max=ohdf.P_MAX_DEFAULT):
        self.x = np.asarray(x, dtype=np.float64)
        self.labels = np.asarray(labels)
        self.kname, self.ell = kname, float(ell)
        self.idx = [np.flatnonzero(self.labels == c) for c in range(int(self.labels.max()) + 1)]
        self.idx = [i for i in self.idx if len(i)]
        self.factors = [ohdf.build(self.x[i], kname, ell, tol, p_max=p_max) for i in self.idx]
        self.K = ohdf.dense_kernel(self.x, kname, ell)
        self.Koff = self.K.copy()
        for i in self.idx:
            self.Koff[np.ix_(i, i)] = 0.0

    @property
    def ranks(self):
        return [f.rank for f in self.factors]

    def apply(self, v):
        v = np.asarray(v, dtype=np.float64)
        out = self.Koff @ v
        for i, f in zip(self.idx, self.factors):
            out[i] += ohdf.matvec(f, v[i])
        return out

    def dense(self):
        """K^ as a dense matrix (for checks on small problems)."""
        M = self.Koff.copy()
        for i, f in zip(self.idx, self.factors):
            M[np.ix_(i, i)] = (f.U * f.S) @ f.U.T
        return M


def block_preconditioner(op, lam):
    """Per cluster the inverse of lambda I + K_{C_i C_i} (exact kernel); returns apply(r)."""
    inv = [np.linalg.inv(lam * np.eye(len(i)) + op.K[np.ix_(i, i)]) for i in op.idx]

    def apply(r):
        z = np.empty_like(r)
        for i, B in zip(op.idx, inv):
            z[i] = B @ r[i]
        return z
    return apply


def pcg(apply_A, apply_M, b, rtol=1e-8, max_iter=1000):
    """Preconditioned CG for symmetric positive definite A from x_0 = 0.
    Returns (x, iterations, relative residual |b - A x| / |b| of the recurrence)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_M(r)
    p = z.copy()
    rz = float(r @ z)
    nb = float(np.linalg.norm(b))
    if nb == 0.0:
        return x, 0, 0.0
    it = 0
    res = 1.0
    for it in range(1, max_iter + 1):
        Ap = apply_A(p)
        alpha = rz / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        res = float(np.linalg.norm(r)) / nb
        if res <= rtol:
            break
        z = apply_M(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, res


def krr_fit(x, y, labels, kname, ell, lam, tol, rtol=1e-8, max_iter=1000):
    """w of (lambda I + K^) w = y by PCG with the block preconditioner; returns (w, iters, res, op)."""
    op = BlockOperator(x, labels, kname, ell, tol)
    M = block_preconditioner(op, lam)
    w, it, res = pcg(lambda v: lam * v + op.apply(v), M, y, rtol, max_iter)
    return w, it, res, op


def kernel_matvec(xq, x, kname, ell, w):
    """K(x*, x) w with the exact kernel (the predictions of Sec. 4.2)."""
    diff = np.asarray(xq, dtype=np.float64)[:, None, :] - np.asarray(x, dtype=np.float64)[None, :, :]
    return ohdf.kernel(kname, np.sqrt((diff * diff).sum(axis=-1)), ell) @ np.asarray(w, dtype=np.float64)
