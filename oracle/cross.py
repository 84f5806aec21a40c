"""Algorithm 1 of Ryan & Damle in its general form, K(X, Y) ~= U diag(S) V^T, plain FP64 numpy.

Test infrastructure (like the rest of ``oracle``): only the tests, the smoke check and the
CPU-baseline leg of the benchmark use it.

Steps, in the paper's order, for two point sets X (m points) and Y (n points):

1. Scale both sets with one map (Sec. 3.3: the expansion needs |x - y| <= 1 for every pair):
   c = mean of the union, R = max distance of a point of either set from c,
   x' = (x - c) / (2R), y' = (y - c) / (2R).
2. Chebyshev coefficients and degree (ChebDegreeNeeded, Remark 3) as in the symmetric case,
   with mu2 = mean_{ij} k(x_i, y_j)^2 over the cross pairs, so that the entrywise Chebyshev
   error sums to at most tol |K_XY|_F / 2 in Frobenius norm (|K_XY|_F = sqrt(m n mu2)).
3. Radial cores r^(k) (Eq. rdef) in the stable basis (``radial.stable_core``).  The core is
   the same matrix on both sides: r^(k)(|x|, |y|) depends on the two radii symmetrically.
4. Two QRs per parity (Eq. svd): B_par(rho_X) = Q_X R_X and B_par(rho_Y) = Q_Y R_Y.
5. SVD of R_X Gamma_k R_Y^T = W_X Sigma W_Y^T (Eq. svd, truncsvd).
6. Truncation (Sec. 3.4-3.5): dropping the singular triple (sigma, w_X, w_Y) of block k
   changes K_XY by at most sigma |H_k| / |S^{d-1}| in Frobenius norm -- by Cauchy-Schwarz on
   the addition theorem, |sum_h Y_k^h(a) Y_k^h(b)| <= |H_k| / |S^{d-1}| for unit a, b, and
   Q_X w_X, Q_Y w_Y are unit vectors.  Triples are dropped globally in increasing order of that
   cost while the summed cost stays <= eta tol |K_XY|_F / 2 (the symmetric rule with sigma in
   place of |lambda|).
7. Assemble U[:, (k, s, h)] = (Q_X W_X)[:, s] Y_k^h(x_hat), V[:, (k, s, h)] =
   (Q_Y W_Y)[:, s] Y_k^h(y_hat), S = sigma_{k,s}.  Algorithm 1 folds sqrt(Sigma) into both
   factors; keeping Sigma as the diagonal S gives the same product U S V^T and the same
   column order as the symmetric factor (k ascending, then sigma decreasing, then h).
"""
from dataclasses import dataclass, field

import numpy as np

from .chebyshev import cheb_coeffs, choose_degree
from .harmonics import directions, harmonics_block
from .hdf import (ETA_DEFAULT, MU2_EXACT_MAX, P_MAX_DEFAULT, Plan, cheb_nodes_count, truncate)
from .kernels import kernel
from .radial import basis_size, radial_basis, stable_core


def center_scale_xy(x, y):
    """Step 1: (x', y', c, R) with one centre and radius for both sets."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    c = np.concatenate([x, y], axis=0).mean(axis=0)
    R = max(float(np.sqrt(((x - c) ** 2).sum(axis=1)).max()),
            float(np.sqrt(((y - c) ** 2).sum(axis=1)).max()))
    if R == 0.0:
        R = 1.0
    return (x - c) / (2.0 * R), (y - c) / (2.0 * R), c, R


def _strided(P):
    n = P.shape[0]
    if n <= MU2_EXACT_MAX:
        return P
    return P[(np.arange(MU2_EXACT_MAX, dtype=np.int64) * n) // MU2_EXACT_MAX]


def mean_square_kernel_xy(xs, ys, kap):
    """mu2 = mean over cross pairs of kappa(|x'_i - y'_j|)^2: exact when a set has at most 512
    points, otherwise on its 512 points with indices floor(t m / 512)."""
    P, Q = _strided(xs), _strided(ys)
    diff = P[:, None, :] - Q[None, :, :]
    return float(np.mean(kap(np.sqrt((diff * diff).sum(axis=-1))) ** 2))


def plan_xy(x, y, kname, ell, tol, eta=ETA_DEFAULT, p_max=P_MAX_DEFAULT):
    """Steps 1-2 for the cross block: scaling, coefficients, degree and the two budgets."""
    xs, ys, c, R = center_scale_xy(x, y)
    m, n = xs.shape[0], ys.shape[0]

    def kap(r):
        return kernel(kname, 2.0 * R * np.asarray(r), ell)

    mu2 = mean_square_kernel_xy(xs, ys, kap)
    a = cheb_coeffs(kap, cheb_nodes_count(p_max))
    tail_budget = 0.5 * tol * np.sqrt(mu2)
    p, tail, reached = choose_degree(a, tail_budget, p_max)
    drop_budget = 0.5 * eta * tol * np.sqrt(float(m) * float(n)) * np.sqrt(mu2)
    return xs, ys, Plan(kname, float(ell), float(tol), float(eta), int(p_max), c, R, mu2, a, p,
                        tail, reached, tail_budget, drop_budget)


@dataclass
class CrossFactor:
    """K(X, Y) ~= U diag(S) V^T."""
    U: np.ndarray
    V: np.ndarray
    S: np.ndarray
    plan: Plan
    d: int
    blocks: list = field(default_factory=list)   # per k: dict(k, s, sig, WX, WY, par)

    @property
    def rank(self):
        return self.U.shape[1]


def build_xy(x, y, kname, ell, tol, eta=ETA_DEFAULT, p_max=P_MAX_DEFAULT, keep_all=False, p=None):
    """Algorithm 1 (general form) by the stable route.  keep_all keeps every singular triple;
    p overrides the chosen degree."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    d = x.shape[1]
    if y.shape[1] != d:
        raise ValueError("X and Y must have the same dimension")
    xs, ys, pl = plan_xy(x, y, kname, ell, tol, eta, p_max)
    if p is not None:
        pl.p = int(p)
    L = pl.L
    cores = stable_core(pl.a, pl.p, d)
    rx = np.sqrt((xs * xs).sum(axis=1))
    ry = np.sqrt((ys * ys).sum(axis=1))
    QX, RX, QY, RY = {}, {}, {}, {}
    for par in (0, 1):
        nb = basis_size(par, L)
        if nb == 0:
            continue
        QX[par], RX[par] = np.linalg.qr(radial_basis(rx, par, nb))
        QY[par], RY[par] = np.linalg.qr(radial_basis(ry, par, nb))
    sigs, wxs, wys = [], [], []
    for k in range(L + 1):
        par = k % 2
        G = RX[par] @ cores[k] @ RY[par].T
        WX, sig, WYt = np.linalg.svd(G)
        q = sig.shape[0]
        sigs.append(sig)
        wxs.append(WX[:, :q])
        wys.append(WYt[:q, :].T)
    kept = truncate(sigs, d, pl.drop_budget, keep_all)
    xhat, yhat = directions(xs), directions(ys)
    ucols, vcols, S, blocks = [], [], [], []
    for k in range(L + 1):
        idx = kept[k]
        par = k % 2
        blocks.append(dict(k=k, par=par, s=len(idx), sig=sigs[k][idx], WX=wxs[k][:, idx], WY=wys[k][:, idx]))
        if not idx:
            continue
        FX = QX[par] @ wxs[k][:, idx]
        FY = QY[par] @ wys[k][:, idx]
        HX, HY = harmonics_block(k, xhat), harmonics_block(k, yhat)
        for s in range(len(idx)):
            ucols.append(FX[:, s:s + 1] * HX)
            vcols.append(FY[:, s:s + 1] * HY)
            S.extend([sigs[k][idx[s]]] * HX.shape[1])
    U = np.concatenate(ucols, axis=1) if ucols else np.zeros((x.shape[0], 0))
    V = np.concatenate(vcols, axis=1) if vcols else np.zeros((y.shape[0], 0))
    return CrossFactor(U, V, np.asarray(S, dtype=np.float64), pl, d, blocks)


def matvec_xy(fac, V):
    """K~_XY V = U (S (V_f^T V)) for V with one row per point of Y."""
    V = np.asarray(V, dtype=np.float64)
    W = fac.S[:, None] * (fac.V.T @ V.reshape(V.shape[0], -1))
    return (fac.U @ W).reshape((fac.U.shape[0],) + V.shape[1:])


def matvec_xy_t(fac, W):
    """K~_XY^T W = V_f (S (U^T W)) for W with one row per point of X."""
    W = np.asarray(W, dtype=np.float64)
    Z = fac.S[:, None] * (fac.U.T @ W.reshape(W.shape[0], -1))
    return (fac.V @ Z).reshape((fac.V.shape[0],) + W.shape[1:])


def dense_kernel_xy(x, y, kname, ell):
    """K_ij = k(|x_i - y_j|) (Sec. 1)."""
    diff = np.asarray(x, dtype=np.float64)[:, None, :] - np.asarray(y, dtype=np.float64)[None, :, :]
    return kernel(kname, np.sqrt((diff * diff).sum(axis=-1)), ell)


def rel_fro_error_xy(fac, x, y, kname, ell):
    """|K_XY - U S V^T|_F / |K_XY|_F."""
    K = dense_kernel_xy(x, y, kname, ell)
    return float(np.linalg.norm(K - (fac.U * fac.S) @ fac.V.T) / np.linalg.norm(K))
