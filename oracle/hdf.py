"""Algorithm 1 of Ryan & Damle in its symmetric form (Remark 1), plain FP64 numpy.

Steps, in the paper's order:

1. Scale (Sec. 3.3 footnote: the point set's diameter is folded into the lengthscale; Sec. 4.1 scales
   points by their maximum norm).  c = mean(x), R = max |x_i - c|, x' = (x - c) / (2R),
   so |x'| <= 1/2 and |x'_i - x'_j| <= 1.  The scaled kernel is kappa(r) = k(2 R r).
   If all points coincide (R = 0) the scale is arbitrary and R = 1 is used.
2. Chebyshev coefficients a_i of kappa(|r|) on [-1, 1] (Sec. 3.3, ChebyshevTransform).
3. Degree (ChebDegreeNeeded, Remark 3): the smallest even p with
   sum_{i>p}|a_i| <= tol * sqrt(mu2) / 2, where mu2 = mean_{ij} K_ij^2, so that the entrywise
   Chebyshev error (Sec. 3.5) sums to at most tol * |K|_F / 2 in Frobenius norm.
4. Radial cores r^(k), k = 0..p/2 (Eq. rdef), in a stable basis (``radial.stable_core``).
5. QR (Eq. svd): the paper factors each Vandermonde block Y^(k) (Eq. vandermonde).  The
   radial functions of all even k (odd k) lie in the span of one basis
   B_par = rho^par [T_l(8 rho^2 - 1)]_l, so one QR per parity serves every k -- the
   Vandermonde matrix formed once, outside the loop over k (Sec. 3.6).  Then G_k = R_par Gamma_k R_par^T.
6. Eigendecomposition (Remark 1) G_k = W_k Lambda_k W_k^T and truncation (Sec. 3.4 with the
   tau of Sec. 3.5 made concrete): dropping eigenpair (lambda, w) of block k changes K by
   at most |lambda| |H_k| / |S^{d-1}| in Frobenius norm (addition theorem at angle 0).
   Eigenpairs are dropped globally in increasing order of that cost, ties broken by
   (k, index), while the summed cost stays <= eta * tol * |K|_F / 2.  Blocks with nothing
   left are dropped whole (Remark 2).
7. Assemble U[:, (k, s, h)] = (Q_par W_k)[:, s] * Y_k^h(x_hat) and S = lambda_{k,s}
   (Algorithm 1's inner loops with the square roots of Sigma kept in the diagonal S of
   Remark 1).  Column order: k ascending, then kept eigenpairs by decreasing |lambda|,
   then h in ``harmonics.index_set`` order.

|K|_F is taken from mu2 = mean K_ij^2: exactly when n <= 512, otherwise over all pairs of
the 512 points with indices floor(t n / 512), t = 0..511 (the estimate only sets the two
error budgets, so a coarse sample suffices).
"""
from dataclasses import dataclass, field

import numpy as np

from .chebyshev import cheb_coeffs, choose_degree
from .gegenbauer import harmonic_count, sphere_area
from .harmonics import directions, harmonics_block
from .kernels import kernel, kernel_dell, kernel_dr
from .radial import basis_size, literal_core, literal_power_core, radial_basis, stable_core

P_MAX_DEFAULT = 64
ETA_DEFAULT = 1.0
MU2_EXACT_MAX = 512


def cheb_nodes_count(p_max):
    """Number of DCT nodes used for the Chebyshev coefficients: 4 (p_max + 2)."""
    return 4 * (int(p_max) + 2)


def center_scale(x):
    """Step 1: (x', c, R) with x' = (x - c) / (2R)."""
    x = np.asarray(x, dtype=np.float64)
    c = x.mean(axis=0)
    y = x - c
    R = float(np.sqrt((y * y).sum(axis=1)).max())
    if R == 0.0:
        R = 1.0
    return y / (2.0 * R), c, R


def mean_square_kernel(xs, kap):
    """mu2 = mean over pairs of kappa(|x'_i - x'_j|)^2 (exact or on the strided subsample)."""
    n = xs.shape[0]
    if n <= MU2_EXACT_MAX:
        P = xs
    else:
        idx = (np.arange(MU2_EXACT_MAX, dtype=np.int64) * n) // MU2_EXACT_MAX
        P = xs[idx]
    diff = P[:, None, :] - P[None, :, :]
    D = np.sqrt((diff * diff).sum(axis=-1))
    return float(np.mean(kap(D) ** 2))


@dataclass
class Plan:
    kernel: str
    ell: float
    tol: float
    eta: float
    p_max: int
    c: np.ndarray
    R: float
    mu2: float
    a: np.ndarray
    p: int
    tail: float
    reached: bool
    tail_budget: float
    drop_budget: float

    @property
    def L(self):
        return self.p // 2

    def kappa(self, r, ell=None):
        return kernel(self.kernel, 2.0 * self.R * np.asarray(r), self.ell if ell is None else ell)


def plan(x, kname, ell, tol, eta=ETA_DEFAULT, p_max=P_MAX_DEFAULT):
    """Steps 1-3: scaling, Chebyshev coefficients, degree and the two error budgets."""
    xs, c, R = center_scale(x)
    n = xs.shape[0]

    def kap(r):
        return kernel(kname, 2.0 * R * np.asarray(r), ell)

    mu2 = mean_square_kernel(xs, kap)
    a = cheb_coeffs(kap, cheb_nodes_count(p_max))
    tail_budget = 0.5 * tol * np.sqrt(mu2)
    p, tail, reached = choose_degree(a, tail_budget, p_max)
    drop_budget = 0.5 * eta * tol * n * np.sqrt(mu2)
    return xs, Plan(kname, float(ell), float(tol), float(eta), int(p_max), c, R, mu2, a, p,
                    tail, reached, tail_budget, drop_budget)


@dataclass
class Factor:
    """K ~= U diag(S) U^T plus what the frozen-structure adjoint needs."""
    U: np.ndarray
    S: np.ndarray
    plan: Plan
    d: int
    blocks: list = field(default_factory=list)   # per k: dict(k, s, lam, W, par)
    Rfac: dict = field(default_factory=dict)     # par -> R factor of B_par
    cores: list = field(default_factory=list)

    @property
    def rank(self):
        return self.U.shape[1]


def truncate(eigs, d, budget, keep_all=False):
    """Step 6: choose kept eigenpairs.  eigs[k] = eigenvalues of G_k.  Returns kept index lists."""
    area = sphere_area(d)
    items = []
    for k, lam in enumerate(eigs):
        hk = harmonic_count(k, d)
        for j, l in enumerate(lam):
            items.append((abs(l) * hk / area, k, j))
    items.sort()
    dropped = set()
    if not keep_all:
        acc = 0.0
        for cost, k, j in items:
            if acc + cost > budget:
                break
            acc += cost
            dropped.add((k, j))
    kept = []
    for k, lam in enumerate(eigs):
        idx = [j for j in range(len(lam)) if (k, j) not in dropped]
        idx.sort(key=lambda j: (-abs(lam[j]), j))
        kept.append(idx)
    return kept


def _assemble(xs, d, Qs, blocks):
    xhat = directions(xs)
    n = xs.shape[0]
    cols, S = [], []
    for b in blocks:
        if b["s"] == 0:
            continue
        F = Qs[b["par"]] @ b["W"]                      # n x s_k
        Y = harmonics_block(b["k"], xhat)              # n x |H_k|
        for s in range(b["s"]):
            cols.append(F[:, s:s + 1] * Y)
            S.extend([b["lam"][s]] * Y.shape[1])
    U = np.concatenate(cols, axis=1) if cols else np.zeros((n, 0))
    return U, np.asarray(S, dtype=np.float64)


def build(x, kname, ell, tol, eta=ETA_DEFAULT, p_max=P_MAX_DEFAULT, keep_all=False, p=None):
    """Algorithm 1 (symmetric, Remark 1) by the stable route.  Returns a Factor.

    keep_all=True keeps every eigenpair (no compression); p overrides the chosen degree.
    """
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[1]
    xs, pl = plan(x, kname, ell, tol, eta, p_max)
    if p is not None:
        pl.p = int(p)
    L = pl.L
    cores = stable_core(pl.a, pl.p, d)
    rho = np.sqrt((xs * xs).sum(axis=1))
    Qs, Rs = {}, {}
    for par in (0, 1):
        nb = basis_size(par, L)
        if nb == 0:
            continue
        Qs[par], Rs[par] = np.linalg.qr(radial_basis(rho, par, nb))
    eigs, vecs = [], []
    for k in range(L + 1):
        R = Rs[k % 2]
        G = R @ cores[k] @ R.T
        lam, W = np.linalg.eigh(0.5 * (G + G.T))
        eigs.append(lam)
        vecs.append(W)
    kept = truncate(eigs, d, pl.drop_budget, keep_all)
    blocks = []
    for k in range(L + 1):
        idx = kept[k]
        blocks.append(dict(k=k, par=k % 2, s=len(idx), lam=eigs[k][idx], W=vecs[k][:, idx]))
    U, S = _assemble(xs, d, Qs, blocks)
    return Factor(U, S, pl, d, blocks, Rs, cores)


def build_literal(x, kname, ell, tol, eta=ETA_DEFAULT, p_max=P_MAX_DEFAULT, keep_all=False, p=None):
    """Algorithm 1 literally: per-k power-basis Vandermonde Y^(k) (Eq. vandermonde), its QR,
    and the App. A core in the power basis.  Accurate only while the power-basis growth
    stays far below 1/eps (Sec. 3.7); used to cross-check the stable route."""
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[1]
    xs, pl = plan(x, kname, ell, tol, eta, p_max)
    if p is not None:
        pl.p = int(p)
    L = pl.L
    Tpp, _ = literal_core(pl.a, pl.p, d)
    rho = np.sqrt((xs * xs).sum(axis=1))
    eigs, vecs, Qk = [], [], []
    for k in range(L + 1):
        Y = rho[:, None] ** (k + 2 * np.arange(L - k + 1))[None, :]
        Q, R = np.linalg.qr(Y)
        C = literal_power_core(Tpp, k, L)
        G = R @ C @ R.T
        lam, W = np.linalg.eigh(0.5 * (G + G.T))
        eigs.append(lam)
        vecs.append(W)
        Qk.append(Q)
    kept = truncate(eigs, d, pl.drop_budget, keep_all)
    xhat = directions(xs)
    cols, S = [], []
    for k in range(L + 1):
        idx = kept[k]
        if not idx:
            continue
        F = Qk[k] @ vecs[k][:, idx]
        Y = harmonics_block(k, xhat)
        for s in range(len(idx)):
            cols.append(F[:, s:s + 1] * Y)
            S.extend([eigs[k][idx[s]]] * Y.shape[1])
    U = np.concatenate(cols, axis=1) if cols else np.zeros((x.shape[0], 0))
    return Factor(U, np.asarray(S), pl, d)


# ------------------------------------------------------------------ operators and checks

def matvec(fac, V):
    """K~ V = U (S (U^T V)) (Sec. 3.6: O(N r) after the factorization)."""
    V = np.asarray(V, dtype=np.float64)
    return fac.U @ (fac.S[:, None] * (fac.U.T @ V.reshape(V.shape[0], -1))).reshape(
        (fac.rank,) + V.shape[1:])


def solve(fac, lam, B):
    """(lam I + K~)^{-1} B, the regularised system of Eq. (opt).

    n <= 4000: dense solve of the assembled n x n matrix.  Otherwise the
    Sherman-Morrison-Woodbury identity (Sec. 1):
        (lam I + U S U^T)^{-1} = (1/lam) [I - U (lam S^{-1} + U^T U)^{-1} U^T].
    """
    U, S = fac.U, fac.S
    B = np.asarray(B, dtype=np.float64)
    n = U.shape[0]
    if n <= 4000:
        Kt = (U * S) @ U.T
        return np.linalg.solve(lam * np.eye(n) + Kt, B)
    core = lam * np.diag(1.0 / S) + U.T @ U
    return (B - U @ np.linalg.solve(core, U.T @ B)) / lam


def dense_kernel(x, kname, ell, rows=None):
    """K_ij = k(|x_i - x_j|) (Sec. 1), optionally only for the given rows."""
    x = np.asarray(x, dtype=np.float64)
    xr = x if rows is None else x[rows]
    diff = xr[:, None, :] - x[None, :, :]
    return kernel(kname, np.sqrt((diff * diff).sum(axis=-1)), ell)


def dense_matvec_rows(x, kname, ell, V, rows, chunk=256):
    """(K V)[rows] exactly, chunked over the rows."""
    out = []
    for s in range(0, len(rows), chunk):
        out.append(dense_kernel(x, kname, ell, rows[s:s + chunk]) @ V)
    return np.concatenate(out, axis=0)


def rel_fro_error(fac, x, kname, ell):
    """|K - U S U^T|_F / |K|_F (the relative error of Sec. 4, in Frobenius norm)."""
    K = dense_kernel(x, kname, ell)
    Kt = (fac.U * fac.S) @ fac.U.T
    return float(np.linalg.norm(K - Kt) / np.linalg.norm(K))


# -------------------------------------------------------- frozen-structure evaluator

def frozen_U(fac, X):
    """U rows at new points X with the build's scaling, degree, cores and eigenvectors frozen.

    U_i(x) = f_{k,s}(|x'|) Y_k^h(x'/|x'|), x' = (x - c)/(2R),
    f_{k,s}(rho) = B_par(rho) R_par^{-1} W_k[:, s]  (so f = Q_par W_k at the build points).
    """
    pl = fac.plan
    X = np.asarray(X, dtype=np.float64)
    xs = (X - pl.c) / (2.0 * pl.R)
    rho = np.sqrt((xs * xs).sum(axis=1))
    xhat = directions(xs)
    L = pl.L
    cols = []
    for b in fac.blocks:
        if b["s"] == 0:
            continue
        nb = basis_size(b["k"], L)
        Bm = radial_basis(rho, b["par"], nb)
        F = Bm @ np.linalg.solve(fac.Rfac[b["par"]], b["W"])
        Y = harmonics_block(b["k"], xhat)
        for s in range(b["s"]):
            cols.append(F[:, s:s + 1] * Y)
    return np.concatenate(cols, axis=1)


def frozen_cores(fac, ell):
    """Gamma_k(ell) with the build's p, c, R frozen (for d/d ell)."""
    pl = fac.plan

    def kap(r):
        return kernel(pl.kernel, 2.0 * pl.R * np.asarray(r), ell)

    a = cheb_coeffs(kap, cheb_nodes_count(pl.p_max))
    a[pl.p + 1:] = 0.0
    return stable_core(a, pl.p, fac.d)


def frozen_apply_S(fac, cores, z):
    """S(ell) z for an r-vector z: block (k, h) gets S_k = W_k^T R Gamma_k R^T W_k."""
    out = np.zeros_like(z)
    col = 0
    for b in fac.blocks:
        if b["s"] == 0:
            continue
        R = fac.Rfac[b["par"]]
        Sk = b["W"].T @ R @ cores[b["k"]] @ R.T @ b["W"]
        hk = harmonic_count(b["k"], fac.d)
        blk = z[col:col + b["s"] * hk].reshape(b["s"], hk)
        out[col:col + b["s"] * hk] = (Sk @ blk).reshape(-1)
        col += b["s"] * hk
    return out


def frozen_f(fac, X, ell, v, w):
    """f(X, ell) = w^T U(X) S(ell) U(X)^T v under frozen structure."""
    U = frozen_U(fac, X)
    cores = frozen_cores(fac, ell)
    return float((U.T @ w) @ frozen_apply_S(fac, cores, U.T @ v))


def adjoint_fd(fac, X, v, w, h=1e-4):
    """grad_x f and d f / d ell of f = w^T K~ v by central differences of the frozen evaluator,
    Richardson-extrapolated over steps h and h/2 (error O(h^4)).

    Moving x_i changes only row i of U: with delta = U_i(x_i +- h e) - U_i(x_i),
    f changes by w_i delta.(S U^T v) + v_i delta.(S U^T w) + w_i v_i delta.(S delta).
    """
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    U0 = frozen_U(fac, X)
    cores0 = frozen_cores(fac, fac.plan.ell)
    av = frozen_apply_S(fac, cores0, U0.T @ v)
    aw = frozen_apply_S(fac, cores0, U0.T @ w)

    def dfs(hh):
        g = np.zeros((n, d))
        for e in range(d):
            res = []
            for sgn in (+1.0, -1.0):
                Xp = X.copy()
                Xp[:, e] += sgn * hh
                delta = frozen_U(fac, Xp) - U0
                quad = np.array([delta[i] @ frozen_apply_S(fac, cores0, delta[i]) for i in range(n)])
                res.append(w * (delta @ av) + v * (delta @ aw) + w * v * quad)
            g[:, e] = (res[0] - res[1]) / (2.0 * hh)
        return g

    g1, g2 = dfs(h), dfs(h / 2.0)
    grad = (4.0 * g2 - g1) / 3.0
    ell = fac.plan.ell

    def fl(hh):
        cp = frozen_cores(fac, ell + hh)
        cm = frozen_cores(fac, ell - hh)
        zw, zv = U0.T @ w, U0.T @ v
        return (zw @ frozen_apply_S(fac, cp, zv) - zw @ frozen_apply_S(fac, cm, zv)) / (2.0 * hh)

    dl = (4.0 * fl(h / 2.0) - fl(h)) / 3.0
    return grad, float(dl)


def dense_gradient(x, kname, ell, v, w):
    """Gradient of w^T K v for the exact kernel matrix:
    d/dx_i = sum_l k'(r_il) (x_i - x_l)/r_il (w_i v_l + w_l v_i),  d/d ell = w^T (dK/d ell) v."""
    x = np.asarray(x, dtype=np.float64)
    diff = x[:, None, :] - x[None, :, :]
    r = np.sqrt((diff * diff).sum(axis=-1))
    kp = kernel_dr(kname, r, ell)
    with np.errstate(invalid="ignore", divide="ignore"):
        coef = np.where(r > 0, kp / np.where(r > 0, r, 1.0), 0.0)
    M = coef * (np.outer(w, v) + np.outer(v, w))
    grad = (M[:, :, None] * diff).sum(axis=1)
    dl = float(w @ kernel_dell(kname, r, ell) @ v)
    return grad, dl
