"""Radial functions r^(k)(|x|, |y|) of Eq. (rdef), by two independent routes.

After the Chebyshev step (Sec. 3.3) the truncated kernel is F(s) = sum_{q<=L} a_{2q} T_q(2s-1)
with s = |x - y|^2 (because T_{2q}(r) = T_q(2 r^2 - 1)), L = p/2.  Sec. 3.3 expands
F(|x|^2 + |y|^2 - 2|x||y|cos g) in Gegenbauer polynomials C_k^alpha(cos g) (Eq. preharm) and
then uses the addition theorem, so that
    r^(k)(a, b) = Z_k * sum_{m,n} b^m a^n T'_{k,m,n} = sum_{m,n} b^m a^n T''_{k,m,n}.

* Literal route (``literal_core`` / ``literal_r``): App. A's closed form
      T'_{j,m,n} = sum_{k3} A_{k3 j} (-2)^{k3} multinom((n+m)/2; (n-k3)/2, (m-k3)/2, k3) c_{n+m},
      c_{2q} = sum_{i=2q}^{p} t_{i,2q} a_i,
  with k3 running over j <= k3 <= min(m, n), k3 = j = m = n (mod 2) (the sum limits of
  App. A, with the inner i-sum collapsed into the monomial coefficient c_{n+m} of the
  truncated series).  The monomial form suffers heavy cancellation (Sec. 3.7), so this
  route runs in mpmath at a working precision chosen from the coefficient growth.
* Stable route (``stable_core``): the Gegenbauer coefficient of F(a^2+b^2-2abt) in t is
  its projection  (1/h_k) int F(.) C_k^alpha(t) (1-t^2)^{alpha-1/2} dt,  evaluated exactly
  (the integrand is a polynomial) by Gauss-Gegenbauer quadrature (library nodes), times
  Z_k.  The result is represented in the basis the Limitations paragraph of Sec. 3.7
  suggests -- orthogonal polynomials of |x|^2 instead of powers of |x| -- here Chebyshev
  T_l(8 s - 1) on s = |x|^2 in [0, 1/4]:
      even k:  r^(k)(a, b) = sum_{l,l'} G[l,l'] T_l(8a^2-1) T_l'(8b^2-1),      l, l' <= L
      odd k:   r^(k)(a, b) = a b sum_{l,l'} G[l,l'] T_l(8a^2-1) T_l'(8b^2-1),  l, l' <= L-1
  (r^(k) is (ab)^k times a polynomial of total degree L-k in a^2, b^2, so these bases are
  exact).  G is found by interpolation at first-kind Chebyshev nodes in 8s-1.
"""
from math import comb, factorial

import numpy as np
from numpy.polynomial.chebyshev import chebvander
from scipy.special import roots_gegenbauer

from .chebyshev import cheb_eval, monomial_coeffs
from .gegenbauer import gegen_norm, gegenbauer, inv_Z


# ----------------------------------------------------------------------------- literal

def literal_core(a, p, d, dps=None):
    """T''[k][(m, n)] = Z_k T'_{k,m,n} of App. A, as mpmath numbers.

    a: Chebyshev coefficients (float), p: even degree, d >= 3.  dps defaults to
    log10(growth) + 30 digits, growth = sum |c_j| (the monomial coefficients).
    Returns (Tpp, ctx) where Tpp[k] is a dict {(m, n): value}.
    """
    import mpmath
    ctx = mpmath.mp.clone() if hasattr(mpmath.mp, "clone") else mpmath.mp
    L = p // 2
    t = monomial_coeffs(p)
    if dps is None:
        growth = 0.0
        for jj in range(0, p + 1, 2):
            growth += abs(sum(t[i][jj] * float(a[i]) for i in range(jj, p + 1)))
        dps = int(np.log10(max(growth, 1.0))) + 30
    ctx.dps = dps
    mpf = ctx.mpf
    aa = [mpf(float(a[i])) if i < len(a) else mpf(0) for i in range(p + 1)]
    c = [mpf(0)] * (p + 1)
    for jj in range(0, p + 1, 2):
        c[jj] = ctx.fsum(t[i][jj] * aa[i] for i in range(jj, p + 1))
    alpha = mpf(d) / 2 - 1
    area = 2 * ctx.pi ** (mpf(d) / 2) / ctx.gamma(mpf(d) / 2)

    def A(deg, pw):
        if deg > pw or (pw - deg) % 2:
            return mpf(0)
        return (ctx.factorial(pw) * (alpha + deg)
                / (mpf(2) ** pw * ctx.factorial((pw - deg) // 2) * ctx.rf(alpha, (pw + deg) // 2 + 1)))

    Tpp = []
    for j in range(L + 1):
        Zj = alpha * area / (j + alpha)
        blk = {}
        for m in range(j, p - j + 1, 2):
            for n in range(j, p - m + 1, 2):
                s = mpf(0)
                for k3 in range(j, min(m, n) + 1, 2):
                    k1, k2 = (n - k3) // 2, (m - k3) // 2
                    multi = factorial(k1 + k2 + k3) // (factorial(k1) * factorial(k2) * factorial(k3))
                    s += A(j, k3) * mpf(-2) ** k3 * multi * c[n + m]
                blk[(m, n)] = Zj * s
        Tpp.append(blk)
    return Tpp, ctx


def literal_r(Tpp, ctx, k, a_, b_):
    """r^(k)(a_, b_) = sum_{m,n} b^m a^n T''_{k,m,n} evaluated in mpmath, returned as float."""
    a_m, b_m = ctx.mpf(float(a_)), ctx.mpf(float(b_))
    return float(ctx.fsum(v * b_m ** m * a_m ** n for (m, n), v in Tpp[k].items()))


def literal_power_core(Tpp, k, L):
    """Power-basis core C_k[l, l'] = T''_{k, k+2l, k+2l'} (Eq. vandermonde), float64."""
    nb = L - k + 1
    C = np.zeros((nb, nb))
    for l in range(nb):
        for lp in range(nb):
            v = Tpp[k].get((k + 2 * l, k + 2 * lp))
            if v is not None:
                C[l, lp] = float(v)
    return C


# ------------------------------------------------------------------------------ stable

def basis_size(k, L):
    """Number of stable-basis functions for parity k % 2: L+1 (even), L (odd)."""
    return L + 1 if k % 2 == 0 else L


def radial_basis(rho, par, nb):
    """B[i, l] = rho_i^par T_l(8 rho_i^2 - 1), l < nb (the stable radial basis).

    T_l comes from numpy's Chebyshev-Vandermonde routine, valid also just outside
    [-1, 1] (points moved past |x'| = 1/2 by a finite difference)."""
    rho = np.asarray(rho, dtype=np.float64)
    B = chebvander(8.0 * rho * rho - 1.0, nb - 1) if nb > 0 else np.zeros(rho.shape + (0,))
    if par:
        B = B * rho[:, None]
    return B


def projection_r(a_cheb, p, d, k, a_, b_):
    """r^(k)(a_, b_) = Z_k (1/h_k) int F(a^2+b^2-2abt) C_k^alpha(t) (1-t^2)^(alpha-1/2) dt.

    Gauss-Gegenbauer quadrature with L+2 nodes integrates the degree <= L + k polynomial
    integrand exactly.  a_, b_ may be arrays of equal shape.
    """
    L = p // 2
    alpha = d / 2.0 - 1.0
    t, w = roots_gegenbauer(L + 2, alpha)
    f = np.array([a_cheb[2 * q] for q in range(L + 1)], dtype=np.float64)
    a_ = np.asarray(a_, dtype=np.float64)
    b_ = np.asarray(b_, dtype=np.float64)
    s = (a_ * a_ + b_ * b_)[..., None] - 2.0 * (a_ * b_)[..., None] * t
    Fv = cheb_eval(f, 2.0 * s - 1.0)
    proj = (Fv * gegenbauer(k, alpha, t) * w).sum(axis=-1) / gegen_norm(k, alpha)
    return inv_Z_to_Z(k, d) * proj


def inv_Z_to_Z(k, d):
    """Z_k = 1 / (1/Z_k)."""
    return 1.0 / inv_Z(k, d)


def stable_core(a_cheb, p, d):
    """Gamma_k (k = 0..L): coefficients of r^(k) in the stable basis (module docstring)."""
    L = p // 2
    cores = []
    for k in range(L + 1):
        nb = basis_size(k, L)
        if nb == 0:
            cores.append(np.zeros((0, 0)))
            continue
        j = np.arange(nb, dtype=np.float64)
        u = np.cos(np.pi * (j + 0.5) / nb)
        rho = np.sqrt((u + 1.0) / 8.0)
        A_, B_ = np.meshgrid(rho, rho, indexing="ij")
        V = projection_r(a_cheb, p, d, k, A_, B_)
        if k % 2:
            V = V / np.outer(rho, rho)
        Phi = np.cos(np.outer(np.arccos(u), np.arange(nb, dtype=np.float64)))
        X = np.linalg.solve(Phi, V)            # Phi^{-1} V
        G = np.linalg.solve(Phi, X.T).T        # Phi^{-1} V Phi^{-T}
        cores.append(0.5 * (G + G.T))
    return cores


def stable_r(cores, k, a_, b_):
    """r^(k)(a_, b_) from the stable core Gamma_k (vectorised over equal-shape a_, b_)."""
    a_ = np.atleast_1d(np.asarray(a_, dtype=np.float64))
    b_ = np.atleast_1d(np.asarray(b_, dtype=np.float64))
    G = cores[k]
    nb = G.shape[0]
    Ba = radial_basis(a_, k % 2, nb)
    Bb = radial_basis(b_, k % 2, nb)
    return np.einsum("il,lm,im->i", Ba, G, Bb)
