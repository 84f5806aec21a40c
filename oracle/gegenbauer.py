"""Gegenbauer algebra used by the expansion (Sec. 3.3 and App. A).

* ``A_coeff(k, i, alpha)`` -- the coefficient of C_k^alpha in cos^i (App. A):
      cos^i g = sum_k A_{ki} C_k^alpha(cos g),  A_{ki} = 0 unless k = i (mod 2), and
      A_{ki} = i! (alpha + k) / (2^i ((i-k)/2)! (alpha)_{(i+k)/2+1}).
  The typeset factor "(i-k)/2" in the denominator is read as the factorial ((i-k)/2)!:
  this is the classical inversion x^i = i!/2^i sum_j (alpha+i-2j)/(j! (alpha)_{i-j+1})
  C^alpha_{i-2j}(x) with j = (i-k)/2 (checked in tests by evaluating both sides).
* ``sphere_area(d)``       -- |S^{d-1}| = 2 pi^{d/2} / Gamma(d/2).
* ``inv_Z(k, d)``          -- 1/Z_k of the addition theorem (Eq. additiontheorem) for
      orthonormal real harmonics on S^{d-1}:  sum_h Y_k^h(x) Y_k^h(y) = C_k^alpha(x.y)/Z_k,
      1/Z_k = (k + alpha) / (alpha |S^{d-1}|), alpha = d/2 - 1, d >= 3.
      The paper names Z_k as a normaliser but gives no formula for it; this value follows
      from the harmonics' orthonormality (pinned in tests by the addition theorem itself).
* ``gegen_norm(n, lam)``   -- h_n^lam = int_{-1}^{1} (C_n^lam)^2 (1-t^2)^{lam-1/2} dt.
* ``harmonic_count(k, d)`` -- |H_k| = C(k+d-1, k) - C(k+d-3, k-2) (App. B).
* ``harmonic_total(L, d)`` -- H_{L,d} = C(L+d-1, d-1) + C(L+d-2, d-1) (App. B).
"""
from math import comb, factorial, gamma, lgamma, pi, exp

import numpy as np
from scipy.special import eval_gegenbauer, poch


def A_coeff(k, i, alpha):
    """Coefficient of C_k^alpha in cos^i (App. A), with ((i-k)/2)! in the denominator."""
    if k > i or (i - k) % 2:
        return 0.0
    j = (i - k) // 2
    return factorial(i) * (alpha + k) / (2.0 ** i * factorial(j) * poch(alpha, (i + k) // 2 + 1))


def sphere_area(d):
    """|S^{d-1}|, the surface area of the unit sphere in R^d."""
    return 2.0 * pi ** (d / 2.0) / gamma(d / 2.0)


def inv_Z(k, d):
    """1/Z_k in Eq. (additiontheorem) for orthonormal real harmonics, d >= 3."""
    alpha = d / 2.0 - 1.0
    return (k + alpha) / (alpha * sphere_area(d))


def gegen_norm(n, lam):
    """h_n^lam = pi 2^(1-2 lam) Gamma(n + 2 lam) / (n! (n + lam) Gamma(lam)^2)."""
    logv = (np.log(pi) + (1.0 - 2.0 * lam) * np.log(2.0) + lgamma(n + 2.0 * lam)
            - lgamma(n + 1.0) - np.log(n + lam) - 2.0 * lgamma(lam))
    return exp(logv)


def gegenbauer(n, lam, t):
    """C_n^lam(t) by the library routine (scipy.special.eval_gegenbauer)."""
    return eval_gegenbauer(n, lam, np.asarray(t, dtype=np.float64))


def harmonic_count(k, d):
    """|H_k| = C(k+d-1, k) - C(k+d-3, k-2) (App. B)."""
    return comb(k + d - 1, k) - (comb(k + d - 3, k - 2) if k >= 2 else 0)


def harmonic_total(L, d):
    """sum_{k<=L} |H_k| = C(L+d-1, d-1) + C(L+d-2, d-1) (App. B)."""
    return comb(L + d - 1, d - 1) + (comb(L + d - 2, d - 1) if L >= 1 else 0)
