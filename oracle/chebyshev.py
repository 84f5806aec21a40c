"""One-dimensional Chebyshev expansion of the scaled kernel (Sec. 3.3, Eq. chebtrunc).

* ``cheb_coeffs``    -- a_i of the even extension k_bar(r) = k(|r|) on [-1, 1] by the
                        discrete cosine transform at first-kind Chebyshev points
                        (the DCT / Clenshaw-Curtis route the paper names in Sec. 3.3).
                        Odd a_i are set to exactly zero (k_bar is even, Sec. 3.3).
* ``choose_degree``  -- ChebDegreeNeeded of Algorithm 1 (Remark 3): the smallest even p
                        whose estimated coefficient tail (``tail_sums``) is within the budget.
* ``monomial_coeffs``-- t_{i,j} of Eq. (chebdef), T_i(r) = sum_j t_{i,j} r^j.
                        The paper's case list starts the recurrence with "1 if i = j",
                        which only holds for i <= 1; the leading coefficient of T_i is
                        2^(i-1).  We use t_00 = t_11 = 1 and
                        t_{i,j} = 2 t_{i-1,j-1} - t_{i-2,j}, the defining three-term
                        recurrence T_i = 2 r T_{i-1} - T_{i-2}.
* ``cheb_eval``      -- sum_i a_i T_i(r) by numpy's Chebyshev-series evaluation.
"""
import numpy as np
from numpy.polynomial.chebyshev import chebval


def cheb_coeffs(f, M):
    """Chebyshev interpolant coefficients a_0..a_{M-1} of the even function f(|r|) on [-1,1].

    f is evaluated at the M first-kind nodes r_j = cos(pi (j + 1/2) / M) and
    a_i = (2/M) sum_j f(|r_j|) cos(i pi (j + 1/2) / M), with a_0 halved (DCT-II).
    """
    M = int(M)
    j = np.arange(M, dtype=np.float64)
    theta = np.pi * (j + 0.5) / M
    vals = np.asarray(f(np.abs(np.cos(theta))), dtype=np.float64)
    i = np.arange(M, dtype=np.float64)
    a = (2.0 / M) * (np.cos(np.outer(i, theta)) @ vals)
    a[0] *= 0.5
    a[1::2] = 0.0
    return a


def tail_sums(a):
    """Estimated tail epsilon_c(p) of Sec. 3.5 for p = 0..M-1, from M computed coefficients:

        tails[p] = sum_{p < i < M} |a_i|  +  sum_{M/2 <= i < M} |a_i|.

    Remark 3 says only that the tail can be estimated cheaply.  The second sum stands in for
    the coefficients beyond M that the DCT cannot see: when |a_i| decays like i^-q with
    q >= 2 (Matern-3/2 decays like i^-4) the upper half of the computed coefficients
    carries at least as much mass as everything beyond M; for geometric decay it is at
    rounding level.
    """
    absa = np.abs(np.asarray(a, dtype=np.float64))
    M = absa.size
    c = np.cumsum(absa[::-1])[::-1]          # c[p] = sum_{i >= p}
    guard = absa[M // 2:].sum()
    return np.append(c[1:], 0.0) + guard


def choose_degree(a, budget, p_max):
    """Smallest even p <= p_max with tail_sums(a)[p] <= budget (Remark 3).

    Returns (p, tail, reached).  When no even p <= p_max meets the budget, p = p_max
    (rounded down to even) and reached is False.
    """
    tails = tail_sums(a)
    p_max = int(p_max) - (int(p_max) % 2)
    for p in range(0, p_max + 1, 2):
        if tails[p] <= budget:
            return p, float(tails[p]), True
    return p_max, float(tails[p_max]), False


def monomial_coeffs(p):
    """t[i, j] with T_i(r) = sum_j t[i, j] r^j for 0 <= i <= p (Eq. chebdef), as Python ints."""
    t = [[0] * (p + 1) for _ in range(p + 1)]
    t[0][0] = 1
    if p >= 1:
        t[1][1] = 1
    for i in range(2, p + 1):
        for j in range(0, i + 1):
            v = -t[i - 2][j]
            if j >= 1:
                v += 2 * t[i - 1][j - 1]
            t[i][j] = v
    return t


def cheb_eval(a, r):
    """sum_i a_i T_i(r) by numpy's Chebyshev-series routine (also valid for |r| > 1)."""
    return chebval(np.asarray(r, dtype=np.float64), np.asarray(a, dtype=np.float64))
