"""Real hyperspherical harmonics Y_k^h on S^{d-1} (Eq. additiontheorem and its footnote).

The index set is H_k = {(mu_1, ..., mu_{d-2}) : k >= mu_1 >= ... >= |mu_{d-2}| >= 0}
(Sec. 3.3).  The paper defers the construction to Avery; we use the standard one in
hyperspherical angles, evaluated here with trigonometry and the library Gegenbauer
routine so that nothing is shared with the polynomial recurrences of the CUDA path:

  x = (x_0, ..., x_{d-1}),  level j = 0..d-3 peels coordinate D_j = d-1-j:
      cos(theta_j) = x_{D_j} / |x_{0..D_j}|,  sin(theta_j) = |x_{0..D_j-1}| / |x_{0..D_j}|,
  and phi = atan2(x_1, x_0).  With mu_0 = k,

  Y = prod_j h_{n_j}^{lam_j}^{-1/2} sin(theta_j)^{|mu_{j+1}|} C_{n_j}^{lam_j}(cos theta_j) * Phi,
      n_j = mu_j - |mu_{j+1}|,  lam_j = |mu_{j+1}| + (d-j-2)/2,
      Phi = 1/sqrt(2 pi) (mu_{d-2} = 0), cos(m phi)/sqrt(pi) (m > 0), sin(|m| phi)/sqrt(pi) (m < 0),

  where cos(mu phi) is used for mu_{d-2} >= 0 and sin(|mu| phi) for mu_{d-2} < 0 (a real
  basis, as the footnote to Eq. additiontheorem asks).  The harmonics are orthonormal on
  S^{d-1} (pinned in tests by exact product quadrature) and satisfy the addition theorem
  with 1/Z_k from ``gegenbauer.inv_Z`` (pinned by evaluating both sides).

Order of H_k: lexicographic ascending in (mu_1, ..., mu_{d-2}).  A zero vector is given
the direction e_0.
"""
import numpy as np

from .gegenbauer import gegen_norm, gegenbauer


def index_set(k, d):
    """The chains of H_k in lexicographic ascending order (App. B counts them)."""
    if d < 3:
        raise ValueError("d >= 3 required")
    if d == 3:
        return [(m,) for m in range(-k, k + 1)]
    out = []
    for m1 in range(0, k + 1):
        for rest in index_set(m1, d - 1):
            out.append((m1,) + rest)
    return out


def directions(x):
    """Unit vectors x/|x| (rows); zero rows map to e_0."""
    x = np.asarray(x, dtype=np.float64)
    nrm = np.sqrt((x * x).sum(axis=1))
    out = np.zeros_like(x)
    nz = nrm > 0
    out[nz] = x[nz] / nrm[nz, None]
    out[~nz, 0] = 1.0
    return out


def angles(xhat):
    """Hyperspherical angles (theta_0..theta_{d-3}, phi) of unit rows xhat (N x d)."""
    N, d = xhat.shape
    thetas = []
    for j in range(d - 2):
        D = d - 1 - j
        below = np.sqrt((xhat[:, :D] ** 2).sum(axis=1))
        thetas.append(np.arctan2(below, xhat[:, D]))
    phi = np.arctan2(xhat[:, 1], xhat[:, 0])
    return thetas, phi


def harmonic(k, chain, xhat):
    """Y_k^chain at unit rows xhat (N x d) by the angle formula above."""
    xhat = np.asarray(xhat, dtype=np.float64)
    N, d = xhat.shape
    thetas, phi = angles(xhat)
    mus = (k,) + tuple(chain)
    val = np.ones(N)
    for j in range(d - 2):
        m_next = abs(mus[j + 1])
        n = mus[j] - m_next
        lam = m_next + (d - j - 2) / 2.0
        val = val * (np.sin(thetas[j]) ** m_next) * gegenbauer(n, lam, np.cos(thetas[j])) \
            / np.sqrt(gegen_norm(n, lam))
    m = mus[-1]
    if m == 0:
        val = val / np.sqrt(2.0 * np.pi)
    elif m > 0:
        val = val * np.cos(m * phi) / np.sqrt(np.pi)
    else:
        val = val * np.sin(-m * phi) / np.sqrt(np.pi)
    return val


def harmonics_block(k, xhat):
    """All harmonics of degree k at xhat: array (N, |H_k|) in index_set order."""
    d = np.asarray(xhat).shape[1]
    return np.stack([harmonic(k, ch, xhat) for ch in index_set(k, d)], axis=1)
