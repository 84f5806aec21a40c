"""Seeded synthetic inputs shaped like the method's workloads.

Only random inputs live here: no step of the factorization is computed in this module.
Both the CUDA path (through tests and bench.py) and the CPU oracle (through tests) are
fed the same arrays from these generators.  Every generator takes a numpy Generator;
``rng(idx)`` seeds PCG64 with 20220207 + idx for workload number idx.

Workloads (Sec. 4 uses normal points scaled to maximum norm 1; the shapes below widen
that to the point distributions the factorization is expected to meet):

  0  ball3_gauss      n=2,000, d=3, uniform in the unit ball, Gaussian l=0.5, tol 1e-6
  1  mixture3_matern  n=1,000,000, d=3, 8-component isotropic Gaussian mixture
                      (means U[-2,2]^3, sigma 0.3, equal weights), Matern-3/2 l=1, tol 1e-8,
                      V with 64 N(0,1) columns
  2  normal5_cauchy   n=4,000,000, d=5, N(0,I) rotated by a random orthogonal matrix and
                      standardised per dimension, Cauchy l=2, tol 1e-4, V with 16 columns
  3  cube4_gauss      n=500,000, d=4, uniform in [-1,1]^4, Gaussian l=0.8, tol 1e-6
  4  batch512_gauss   512 sets, n log-uniform in [1000, 65536], d=3, uniform in a ball of
                      radius U[0.5, 2], Gaussian l ~ U[0.3, 1.5], tol 1e-6, V with 8 columns
  5  fig1_cauchy      the time-vs-n workload of Sec. 4.1 / Fig. 1: N(0,I) points scaled to max
                      norm 1, d in {3, 4, 5, 6}, n from 10^4 to 10^7, Cauchy sigma = l = 1,
                      tol 1e-3 (the figure's caption; the text says 0.005)
  7  fig3_rank5       the error-vs-rank workload of Sec. 4.1 / Fig. 3: 5,000 points in d = 5
                      generated as workload 5, the four kernels with sigma = 1 (the Gaussian in
                      the paper's exp(-(r/sigma)^2) form, i.e. l = 1/sqrt(2) here), tolerances
                      from 1e-1 to 1e-7
  8  krr8_clusters    the kernel-ridge-regression row (Sec. 4.2) on synthetic data shaped like
                      its dataset (20,640 points, 8 features scaled to [0, 1], a 2/3 - 1/3
                      train/test split): a 24-component mixture with anisotropic spreads,
                      targets = a random smooth function (four random plane waves) plus noise;
                      30 k-means clusters from seeded initial centres; Gaussian l = 0.5,
                      lambda = 1, HDF blocks at tol 1e-3 (lambda above tol max_i |K_ii|_F keeps
                      lambda I + K^ positive definite)
  6  cross3_gauss     the non-symmetric row K(X, Y): X = 1,000,000 points of the 8-component
                      mixture of workload 1, Y = 250,000 points of N(0, 1.2^2 I) (a wider
                      cloud around them: off-diagonal and cross-kernel blocks, Sec. 2 and 5),
                      Gaussian l=1.5, tol 1e-6, V and W with 16 N(0,1) columns
"""
import numpy as np

SEED_BASE = 20220207


def rng(idx):
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(idx)))


def uniform_ball(g, n, d, radius=1.0):
    """Uniform in the d-ball: direction = normalised N(0, I), radius * U^(1/d)."""
    dirs = g.standard_normal((n, d))
    nrm = np.linalg.norm(dirs, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return radius * dirs / nrm * g.random((n, 1)) ** (1.0 / d)


def gaussian_mixture(g, n, d=3, components=8, lo=-2.0, hi=2.0, sigma=0.3):
    """Equal-weight isotropic Gaussian mixture with means uniform in [lo, hi]^d."""
    means = g.uniform(lo, hi, size=(components, d))
    lab = g.integers(0, components, size=n)
    return means[lab] + sigma * g.standard_normal((n, d))


def rotated_standard_normal(g, n, d=5):
    """N(0, I) times a random orthogonal matrix (QR of a Gaussian), standardised per dimension."""
    Q, R = np.linalg.qr(g.standard_normal((d, d)))
    Q = Q * np.sign(np.diag(R))[None, :]
    x = g.standard_normal((n, d)) @ Q
    x -= x.mean(axis=0)
    x /= x.std(axis=0)
    return x


def uniform_cube(g, n, d=4):
    return g.uniform(-1.0, 1.0, size=(n, d))


def normal_maxnorm1(g, n, d):
    """N(0, I) scaled so that the largest norm is 1 (Sec. 4.1)."""
    x = g.standard_normal((n, d))
    return x / np.linalg.norm(x, axis=1).max()


def vectors(g, n, c):
    """c columns of N(0,1), column-major as an (n, c) Fortran-ordered array."""
    return np.asfortranarray(g.standard_normal((n, c)))


def batch_sets(g, nsets=512, nmin=1000, nmax=65536, d=3):
    """Ragged sets: sizes log-uniform in [nmin, nmax], radius U[0.5, 2], lengthscale U[0.3, 1.5].

    Returns (x concatenated (sum n, d), offsets (nsets+1,), lengthscales (nsets,))."""
    sizes = np.floor(np.exp(g.uniform(np.log(nmin), np.log(nmax), size=nsets))).astype(np.int64)
    radii = g.uniform(0.5, 2.0, size=nsets)
    ells = g.uniform(0.3, 1.5, size=nsets)
    xs = [uniform_ball(g, int(m), d, r) for m, r in zip(sizes, radii)]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(xs, axis=0), offsets, ells


WORKLOADS = {
    "ball3_gauss": dict(idx=0, n=2000, d=3, kernel="gaussian", ell=0.5, tol=1e-6, ncols=1),
    "mixture3_matern": dict(idx=1, n=1_000_000, d=3, kernel="matern32", ell=1.0, tol=1e-8, ncols=64),
    "normal5_cauchy": dict(idx=2, n=4_000_000, d=5, kernel="cauchy", ell=2.0, tol=1e-4, ncols=16),
    "cube4_gauss": dict(idx=3, n=500_000, d=4, kernel="gaussian", ell=0.8, tol=1e-6, ncols=1),
    "batch512_gauss": dict(idx=4, nsets=512, d=3, kernel="gaussian", tol=1e-6, ncols=8),
    "fig1_cauchy": dict(idx=5, n=10_000_000, d=3, dims=(3, 4, 5, 6), sizes=(10_000, 100_000, 1_000_000, 10_000_000),
                        kernel="cauchy", ell=1.0, tol=1e-3, ncols=1),
    "fig3_rank5": dict(idx=7, n=5000, d=5, kernels=(("cauchy", 1.0), ("gaussian", 0.5 ** 0.5), ("matern32", 1.0),
                                                   ("matern52", 1.0)),
                       tols=(1e-1, 3e-2, 1e-2, 3e-3, 1e-3, 3e-4, 1e-4, 1e-5, 1e-6, 1e-7), kernel="cauchy", ell=1.0,
                       tol=1e-3, ncols=1),
    "krr8_clusters": dict(idx=8, n=20640, d=8, kernel="gaussian", ell=0.5, lam=1.0, tol=1e-3, clusters=30,
                          components=24, ncols=1),
    "cross3_gauss": dict(idx=6, n=1_000_000, n_y=250_000, d=3, kernel="gaussian", ell=1.5, tol=1e-6,
                         ncols=16),
}


def cross_sets(name="cross3_gauss", m=None, n=None):
    """(X, Y) of a two-set workload: X from the mixture, Y from N(0, 1.2^2 I)."""
    w = WORKLOADS[name]
    m = w["n"] if m is None else int(m)
    n = w["n_y"] if n is None else int(n)
    g = rng(w["idx"])
    x = gaussian_mixture(g, m, w["d"])
    y = g.standard_normal((n, w["d"])) * 1.2
    return x, y


def points(name, n=None, idx=None):
    """Points of a named workload (optionally with a smaller n, same distribution)."""
    w = WORKLOADS[name]
    n = w["n"] if n is None else int(n)
    g = rng(w["idx"] if idx is None else idx)
    if name == "ball3_gauss":
        return uniform_ball(g, n, 3)
    if name == "mixture3_matern":
        return gaussian_mixture(g, n, 3)
    if name == "normal5_cauchy":
        return rotated_standard_normal(g, n, 5)
    if name == "cube4_gauss":
        return uniform_cube(g, n, 4)
    raise ValueError(name)


def maxnorm1_points(name, n, d):
    """Points of the Sec. 4.1 workloads (fig1_cauchy, fig3_rank5): N(0, I) scaled to max norm 1,
    one seeded stream per (workload, d)."""
    w = WORKLOADS[name]
    return normal_maxnorm1(rng(w["idx"] * 100 + d), int(n), d)


def krr_data(name="krr8_clusters", n=None):
    """(x_train, y_train, x_test, y_test, init_idx) of the regression workload: features are
    min-max scaled to [0, 1]; init_idx are distinct training indices for the k-means centres."""
    w = WORKLOADS[name]
    n = w["n"] if n is None else int(n)
    d, q = w["d"], w["components"]
    g = rng(w["idx"])
    means = g.uniform(0.2, 0.8, size=(q, d))
    spreads = g.uniform(0.03, 0.12, size=(q, d))
    weights = g.dirichlet(np.full(q, 2.0))
    comp = g.choice(q, size=n, p=weights)
    x = means[comp] + spreads[comp] * g.standard_normal((n, d))
    x = (x - x.min(axis=0)) / (x.max(axis=0) - x.min(axis=0))
    dirs = g.standard_normal((4, d))
    freqs = g.uniform(1.0, 3.0, size=4)
    phases = g.uniform(0.0, 2 * np.pi, size=4)
    amps = g.uniform(0.5, 1.5, size=4)
    y = (amps[None, :] * np.sin(freqs[None, :] * (x @ dirs.T) + phases[None, :])).sum(axis=1)
    y = y + 0.1 * g.standard_normal(n)
    perm = g.permutation(n)
    ntr = (2 * n) // 3
    tr, te = perm[:ntr], perm[ntr:]
    init = g.choice(ntr, size=w["clusters"], replace=False)
    return x[tr], y[tr], x[te], y[te], np.sort(init).astype(np.int64)

