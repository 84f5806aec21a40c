"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test checks an oracle function against something other than itself: a closed form,
a library routine on a special case, an identity the paper states, a brute-force sum, or
the paper's error-versus-tolerance claim.
"""
import numpy as np
import pytest
from scipy.special import eval_chebyu, eval_legendre, ive, roots_gegenbauer

from oracle import chebyshev, gegenbauer as G, harmonics, hdf, kernels, radial
from paper_2202_03655_gb300 import workloads as W


# --------------------------------------------------------------------------- Chebyshev

@pytest.mark.parametrize("c", [0.5, 2.0, 4.0, 8.0])
def test_cheb_gaussian_closed_form(c):
    """exp(-beta r^2) has a_{2q} = 2 (-1)^q e^{-beta/2} I_q(beta/2) (generating function of I_q)."""
    beta = 0.5 * c * c
    a = chebyshev.cheb_coeffs(lambda r: np.exp(-beta * r * r), 200)
    q = np.arange(40)
    ref = 2.0 * (-1.0) ** q * ive(q, beta / 2.0)
    ref[0] *= 0.5
    assert np.allclose(a[0:80:2], ref, rtol=0, atol=1e-14)
    assert np.all(a[1::2] == 0.0)


@pytest.mark.parametrize("c", [0.5, 3.0, 6.5])
def test_cheb_cauchy_closed_form(c):
    """1/(1+c^2 r^2) = (1/sqrt(1+c^2)) [1 + 2 sum_q (-z)^q T_{2q}(r)], z = (sqrt(1+c^2)-1)^2/c^2."""
    a = chebyshev.cheb_coeffs(lambda r: 1.0 / (1.0 + c * c * r * r), 400)
    s = np.sqrt(1.0 + c * c)
    z = (s - 1.0) ** 2 / (c * c)
    q = np.arange(60)
    ref = 2.0 * (-z) ** q / s
    ref[0] *= 0.5
    assert np.allclose(a[0:120:2], ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("kname", kernels.KERNELS)
def test_cheb_truncation_error_within_tail(kname):
    """max |kappa - sum_{i<=p} a_i T_i| <= sum_{i>p} |a_i| on a 10^4-point grid (Sec. 3.5)."""
    kap = lambda r: kernels.kernel(kname, 5.0 * r, 1.0)
    a = chebyshev.cheb_coeffs(kap, 600)
    r = np.linspace(-1, 1, 10001)
    for p in (10, 20, 40):
        ap = a.copy()
        ap[p + 1:] = 0.0
        err = np.abs(kap(np.abs(r)) - chebyshev.cheb_eval(ap, r)).max()
        assert err <= chebyshev.tail_sums(a)[p] * (1 + 1e-9) + 1e-15


def test_cheb_elliott_paget_gaussian():
    """Sec. 3.5's bound |tail| <= max|k^(p+1)| / (2^p (p+1)!) for a Gaussian (derivatives of
    exp(-r^2/2) are bounded by sqrt((p+1)!) times exp's Hermite envelope < (p+1)!^(1/2) 1.09)."""
    kap = lambda r: np.exp(-0.5 * (2.0 * r) ** 2)
    a = chebyshev.cheb_coeffs(kap, 400)
    r = np.linspace(-1, 1, 4001)
    from math import factorial, sqrt
    for p in (8, 12, 16):
        ap = a.copy()
        ap[p + 1:] = 0.0
        err = np.abs(kap(np.abs(r)) - chebyshev.cheb_eval(ap, r)).max()
        # |d^m/dr^m e^{-2 r^2}| = 2^m |He_m(2r) e^{-2r^2}| <= 2^m 1.09 sqrt(m!)  (Cramer's bound)
        m = p + 1
        bound = 2.0 ** m * 1.09 * sqrt(factorial(m)) / (2.0 ** p * factorial(m))
        assert err <= bound


def test_monomial_coeffs_match_trig_definition():
    """T_i(r) = sum_j t_ij r^j reproduces cos(i arccos r) (Eq. chebdef, corrected start)."""
    t = chebyshev.monomial_coeffs(20)
    r = np.linspace(-1, 1, 101)
    for i in range(21):
        poly = sum(t[i][j] * r ** j for j in range(i + 1))
        assert np.allclose(poly, np.cos(i * np.arccos(r)), atol=1e-9)
    assert t[6][6] == 32 and t[6][0] == -1


def test_choose_degree_is_smallest_even():
    a = np.zeros(50)
    a[0:50:2] = 0.5 ** np.arange(25)
    p, tail, ok = chebyshev.choose_degree(a, 1e-3, 40)
    assert ok and p % 2 == 0
    tails = chebyshev.tail_sums(a)
    assert tail <= 1e-3 and (p == 0 or tails[p - 2] > 1e-3)
    p2, tail2, ok2 = chebyshev.choose_degree(a, 1e-30, 10)
    assert not ok2 and p2 == 10


# ------------------------------------------------------------------------- Gegenbauer

@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5, 2.5])
def test_cos_power_gegenbauer_identity(alpha):
    """cos^i g = sum_k A_ki C_k^alpha(cos g) (App. A), checked by evaluation."""
    t = np.linspace(-1, 1, 37)
    for i in range(0, 16):
        rhs = sum(G.A_coeff(k, i, alpha) * G.gegenbauer(k, alpha, t) for k in range(i + 1))
        assert np.allclose(rhs, t ** i, atol=1e-12)


def test_gegenbauer_special_cases():
    """C^{1/2} = Legendre, C^1 = Chebyshev U (library special cases)."""
    t = np.linspace(-1, 1, 21)
    for n in range(12):
        assert np.allclose(G.gegenbauer(n, 0.5, t), eval_legendre(n, t), atol=1e-12)
        assert np.allclose(G.gegenbauer(n, 1.0, t), eval_chebyu(n, t), atol=1e-12)


@pytest.mark.parametrize("lam", [0.5, 1.0, 2.5, 7.5])
def test_gegen_norm_by_quadrature(lam):
    t, w = roots_gegenbauer(40, lam)
    for n in range(15):
        assert np.isclose((G.gegenbauer(n, lam, t) ** 2 * w).sum(), G.gegen_norm(n, lam), rtol=1e-12)


# ------------------------------------------------------------------------- harmonics

@pytest.mark.parametrize("d", [3, 4, 5, 6])
def test_harmonic_counts(d):
    """|H_k| by enumeration equals App. B's binomial formula; totals telescope (App. B)."""
    tot = 0
    for k in range(9):
        cnt = len(harmonics.index_set(k, d))
        assert cnt == G.harmonic_count(k, d)
        tot += cnt
        assert tot == G.harmonic_total(k, d)


def _sphere_quadrature(d, npts):
    """Exact product quadrature on S^{d-1}: Gauss-Gegenbauer in each cos(theta_j), trapezoid in phi."""
    grids, weights = [], []
    for j in range(d - 2):
        a_j = (d - j - 2) / 2.0
        t, w = roots_gegenbauer(npts, a_j)
        grids.append(np.arccos(t))
        weights.append(w)
    nphi = 2 * npts + 1
    phi = 2 * np.pi * np.arange(nphi) / nphi
    mesh = np.meshgrid(*grids, phi, indexing="ij")
    wmesh = np.meshgrid(*weights, np.full(nphi, 2 * np.pi / nphi), indexing="ij")
    wt = np.prod(np.stack([m.ravel() for m in wmesh]), axis=0)
    th = [m.ravel() for m in mesh[:-1]]
    ph = mesh[-1].ravel()
    # rebuild Cartesian coordinates from the angles (coordinate d-1-j peeled at level j)
    N = ph.size
    x = np.zeros((N, d))
    s = np.ones(N)
    for j in range(d - 2):
        x[:, d - 1 - j] = s * np.cos(th[j])
        s = s * np.sin(th[j])
    x[:, 0] = s * np.cos(ph)
    x[:, 1] = s * np.sin(ph)
    return x, wt


@pytest.mark.parametrize("d", [3, 4, 5])
def test_harmonics_orthonormal(d):
    """int_{S^{d-1}} Y_a Y_b = delta_ab under an exact product quadrature."""
    x, w = _sphere_quadrature(d, 9)
    Y = np.concatenate([harmonics.harmonics_block(k, x) for k in range(6)], axis=1)
    gram = (Y * w[:, None]).T @ Y
    assert np.abs(gram - np.eye(gram.shape[0])).max() < 1e-11


@pytest.mark.parametrize("d", [3, 4, 5, 7])
def test_addition_theorem(d):
    """sum_h Y_k^h(x) Y_k^h(y) = C_k^alpha(x.y) / Z_k (Eq. additiontheorem)."""
    g = np.random.default_rng(5)
    X = harmonics.directions(g.standard_normal((20, d)))
    Yv = harmonics.directions(g.standard_normal((20, d)))
    alpha = d / 2.0 - 1.0
    for k in range(10):
        lhs = (harmonics.harmonics_block(k, X) * harmonics.harmonics_block(k, Yv)).sum(axis=1)
        rhs = G.inv_Z(k, d) * G.gegenbauer(k, alpha, (X * Yv).sum(axis=1))
        assert np.allclose(lhs, rhs, atol=1e-12 * max(1.0, np.abs(rhs).max()))


def test_d3_textbook_spherical_harmonics():
    """d = 3: Y_0 = 1/(2 sqrt(pi)), Y_1^0 = sqrt(3/(4 pi)) z, Y_2^0 = sqrt(5/(16 pi)) (3z^2 - 1),
    Y_1^{+1} = sqrt(3/(4 pi)) x, Y_1^{-1} = sqrt(3/(4 pi)) y (real basis)."""
    g = np.random.default_rng(3)
    X = harmonics.directions(g.standard_normal((10, 3)))
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    assert np.allclose(harmonics.harmonic(0, (0,), X), 0.5 / np.sqrt(np.pi))
    assert np.allclose(harmonics.harmonic(1, (0,), X), np.sqrt(3 / (4 * np.pi)) * z)
    assert np.allclose(harmonics.harmonic(1, (1,), X), np.sqrt(3 / (4 * np.pi)) * x)
    assert np.allclose(harmonics.harmonic(1, (-1,), X), np.sqrt(3 / (4 * np.pi)) * y)
    assert np.allclose(harmonics.harmonic(2, (0,), X), np.sqrt(5 / (16 * np.pi)) * (3 * z * z - 1))


# ---------------------------------------------------------------------------- radial

@pytest.mark.parametrize("kname,ell", [("gaussian", 0.8), ("cauchy", 1.0), ("matern52", 1.5)])
@pytest.mark.parametrize("d", [3, 4, 5])
def test_literal_equals_stable_route(kname, ell, d):
    """App. A's closed form T'' (mpmath) and the Gegenbauer-projection core agree (T3)."""
    pytest.importorskip("mpmath")
    g = np.random.default_rng(11)
    x = g.standard_normal((64, d))
    _, pl = hdf.plan(x, kname, ell, 1e-6, p_max=32)
    Tpp, ctx = radial.literal_core(pl.a, pl.p, d)
    cores = radial.stable_core(pl.a, pl.p, d)
    ab = g.random((12, 2)) * 0.5
    scale = max(abs(radial.literal_r(Tpp, ctx, 0, 0.5, 0.5)), 1.0)
    for k in range(pl.L + 1):
        lit = np.array([radial.literal_r(Tpp, ctx, k, a_, b_) for a_, b_ in ab])
        st = radial.stable_r(cores, k, ab[:, 0], ab[:, 1])
        assert np.abs(lit - st).max() <= 1e-12 * scale


@pytest.mark.parametrize("d", [3, 4, 5])
@pytest.mark.parametrize("kname", ["gaussian", "cauchy", "matern32"])
def test_expansion_brute_force(d, kname):
    """Without compression, U S U^T reproduces the truncated series sum_{i<=p} a_i T_i(|x_i - x_j|)
    to rounding (T1: the derivation of Sec. 3.3 / App. A is exact)."""
    g = np.random.default_rng(7 + d)
    x = g.standard_normal((14, d))
    for p in (6, 12):
        f = hdf.build(x, kname, 1.3, 1e-6, keep_all=True, p=p)
        xs, pl = hdf.plan(x, kname, 1.3, 1e-6)
        D = np.sqrt(((xs[:, None] - xs[None]) ** 2).sum(-1))
        a = pl.a.copy()
        a[p + 1:] = 0.0
        Fm = chebyshev.cheb_eval(a, D)
        assert np.abs((f.U * f.S) @ f.U.T - Fm).max() <= 1e-12 * np.abs(Fm).max()


def test_literal_pipeline_brute_force():
    """Algorithm 1 literally (per-k power-basis QR, App. A core) on a tiny benign case."""
    pytest.importorskip("mpmath")
    g = np.random.default_rng(2)
    x = g.standard_normal((14, 3))
    f = hdf.build_literal(x, "gaussian", 2.0, 1e-6, keep_all=True, p=8)
    xs, pl = hdf.plan(x, "gaussian", 2.0, 1e-6)
    D = np.sqrt(((xs[:, None] - xs[None]) ** 2).sum(-1))
    a = pl.a.copy()
    a[9:] = 0.0
    Fm = chebyshev.cheb_eval(a, D)
    assert np.abs((f.U * f.S) @ f.U.T - Fm).max() <= 1e-11 * np.abs(Fm).max()


# -------------------------------------------------------------------------- pipeline

def test_scaling_properties():
    x = W.points("mixture3_matern", n=5000)
    xs, c, R = hdf.center_scale(x)
    assert np.sqrt((xs ** 2).sum(1)).max() == pytest.approx(0.5)
    assert np.allclose(xs * 2 * R + c, x)


def test_mean_square_exact_small():
    g = np.random.default_rng(0)
    x = g.standard_normal((300, 3))
    xs, c, R = hdf.center_scale(x)
    K = hdf.dense_kernel(x, "cauchy", 0.7)
    kap = lambda r: kernels.kernel("cauchy", 2 * R * r, 0.7)
    assert hdf.mean_square_kernel(xs, kap) == pytest.approx(np.mean(K ** 2), rel=1e-12)


@pytest.mark.parametrize("kname,ell,tols", [("gaussian", 0.5, (1e-2, 1e-4, 1e-6)),
                                             ("cauchy", 0.5, (1e-2, 1e-4, 1e-6)),
                                             ("matern52", 1.0, (1e-2, 1e-3, 1e-4))])
def test_error_tracks_tolerance(kname, ell, tols):
    """|K - U S U^T|_F / |K|_F <= tol and falls as tol falls (abstract; Remark 3; T5)."""
    x = W.points("ball3_gauss")
    errs, ranks = [], []
    for tol in tols:
        f = hdf.build(x, kname, ell, tol)
        assert f.plan.reached
        e = hdf.rel_fro_error(f, x, kname, ell)
        assert e <= tol
        # the a-priori bound behind the truncation rule holds as well
        errs.append(e)
        ranks.append(f.rank)
    assert errs[0] > errs[1] > errs[2]
    assert ranks[0] < ranks[1] < ranks[2]


def test_truncation_budget_respected():
    x = W.points("ball3_gauss", n=800)
    f = hdf.build(x, "gaussian", 0.5, 1e-5)
    full = hdf.build(x, "gaussian", 0.5, 1e-5, keep_all=True)
    area = G.sphere_area(3)
    kept = {(b["k"], round(float(l), 12)) for b in f.blocks for l in b["lam"]}
    dropped = 0.0
    for b in full.blocks:
        for l in b["lam"]:
            if (b["k"], round(float(l), 12)) not in kept:
                dropped += abs(l) * G.harmonic_count(b["k"], 3) / area
    assert dropped <= f.plan.drop_budget * (1 + 1e-12)
    # |K - K~|_F <= n * tail + dropped cost (the bound the two budgets split)
    K = hdf.dense_kernel(x, "gaussian", 0.5)
    err = np.linalg.norm(K - (f.U * f.S) @ f.U.T)
    assert err <= x.shape[0] * f.plan.tail + dropped + 1e-9


def test_solve_dense_and_woodbury_agree():
    g = np.random.default_rng(4)
    x = g.standard_normal((400, 3))
    f = hdf.build(x, "gaussian", 1.0, 1e-8)
    B = g.standard_normal((400, 2))
    X1 = hdf.solve(f, 0.1, B)
    core = 0.1 * np.diag(1.0 / f.S) + f.U.T @ f.U
    X2 = (B - f.U @ np.linalg.solve(core, f.U.T @ B)) / 0.1
    assert np.allclose(X1, X2, rtol=1e-7, atol=1e-9)
    assert np.allclose(0.1 * X1 + hdf.matvec(f, X1), B, atol=1e-9)


def test_adjoint_fd_matches_dense_gradient():
    """Frozen-structure gradient (central differences) agrees with the exact kernel gradient
    within the approximation's slack."""
    g = np.random.default_rng(8)
    x = W.uniform_cube(g, 60, 4)
    f = hdf.build(x, "gaussian", 0.8, 1e-9)
    v, w = g.standard_normal(60), g.standard_normal(60)
    grad, dl = hdf.adjoint_fd(f, x, v, w)
    gd, dld = hdf.dense_gradient(x, "gaussian", 0.8, v, w)
    assert np.linalg.norm(grad - gd) / np.linalg.norm(gd) < 1e-5
    assert abs(dl - dld) / abs(dld) < 1e-5
