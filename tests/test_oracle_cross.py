"""Pins of the non-symmetric oracle (Algorithm 1, K(X, Y) ~= U S V^T) against facts fixed by
the paper and by mathematics (no GPU): the truncated Chebyshev series by brute force, the
symmetric factor (Remark 1) when X = Y, transposition, translation invariance, the dense
cross-kernel error against the tolerance, and the truncation budget."""
import numpy as np
import pytest

from oracle import chebyshev, cross, gegenbauer as G, hdf
from paper_2202_03655_gb300 import workloads as W


def _pair(seed, m, n, d, shift=0.7):
    g = np.random.default_rng(seed)
    x = W.uniform_ball(g, m, d, 1.0)
    y = g.standard_normal((n, d)) * 0.6 + shift
    return x, y


def test_joint_scaling_bounds_every_cross_distance():
    x, y = _pair(1, 300, 170, 4)
    xs, ys, c, R = cross.center_scale_xy(x, y)
    assert max(np.sqrt((xs ** 2).sum(1)).max(), np.sqrt((ys ** 2).sum(1)).max()) == pytest.approx(0.5)
    D = np.sqrt(((xs[:, None] - ys[None]) ** 2).sum(-1))
    assert D.max() <= 1.0 + 1e-15
    assert np.allclose(xs * 2 * R + c, x) and np.allclose(ys * 2 * R + c, y)
    assert np.allclose(c, np.concatenate([x, y]).mean(0))


def test_cross_mean_square_exact_small():
    x, y = _pair(2, 200, 90, 3)
    xs, ys, c, R = cross.center_scale_xy(x, y)
    K = cross.dense_kernel_xy(x, y, "cauchy", 0.7)
    kap = lambda r: hdf.kernel("cauchy", 2 * R * r, 0.7)
    assert cross.mean_square_kernel_xy(xs, ys, kap) == pytest.approx(np.mean(K ** 2), rel=1e-12)


@pytest.mark.parametrize("d", [3, 4, 5])
@pytest.mark.parametrize("kname", ["gaussian", "cauchy", "matern32"])
def test_cross_expansion_brute_force(d, kname):
    """Without compression, U S V^T equals sum_{i<=p} a_i T_i(|x'_i - y'_j|) to rounding (the
    derivation of Sec. 3.3 / App. A holds for any pair of points within distance 1)."""
    x, y = _pair(10 + d, 9, 13, d)
    for p in (6, 12):
        f = cross.build_xy(x, y, kname, 1.3, 1e-6, keep_all=True, p=p)
        xs, ys, pl = cross.plan_xy(x, y, kname, 1.3, 1e-6)
        D = np.sqrt(((xs[:, None] - ys[None]) ** 2).sum(-1))
        a = pl.a.copy()
        a[p + 1:] = 0.0
        Fm = chebyshev.cheb_eval(a, D)
        assert np.abs((f.U * f.S) @ f.V.T - Fm).max() <= 1e-12 * np.abs(Fm).max()


@pytest.mark.parametrize("kname,ell,tol", [("gaussian", 0.5, 1e-6), ("cauchy", 1.0, 1e-4)])
def test_cross_equals_symmetric_when_x_is_y(kname, ell, tol):
    """X = Y: the SVD of the symmetric R Gamma_k R^T has sigma = |lambda| (Remark 1), the joint
    scaling and the budgets coincide with the symmetric ones, so the same pairs are kept and
    U S V^T = U S U^T of the symmetric factor."""
    x = W.points("ball3_gauss", n=600)
    fc = cross.build_xy(x, x, kname, ell, tol)
    fs = hdf.build(x, kname, ell, tol)
    assert fc.plan.p == fs.plan.p
    assert fc.plan.drop_budget == pytest.approx(fs.plan.drop_budget, rel=1e-12)
    for bc, bs in zip(fc.blocks, fs.blocks):
        assert bc["s"] == bs["s"]
        assert np.allclose(np.sort(bc["sig"]), np.sort(np.abs(bs["lam"])), rtol=1e-9, atol=1e-14)
    Kc = (fc.U * fc.S) @ fc.V.T
    Ks = (fs.U * fs.S) @ fs.U.T
    assert np.abs(Kc - Ks).max() <= 1e-10 * np.abs(Ks).max()


def test_cross_transpose():
    """build_xy(Y, X) approximates K_YX = K_XY^T with the same singular values."""
    x, y = _pair(3, 400, 250, 4)
    f = cross.build_xy(x, y, "gaussian", 0.8, 1e-6)
    g = cross.build_xy(y, x, "gaussian", 0.8, 1e-6)
    assert f.rank == g.rank
    assert np.allclose(np.sort(f.S), np.sort(g.S), rtol=1e-9)
    Kf = (f.U * f.S) @ f.V.T
    Kg = (g.U * g.S) @ g.V.T
    assert np.abs(Kf - Kg.T).max() <= 1e-10 * np.abs(Kf).max()
    v = np.random.default_rng(0).standard_normal((400, 2))
    assert np.allclose(cross.matvec_xy_t(f, v), cross.matvec_xy(g, v), rtol=0, atol=1e-10 * np.abs(v).sum())


def test_cross_translation_invariant():
    """Shifting both sets by one vector moves the joint centre with them: K~ is unchanged."""
    x, y = _pair(4, 300, 200, 3)
    t = np.array([3.0, -1.0, 0.5])
    f = cross.build_xy(x, y, "matern52", 1.0, 1e-5)
    g = cross.build_xy(x + t, y + t, "matern52", 1.0, 1e-5)
    Kf = (f.U * f.S) @ f.V.T
    Kg = (g.U * g.S) @ g.V.T
    assert f.rank == g.rank
    assert np.abs(Kf - Kg).max() <= 1e-10 * np.abs(Kf).max()


@pytest.mark.parametrize("kname,ell,tols", [("gaussian", 0.5, (1e-2, 1e-4, 1e-6)),
                                             ("cauchy", 1.5, (1e-2, 1e-4, 1e-6)),
                                             ("matern52", 1.5, (1e-2, 1e-3, 1e-4))])
def test_cross_error_tracks_tolerance(kname, ell, tols):
    """|K_XY - U S V^T|_F / |K_XY|_F <= tol and falls as tol falls (abstract; Remark 3)."""
    x, y = _pair(5, 700, 450, 3, shift=0.4)
    errs, ranks = [], []
    for tol in tols:
        f = cross.build_xy(x, y, kname, ell, tol)
        assert f.plan.reached
        e = cross.rel_fro_error_xy(f, x, y, kname, ell)
        assert e <= tol
        errs.append(e)
        ranks.append(f.rank)
    assert errs[0] > errs[1] > errs[2]
    assert ranks[0] < ranks[1] < ranks[2]


def test_cross_truncation_budget_and_bound():
    """The dropped cost stays within the budget, and |K - K~|_F <= sqrt(mn) tail + dropped."""
    x, y = _pair(6, 500, 300, 4)
    f = cross.build_xy(x, y, "gaussian", 0.6, 1e-5)
    full = cross.build_xy(x, y, "gaussian", 0.6, 1e-5, keep_all=True)
    area = G.sphere_area(4)
    dropped = 0.0
    for bf, bk in zip(full.blocks, f.blocks):
        kept = list(np.round(bk["sig"], 12))
        for s in bf["sig"]:
            key = np.round(s, 12)
            if key in kept:
                kept.remove(key)
            else:
                dropped += s * G.harmonic_count(bf["k"], 4) / area
    assert dropped <= f.plan.drop_budget * (1 + 1e-12)
    K = cross.dense_kernel_xy(x, y, "gaussian", 0.6)
    err = np.linalg.norm(K - (f.U * f.S) @ f.V.T)
    assert err <= np.sqrt(500.0 * 300.0) * f.plan.tail + dropped + 1e-9


def test_cross_rectangular_extremes():
    """One point against many, and a set smaller than the radial basis."""
    x, y = _pair(7, 1, 400, 3)
    f = cross.build_xy(x, y, "gaussian", 0.7, 1e-6)
    K = cross.dense_kernel_xy(x, y, "gaussian", 0.7)
    assert np.linalg.norm(K - (f.U * f.S) @ f.V.T) <= 1e-6 * np.linalg.norm(K)
    x, y = _pair(8, 5, 3, 5)
    f = cross.build_xy(x, y, "gaussian", 1.0, 1e-6)
    assert f.plan.reached and f.plan.L + 1 > 5             # more basis functions than points
    assert all(b["s"] <= 3 for b in f.blocks)               # rank of each R^(k) <= min(m, n)
    K = cross.dense_kernel_xy(x, y, "gaussian", 1.0)
    assert np.linalg.norm(K - (f.U * f.S) @ f.V.T) <= 1e-6 * np.linalg.norm(K)
