"""The seeded input generators produce the recipes the benchmark and the parity tests state
(shapes, scalings, determinism); no arithmetic of the method is involved."""
import numpy as np

from paper_2202_03655_gb300 import workloads as W


def test_generators_are_deterministic():
    a = W.points("cube4_gauss", n=1000)
    b = W.points("cube4_gauss", n=1000)
    assert np.array_equal(a, b)
    x1, y1 = W.cross_sets(m=500, n=200)
    x2, y2 = W.cross_sets(m=500, n=200)
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2)


def test_point_recipes():
    x = W.points("ball3_gauss")
    assert x.shape == (2000, 3) and np.linalg.norm(x, axis=1).max() <= 1.0
    c = W.points("cube4_gauss", n=5000)
    assert c.shape == (5000, 4) and np.abs(c).max() <= 1.0
    z = W.points("normal5_cauchy", n=20000)
    assert np.allclose(z.mean(axis=0), 0.0, atol=1e-12) and np.allclose(z.std(axis=0), 1.0)
    for d in (3, 6):
        f = W.maxnorm1_points("fig1_cauchy", 3000, d)
        assert f.shape == (3000, d) and np.isclose(np.linalg.norm(f, axis=1).max(), 1.0)


def test_batch_sets_recipe():
    x, off, ells = W.batch_sets(W.rng(4))
    sizes = np.diff(off)
    assert len(ells) == 512 and sizes.min() >= 1000 and sizes.max() <= 65536
    assert off[0] == 0 and off[-1] == len(x) and np.all((ells >= 0.3) & (ells <= 1.5))


def test_cross_and_regression_recipes():
    x, y = W.cross_sets()
    assert x.shape == (1_000_000, 3) and y.shape == (250_000, 3)
    xtr, ytr, xte, yte, init = W.krr_data()
    assert xtr.shape == (13760, 8) and xte.shape == (6880, 8)
    allx = np.concatenate([xtr, xte])
    assert np.isclose(allx.min(), 0.0) and np.isclose(allx.max(), 1.0)
    assert np.allclose(allx.min(axis=0), 0.0) and np.allclose(allx.max(axis=0), 1.0)
    assert len(init) == 30 and len(np.unique(init)) == 30 and init.max() < len(xtr)
