"""Pins of the oracle's kernel formulas (Sec. 4.1) and of their derivatives (no GPU).

The Matern kernels of Sec. 4.1 (nu = 3/2, 5/2) are special cases of the general Matern form
    k_nu(r) = 2^(1-nu) / Gamma(nu) * u^nu K_nu(u),   u = sqrt(2 nu) r / l,
with K_nu the modified Bessel function of the second kind.  The oracle writes the two
half-integer cases in closed form; here they are checked against that general form through
scipy's Bessel routine, against values the definitions fix by hand, and their derivatives
against the Bessel identity d/du [u^nu K_nu(u)] = -u^nu K_(nu-1)(u) and against Richardson
central differences of the kernel itself.
"""
import math

import numpy as np
import pytest
from scipy.special import gamma, kv

from oracle import chebyshev, hdf, kernels
from paper_2202_03655_gb300 import workloads as W

MATERN_NU = {"matern32": 1.5, "matern52": 2.5}


def matern_bessel(nu, r, ell):
    """The general Matern kernel through K_nu (k(0) = 1 as the limit)."""
    r = np.asarray(r, dtype=np.float64)
    u = math.sqrt(2.0 * nu) * np.abs(r) / ell
    out = np.ones_like(u)
    pos = u > 0
    out[pos] = 2.0 ** (1.0 - nu) / gamma(nu) * u[pos] ** nu * kv(nu, u[pos])
    return out


def richardson_derivative(fn, x, h):
    """(4 D(h/2) - D(h)) / 3 with central differences D: error O(h^4)."""
    d1 = (fn(x + h) - fn(x - h)) / (2.0 * h)
    d2 = (fn(x + 0.5 * h) - fn(x - 0.5 * h)) / h
    return (4.0 * d2 - d1) / 3.0


@pytest.mark.parametrize("kname", sorted(MATERN_NU))
@pytest.mark.parametrize("ell", [0.3, 1.0, 2.5])
def test_matern_equals_bessel_form(kname, ell):
    r = np.linspace(0.0, 8.0, 801)
    ref = matern_bessel(MATERN_NU[kname], r, ell)
    assert np.allclose(kernels.kernel(kname, r, ell), ref, rtol=1e-12, atol=1e-15)


def test_kernel_values_fixed_by_the_definitions():
    """Hand values: k(0) = 1; Gaussian k(l) = e^(-1/2); Cauchy k(l) = 1/2;
    Matern-3/2 at r = l/sqrt3: (1 + 1) e^-1; Matern-5/2 at r = l/sqrt5: (1 + 1 + 1/3) e^-1."""
    ell = 1.7
    for k in kernels.KERNELS:
        assert kernels.kernel(k, 0.0, ell) == 1.0
    assert math.isclose(kernels.kernel("gaussian", ell, ell), math.exp(-0.5), rel_tol=1e-15)
    assert math.isclose(kernels.kernel("cauchy", ell, ell), 0.5, rel_tol=1e-15)
    assert math.isclose(kernels.kernel("matern32", ell / math.sqrt(3.0), ell), 2.0 / math.e, rel_tol=1e-14)
    assert math.isclose(kernels.kernel("matern52", ell / math.sqrt(5.0), ell), (7.0 / 3.0) / math.e, rel_tol=1e-14)
    # isotropic: the sign of r does not matter
    for k in kernels.KERNELS:
        assert kernels.kernel(k, -0.7, ell) == kernels.kernel(k, 0.7, ell)


@pytest.mark.parametrize("kname", sorted(MATERN_NU))
def test_matern_derivative_bessel_identity(kname):
    """dk/dz = -c_nu a (a z)^nu K_(nu-1)(a z), a = sqrt(2 nu), c_nu = 2^(1-nu)/Gamma(nu)."""
    nu = MATERN_NU[kname]
    a = math.sqrt(2.0 * nu)
    z = np.linspace(0.01, 6.0, 300)
    ref = -(2.0 ** (1.0 - nu) / gamma(nu)) * a * (a * z) ** nu * kv(nu - 1.0, a * z)
    assert np.allclose(kernels.kernel_dz(kname, z), ref, rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("kname", kernels.KERNELS)
def test_kernel_dz_and_dr_by_differences(kname):
    ell = 0.9
    z = np.linspace(0.05, 5.0, 120)
    fd = richardson_derivative(lambda t: kernels.kernel(kname, t, 1.0), z, 1e-3)
    assert np.allclose(kernels.kernel_dz(kname, z), fd, rtol=1e-8, atol=1e-11)
    r = z * ell
    fdr = richardson_derivative(lambda t: kernels.kernel(kname, t, ell), r, 1e-3)
    assert np.allclose(kernels.kernel_dr(kname, r, ell), fdr, rtol=1e-8, atol=1e-11)
    assert np.all(kernels.kernel_dz(kname, np.array([0.0])) == 0.0)


@pytest.mark.parametrize("kname", kernels.KERNELS)
def test_kernel_dell_by_differences(kname):
    r = np.linspace(0.0, 4.0, 81)
    for ell in (0.5, 1.3):
        fd = richardson_derivative(lambda e: kernels.kernel(kname, r, e), ell, 1e-3)
        assert np.allclose(kernels.kernel_dell(kname, r, ell), fd, rtol=1e-8, atol=1e-11)


@pytest.mark.parametrize("kname", kernels.KERNELS)
def test_adjoint_fd_matches_dense_gradient_every_kernel(kname):
    """The dense-kernel gradient (built on kernel_dr and kernel_dell) and the frozen-structure
    central differences (built on kernel values only) agree for every kernel.

    Bounds.  Differentiating the truncated expansion amplifies its error: the point gradient
    differs from the dense one by 20 to 30 times |K - K~|_F / |K|_F on these cases, so it is
    held to 100 times.  The l-derivative is checked on the factor that keeps every eigenpair,
    where its only error is the Chebyshev truncation of d kappa / d l at the build's p (the
    frozen eigenvectors of a truncated factor need not span d S / d l); it is held to 10 times
    that tail, taken from differences of the kernel's own coefficients.  A wrong constant or
    sign in a derivative formula gives an O(1) disagreement."""
    ell, n = 2.0, 40
    g = np.random.default_rng(8)
    x = W.uniform_cube(g, n, 4)
    v, w = g.standard_normal(n), g.standard_normal(n)
    gd, dld = hdf.dense_gradient(x, kname, ell, v, w)
    f = hdf.build(x, kname, ell, 1e-6, p_max=24)
    grad, _ = hdf.adjoint_fd(f, x, v, w)
    err = max(hdf.rel_fro_error(f, x, kname, ell), 1e-9)
    assert np.linalg.norm(grad - gd) / np.linalg.norm(gd) < 100.0 * err
    fa = hdf.build(x, kname, ell, 1e-6, p_max=24, keep_all=True)
    grad_a, dl = hdf.adjoint_fd(fa, x, v, w)
    err_a = max(hdf.rel_fro_error(fa, x, kname, ell), 1e-9)
    assert np.linalg.norm(grad_a - gd) / np.linalg.norm(gd) < 100.0 * err_a
    R, M, h = fa.plan.R, hdf.cheb_nodes_count(24), 1e-4
    coef = lambda e: chebyshev.cheb_coeffs(lambda r: kernels.kernel(kname, 2.0 * R * np.asarray(r), e), M)
    da = (coef(ell + h) - coef(ell - h)) / (2.0 * h)
    dtail = max(chebyshev.tail_sums(da)[fa.plan.p], 1e-12)
    assert abs(dl - dld) / abs(dld) < 10.0 * max(dtail, err_a)
