"""Isotropic kernels k(r; l) (Sec. 4.1) and their derivatives, in FP64 numpy.

Sec. 4.1 lists the Cauchy, Gaussian and Matern (nu = 1.5, 2.5) kernels with a
lengthscale sigma.  The Gaussian here uses the exp(-r^2 / (2 l^2)) convention of the
workloads this library targets (the paper writes exp(-(r/sigma)^2); that is the same
family with sigma = sqrt(2) l).  The other three follow Sec. 4.1 with sigma = l.
"""
import numpy as np

KERNELS = ("gaussian", "cauchy", "matern32", "matern52")
SQRT3 = np.sqrt(3.0)
SQRT5 = np.sqrt(5.0)


def _check(name):
    if name not in KERNELS:
        raise ValueError(f"unknown kernel {name!r}; expected one of {KERNELS}")


def kernel(name, r, ell):
    """k(|r|; ell) for the kernels of Sec. 4.1 (Gaussian in the exp(-r^2/(2 l^2)) form)."""
    _check(name)
    z = np.abs(np.asarray(r, dtype=np.float64)) / ell
    if name == "gaussian":
        return np.exp(-0.5 * z * z)
    if name == "cauchy":
        return 1.0 / (1.0 + z * z)
    if name == "matern32":
        s = SQRT3 * z
        return (1.0 + s) * np.exp(-s)
    s = SQRT5 * z
    return (1.0 + s + s * s / 3.0) * np.exp(-s)


def kernel_dz(name, z):
    """d k / d z as a function of z = r / ell (z >= 0)."""
    _check(name)
    z = np.asarray(z, dtype=np.float64)
    if name == "gaussian":
        return -z * np.exp(-0.5 * z * z)
    if name == "cauchy":
        return -2.0 * z / (1.0 + z * z) ** 2
    if name == "matern32":
        s = SQRT3 * z
        return -3.0 * z * np.exp(-s)
    s = SQRT5 * z
    return -(5.0 / 3.0) * z * (1.0 + s) * np.exp(-s)


def kernel_dr(name, r, ell):
    """d k(r; ell) / d r."""
    return kernel_dz(name, np.abs(r) / ell) / ell


def kernel_dell(name, r, ell):
    """d k(r; ell) / d ell = k'(z) * (-z / ell) with z = r / ell."""
    z = np.abs(np.asarray(r, dtype=np.float64)) / ell
    return kernel_dz(name, z) * (-z / ell)
