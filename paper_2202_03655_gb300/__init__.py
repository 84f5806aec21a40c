"""GB300-native Harmonic Decomposition Factorization (Ryan & Damle, ICML 2022).

The compute path is the C-ABI library ``libhdf.so`` built from ``csrc/`` (hand-written
sm_103a CUDA kernels plus a C++ host planner); ``hdf`` is its thin ctypes binding and
``autograd`` wraps the adjoint in a ``torch.autograd.Function``.  ``workloads`` holds the
seeded synthetic input generators.  Submodules are imported on first use so that the
input generators can be used without loading the CUDA library.
"""
import importlib

__all__ = ["hdf", "autograd", "workloads", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
