"""torch.autograd.Function around the HDF matvec and its adjoint.

``kernel_matvec(x, ell, v, ...)`` returns K~(x, ell) v, building the factor in the forward
pass.  Backward uses the library's adjoint (hdf_matvec_adjoint) under frozen-structure
semantics: the scaling, degree, radial-basis factor and kept eigenvectors of the forward
build are held fixed while differentiating.  The gradient with respect to v is K~ w
(K~ is symmetric).  All compute runs in libhdf.so.
"""
import torch

from . import hdf


class HDFMatvec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, ell, v, kernel, tol, precision, p_max):
        f = hdf.build(x.detach(), kernel, float(ell), tol, precision=precision, p_max=p_max)
        y = f.matvec(v.detach())
        ctx.factor = f
        ctx.save_for_backward(x, v)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, v = ctx.saved_tensors
        f = ctx.factor
        gy = gy.contiguous().to(f.dtype)
        gx = gell = gv = None
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            G, dl, _ = f.adjoint(x.detach(), v.detach(), gy)
            gx = G.to(x.dtype)
            gell = torch.tensor(dl, dtype=torch.float64)
        if ctx.needs_input_grad[2]:
            gv = f.matvec(gy)
        return gx, gell, gv, None, None, None, None


def kernel_matvec(x, ell, v, kernel="gaussian", tol=1e-6, precision="fp64", p_max=None):
    """K~(x, ell) v with gradients for x (float64 CUDA, (n, d)), ell (0-d tensor) and v."""
    if not isinstance(ell, torch.Tensor):
        ell = torch.tensor(float(ell), dtype=torch.float64)
    return HDFMatvec.apply(x, ell, v, kernel, tol, precision, p_max)
