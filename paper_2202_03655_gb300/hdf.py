"""Thin ctypes binding of libhdf.so (argument marshalling only).

Every step of the factorization runs inside the library; this module only converts
torch tensors and numpy arrays to pointers, sizes and streams, and library status codes
to exceptions.  If the library has not been built the first call raises: there is no
fallback path.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhdf.so")

KERNELS = {"gaussian": 0, "cauchy": 1, "matern32": 2, "matern52": 3}
PRECISIONS = {"fp64": 0, "fp32": 1}
STATUS = {0: "HDF_OK", 1: "HDF_EINVAL", 2: "HDF_ENOMEM", 3: "HDF_ECUDA", 4: "HDF_ETOL_UNREACHABLE",
          5: "HDF_ENOTFINITE", 6: "HDF_ESINGULAR", 7: "HDF_ETIMEOUT", 8: "HDF_ETOOBIG"}
HDF_OK, HDF_ETOL_UNREACHABLE = 0, 4
MAX_D, MAX_L, NPHASE = 8, 64, 8

# Every exported entry point with its ctypes signature (include/hdf.h).
_c_int, _c_i64, _c_dbl, _vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
_pdbl = ctypes.POINTER(ctypes.c_double)


class HdfOptions(ctypes.Structure):
    _fields_ = [("p_max", _c_int), ("eta", _c_dbl), ("flags", _c_int)]


class HdfInfo(ctypes.Structure):
    _fields_ = [("n", _c_i64), ("d", _c_int), ("precision", _c_int), ("p", _c_int), ("L", _c_int),
                ("reached", _c_int), ("rank", _c_i64), ("ldu", _c_i64), ("nharm", _c_i64),
                ("center", _c_dbl * MAX_D), ("radius", _c_dbl), ("mu2", _c_dbl), ("cheb_tail", _c_dbl),
                ("tail_budget", _c_dbl), ("drop_budget", _c_dbl), ("dropped_cost", _c_dbl),
                ("err_bound", _c_dbl), ("s_k", _c_int * (MAX_L + 1)), ("t_ms", _c_dbl * NPHASE),
                ("n_y", _c_i64), ("matrix_free", _c_int), ("mf_row", _c_i64), ("lu_ms", _c_dbl)]


SIGNATURES = {
    "hdf_build": (_c_int, [_vp, _c_i64, _c_int, _c_int, _c_dbl, _c_dbl, _c_int, ctypes.POINTER(HdfOptions),
                           _vp, ctypes.POINTER(_vp)]),
    "hdf_build_cross": (_c_int, [_vp, _c_i64, _vp, _c_i64, _c_int, _c_int, _c_dbl, _c_dbl, _c_int,
                                 ctypes.POINTER(HdfOptions), _vp, ctypes.POINTER(_vp)]),
    "hdf_matvec": (_c_int, [_vp, _vp, _c_i64, _c_int, _vp, _c_i64, _vp]),
    "hdf_matvec_transpose": (_c_int, [_vp, _vp, _c_i64, _c_int, _vp, _c_i64, _vp]),
    "hdf_matvec_noalloc": (_c_int, [_vp, _vp, _c_i64, _c_int, _vp, _c_i64, _vp]),
    "hdf_solve": (_c_int, [_vp, _c_dbl, _vp, _c_i64, _c_int, _vp, _c_i64, _c_int, _vp]),
    "hdf_matvec_adjoint": (_c_int, [_vp, _vp, _vp, _c_i64, _vp, _c_i64, _c_int, _vp, _pdbl, _pdbl, _vp]),
    "hdf_factor_info": (_c_int, [_vp, ctypes.POINTER(HdfInfo)]),
    "hdf_factor_device": (_c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "hdf_factor_export": (_c_int, [_vp, _vp, _pdbl]),
    "hdf_factor_export_y": (_c_int, [_vp, _vp]),
    "hdf_free": (None, [_vp]),
    "hdf_device_errors": (_c_int, [_vp, ctypes.POINTER(_c_int)]),
    "hdf_matvec_timings": (_c_int, [_vp, _pdbl]),
    "hdf_cheb_nodes": (_c_int, [_c_int]),
    "hdf_cheb_coeffs": (_c_int, [_c_int, _c_dbl, _c_dbl, _c_int, _pdbl]),
    "hdf_choose_degree": (_c_int, [_pdbl, _c_int, _c_dbl, _c_int, ctypes.POINTER(_c_int), _pdbl,
                                   ctypes.POINTER(_c_int)]),
    "hdf_radial_cores": (_c_int, [_pdbl, _c_int, _c_int, _pdbl, ctypes.POINTER(_c_i64)]),
    "hdf_build_batched": (_c_int, [_c_int, ctypes.POINTER(_c_i64), _vp, _c_int, _c_int, _pdbl, _c_dbl, _c_int,
                                   ctypes.POINTER(HdfOptions), _vp, ctypes.POINTER(_vp)]),
    "hdf_batch_matvec": (_c_int, [_vp, _vp, _c_i64, _c_int, _vp, _c_i64, _vp]),
    "hdf_batch_info": (_c_int, [_vp, _c_int, ctypes.POINTER(HdfInfo)]),
    "hdf_batch_timings": (_c_int, [_vp, _pdbl]),
    "hdf_batch_device_errors": (_c_int, [_vp, ctypes.POINTER(_c_int)]),
    "hdf_batch_export": (_c_int, [_vp, _c_int, _vp, _pdbl]),
    "hdf_batch_free": (None, [_vp]),
    "hdf_kmeans": (_c_int, [_vp, _c_i64, _c_int, _c_int, ctypes.POINTER(_c_i64), _c_int, _vp, _vp,
                            ctypes.POINTER(_c_int), _vp]),
    "hdf_kernel_matvec": (_c_int, [_vp, _c_i64, _vp, _c_i64, _c_int, _c_int, _c_dbl, _vp, _vp, _vp]),
    "hdf_krr_build": (_c_int, [_vp, _c_i64, _c_int, _vp, _c_int, _c_dbl, _c_dbl, _c_dbl, _c_int,
                               ctypes.POINTER(HdfOptions), _vp, ctypes.POINTER(_vp)]),
    "hdf_krr_apply": (_c_int, [_vp, _vp, _vp, _vp]),
    "hdf_krr_precond": (_c_int, [_vp, _vp, _vp, _vp]),
    "hdf_krr_solve": (_c_int, [_vp, _vp, _c_dbl, _c_int, _vp, ctypes.POINTER(_c_int), _pdbl, _vp]),
    "hdf_krr_info": (_c_int, [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_i64), _pdbl]),
    "hdf_krr_free": (None, [_vp]),
    "hdf_set_wait_limit": (_c_int, [ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
    "hdf_debug_fail_alloc": (None, [ctypes.c_longlong]),
    "hdf_check_tf32_rounding": (_c_int, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "hdf_status_string": (ctypes.c_char_p, [_c_int]),
    "hdf_last_error": (ctypes.c_char_p, []),
    "hdf_launch_count": (ctypes.c_longlong, []),
}

_lib = None


class HdfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load libhdf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                               "g.build()'` (there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, allow=(HDF_OK,)):
    if status not in allow:
        raise HdfError(status, lib().hdf_last_error().decode())
    return status


def _dptr(a):
    return a.ctypes.data_as(_pdbl)


# ------------------------------------------------------------------ host planner calls

def cheb_nodes(p_max):
    return lib().hdf_cheb_nodes(int(p_max))


def cheb_coeffs(kernel, lengthscale, two_r, M):
    a = np.zeros(int(M))
    _check(lib().hdf_cheb_coeffs(KERNELS[kernel], float(lengthscale), float(two_r), int(M), _dptr(a)))
    return a


def choose_degree(a, budget, p_max):
    a = np.ascontiguousarray(a, dtype=np.float64)
    p, tail, ok = _c_int(), _c_dbl(), _c_int()
    _check(lib().hdf_choose_degree(_dptr(a), a.size, float(budget), int(p_max), ctypes.byref(p),
                                   ctypes.byref(tail), ctypes.byref(ok)))
    return p.value, tail.value, bool(ok.value)


def radial_cores(a, p, d):
    a = np.ascontiguousarray(a, dtype=np.float64)
    cnt = _c_i64()
    _check(lib().hdf_radial_cores(_dptr(a), int(p), int(d), None, ctypes.byref(cnt)))
    buf = np.zeros(cnt.value)
    _check(lib().hdf_radial_cores(_dptr(a), int(p), int(d), _dptr(buf), ctypes.byref(cnt)))
    L = p // 2
    out, off = [], 0
    for k in range(L + 1):
        nb = L + 1 if k % 2 == 0 else L
        out.append(buf[off:off + nb * nb].reshape(nb, nb))
        off += nb * nb
    return out


def set_wait_limit(cycles):
    """Limit (clock cycles) of the tensor-core kernels' waits on the current device; <= 0 restores
    the default.  Returns the previous limit."""
    prev = ctypes.c_longlong()
    _check(lib().hdf_set_wait_limit(int(cycles), ctypes.byref(prev)))
    return prev.value


def check_tf32_rounding():
    """Mismatches of the library's TF32 operand rounding against the device's conversion
    instruction over all finite FP32 values: (below 2^127 in magnitude, top binade)."""
    out = (ctypes.c_ulonglong * 2)()
    _check(lib().hdf_check_tf32_rounding(out))
    return int(out[0]), int(out[1])


def debug_fail_alloc(after):
    """Make the device allocation `after` allocations from now report out-of-memory (once);
    a negative value cancels."""
    lib().hdf_debug_fail_alloc(int(after))


def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(lib().hdf_launch_count())


# --------------------------------------------------------------------- device calls

def _stream_handle(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return _vp(s.cuda_stream)


class Factor:
    """K ~= U diag(S) U^T held by the library (U and S in device memory), or, from
    build_cross, K(X, Y) ~= U diag(S) V^T with n = |X| rows of U and n_y = |Y| rows of V."""

    def __init__(self, handle, status):
        self._h = handle
        self.status = status
        self.info = HdfInfo()
        _check(lib().hdf_factor_info(self._h, ctypes.byref(self.info)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.hdf_free(h)
            self._h = None

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.info.precision == 0 else torch.float32

    @property
    def n(self):
        return self.info.n

    @property
    def n_y(self):
        """Rows of the second factor (points of Y) of a cross factor; 0 if symmetric."""
        return self.info.n_y

    @property
    def cross(self):
        return self.info.n_y > 0

    @property
    def rank(self):
        return self.info.rank

    @property
    def s_k(self):
        return [self.info.s_k[k] for k in range(self.info.L + 1)]

    def _block(self, V, rows=None):
        import torch
        rows = self.n if rows is None else rows
        if not (V.is_cuda and V.dtype == self.dtype):
            raise ValueError(f"expected a CUDA tensor of dtype {self.dtype}")
        if V.dim() == 1:
            V = V.reshape(-1, 1)
        if V.shape[0] != rows:
            raise ValueError(f"first dimension must be {rows}")
        # column-major n x c: a (c, n) row-major tensor transposed
        Vc = V.t().contiguous()
        return Vc

    def matvec(self, V, stream=None):
        """Y = K~ V for V of shape (n,) or (n, c) on the device (Sec. 3.6).  For a cross
        factor V has n_y rows and Y has n rows."""
        import torch
        vec = V.dim() == 1
        nin = self.n_y if self.cross else self.n
        Vc = self._block(V, nin)
        c = Vc.shape[0]
        Yc = torch.empty((c, self.n), dtype=Vc.dtype, device=Vc.device)
        _check(lib().hdf_matvec(self._h, _vp(Vc.data_ptr()), nin, c, _vp(Yc.data_ptr()), self.n,
                                _stream_handle(stream)))
        Y = Yc.t()
        return Y.reshape(-1) if vec else Y

    def matvec_t(self, W, stream=None):
        """Y = K~^T W (hdf_matvec_transpose).  For a cross factor W has n rows and Y has n_y."""
        import torch
        vec = W.dim() == 1
        nout = self.n_y if self.cross else self.n
        Wc = self._block(W, self.n)
        c = Wc.shape[0]
        Yc = torch.empty((c, nout), dtype=Wc.dtype, device=Wc.device)
        _check(lib().hdf_matvec_transpose(self._h, _vp(Wc.data_ptr()), self.n, c, _vp(Yc.data_ptr()), nout,
                                          _stream_handle(stream)))
        Y = Yc.t()
        return Y.reshape(-1) if vec else Y

    def matvec_ptr(self, V_ptr, ldv, ncols, Y_ptr, ldy, stream=None):
        """Raw-pointer form of matvec (column-major blocks already on the device)."""
        _check(lib().hdf_matvec(self._h, _vp(V_ptr), int(ldv), int(ncols), _vp(Y_ptr), int(ldy),
                                _stream_handle(stream)))

    def matvec_noalloc_ptr(self, V_ptr, ldv, ncols, Y_ptr, ldy, stream=None):
        """K~ V through hdf_matvec_noalloc (work space in the library's fixed array)."""
        _check(lib().hdf_matvec_noalloc(self._h, _vp(V_ptr), int(ldv), int(ncols), _vp(Y_ptr), int(ldy),
                                        _stream_handle(stream)))

    def adjoint(self, x, V, W, stream=None):
        """Gradient of f = sum_j W[:, j]^T K~ V[:, j] under frozen structure.

        x: the build points (CUDA float64, (n, d)); V, W: (n,) or (n, c) of the bulk dtype.
        Returns (grad_x (n, d) bulk dtype, d f / d l, f)."""
        import torch
        Vc, Wc = self._block(V), self._block(W)
        c = Vc.shape[0]
        if Wc.shape[0] != c:
            raise ValueError("V and W must have the same number of columns")
        x = x.contiguous()
        G = torch.empty((self.n, self.info.d), dtype=self.dtype, device=x.device)
        gl, val = _c_dbl(), _c_dbl()
        _check(lib().hdf_matvec_adjoint(self._h, _vp(x.data_ptr()), _vp(Vc.data_ptr()), self.n,
                                        _vp(Wc.data_ptr()), self.n, c, _vp(G.data_ptr()),
                                        ctypes.byref(gl), ctypes.byref(val), _stream_handle(stream)))
        return G, gl.value, val.value

    def solve(self, lam, B, refine_steps=1, stream=None):
        """X = (lam I + K~)^{-1} B (Eq. opt via Woodbury), with iterative refinement."""
        import torch
        vec = B.dim() == 1
        Bc = self._block(B)
        c = Bc.shape[0]
        Xc = torch.empty_like(Bc)
        _check(lib().hdf_solve(self._h, float(lam), _vp(Bc.data_ptr()), self.n, c, _vp(Xc.data_ptr()), self.n,
                               int(refine_steps), _stream_handle(stream)))
        _check(lib().hdf_factor_info(self._h, ctypes.byref(self.info)))     # t_ms[6]: Gram time
        X = Xc.t()
        return X.reshape(-1) if vec else X

    def matvec_timings(self):
        """(U^T V ms, reduce ms, U W ms) of the most recent matvec (device events)."""
        out = np.zeros(3)
        _check(lib().hdf_matvec_timings(self._h, _dptr(out)))
        return out

    def device_errors(self):
        """1 if a kernel on this factor gave up a bounded wait since the last check (clears it)."""
        fl = _c_int()
        _check(lib().hdf_device_errors(self._h, ctypes.byref(fl)))
        return fl.value

    def free(self):
        """Release the factor's device memory now."""
        h = getattr(self, "_h", None)
        if h is not None:
            lib().hdf_free(h)
            self._h = None

    def device_U(self):
        """(U pointer, ldu, S pointer) in device memory."""
        u, s = _vp(), _vp()
        _check(lib().hdf_factor_device(self._h, ctypes.byref(u), ctypes.byref(s)))
        return u.value, self.info.ldu, s.value

    def export(self):
        """(U as numpy (n, rank), S as numpy (rank,) float64)."""
        dt = np.float64 if self.info.precision == 0 else np.float32
        U = np.zeros((self.n, self.rank), dtype=dt)
        S = np.zeros(self.rank)
        _check(lib().hdf_factor_export(self._h, _vp(U.ctypes.data), _dptr(S)))
        return U, S

    def export_y(self):
        """The second factor V of a cross factor as numpy (n_y, rank)."""
        dt = np.float64 if self.info.precision == 0 else np.float32
        V = np.zeros((self.n_y, self.rank), dtype=dt)
        _check(lib().hdf_factor_export_y(self._h, _vp(V.ctypes.data)))
        return V


FLAG_CUDA_CORES = 1
FLAG_MATRIX_FREE = 2


def build(x, kernel, lengthscale, tol, precision="fp64", p_max=None, eta=None, stream=None, flags=0):
    """Factor K(x, x) for points x (torch CUDA float64, shape (n, d)).

    Returns a Factor; a factor capped at p_max (HDF_ETOL_UNREACHABLE) is returned with
    ``status`` set and ``info.reached == 0``.
    """
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.dim() == 2):
        raise ValueError("x must be a CUDA float64 tensor of shape (n, d)")
    x = x.contiguous()
    opt = HdfOptions(int(p_max or 0), float(eta or 0.0), int(flags))
    h = _vp()
    st = lib().hdf_build(_vp(x.data_ptr()), x.shape[0], x.shape[1], KERNELS[kernel], float(lengthscale),
                         float(tol), PRECISIONS[precision], ctypes.byref(opt), _stream_handle(stream),
                         ctypes.byref(h))
    _check(st, allow=(HDF_OK, HDF_ETOL_UNREACHABLE))
    return Factor(h, st)


def build_cross(x, y, kernel, lengthscale, tol, precision="fp64", p_max=None, eta=None, stream=None, flags=0):
    """Factor K(x, y) ~= U S V^T for two point sets (torch CUDA float64, shapes (m, d), (n, d)),
    Algorithm 1 in its general form (hdf_build_cross)."""
    import torch
    for t in (x, y):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.dim() == 2):
            raise ValueError("x and y must be CUDA float64 tensors of shape (m, d), (n, d)")
    if x.shape[1] != y.shape[1]:
        raise ValueError("x and y must have the same dimension")
    x, y = x.contiguous(), y.contiguous()
    opt = HdfOptions(int(p_max or 0), float(eta or 0.0), int(flags))
    h = _vp()
    st = lib().hdf_build_cross(_vp(x.data_ptr()), x.shape[0], _vp(y.data_ptr()), y.shape[0], x.shape[1],
                               KERNELS[kernel], float(lengthscale), float(tol), PRECISIONS[precision],
                               ctypes.byref(opt), _stream_handle(stream), ctypes.byref(h))
    _check(st, allow=(HDF_OK, HDF_ETOL_UNREACHABLE))
    return Factor(h, st)


class Batch:
    """Many independent factors built and applied together (hdf_build_batched)."""

    def __init__(self, handle, status, offsets, precision):
        self._h = handle
        self.status = status
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.nsets = len(self.offsets) - 1
        self.precision = precision

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.hdf_batch_free(h)
            self._h = None

    def free(self):
        h = getattr(self, "_h", None)
        if h is not None:
            lib().hdf_batch_free(h)
            self._h = None

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    def info(self, s):
        I = HdfInfo()
        _check(lib().hdf_batch_info(self._h, int(s), ctypes.byref(I)))
        return I

    def timings(self):
        out = np.zeros(NPHASE)
        _check(lib().hdf_batch_timings(self._h, _dptr(out)))
        return out

    def device_errors(self):
        """1 if a kernel of the batch's matvec gave up a bounded wait since the last call, else 0."""
        fl = _c_int(0)
        _check(lib().hdf_batch_device_errors(self._h, ctypes.byref(fl)))
        return fl.value

    def matvec_ptr(self, V_ptr, ldv, ncols, Y_ptr, ldy, stream=None):
        _check(lib().hdf_batch_matvec(self._h, _vp(V_ptr), int(ldv), int(ncols), _vp(Y_ptr), int(ldy),
                                      _stream_handle(stream)))

    def matvec(self, V, stream=None):
        """V: (sum n, c) tensor of the bulk dtype; returns K~_s V_s stacked the same way."""
        import torch
        vec = V.dim() == 1
        V2 = V.reshape(V.shape[0], -1)
        Vc = V2.t().contiguous()
        Yc = torch.empty_like(Vc)
        ntot = int(self.offsets[-1])
        self.matvec_ptr(Vc.data_ptr(), ntot, Vc.shape[0], Yc.data_ptr(), ntot, stream)
        Y = Yc.t()
        return Y.reshape(-1) if vec else Y

    def export(self, s):
        I = self.info(s)
        dt = np.float64 if I.precision == 0 else np.float32
        U = np.zeros((I.n, I.rank), dtype=dt)
        S = np.zeros(I.rank)
        _check(lib().hdf_batch_export(self._h, int(s), _vp(U.ctypes.data), _dptr(S)))
        return U, S


def build_batched(x, offsets, kernel, lengthscales, tol, precision="fp32", p_max=None, eta=None, stream=None):
    """Factor the sets x[offsets[s]:offsets[s+1]] (x: CUDA float64 (sum n, d))."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.dim() == 2):
        raise ValueError("x must be a CUDA float64 tensor of shape (N, d)")
    x = x.contiguous()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    ells = np.ascontiguousarray(lengthscales, dtype=np.float64)
    opt = HdfOptions(int(p_max or 0), float(eta or 0.0), 0)
    h = _vp()
    st = lib().hdf_build_batched(len(off) - 1, off.ctypes.data_as(ctypes.POINTER(_c_i64)), _vp(x.data_ptr()),
                                 x.shape[1], KERNELS[kernel], _dptr(ells), float(tol), PRECISIONS[precision],
                                 ctypes.byref(opt), _stream_handle(stream), ctypes.byref(h))
    _check(st, allow=(HDF_OK, HDF_ETOL_UNREACHABLE))
    return Batch(h, st, off, precision)


# ---------------------------------------------------------- kernel ridge regression

def _f64_vec(v, n):
    import torch
    if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float64 and v.numel() == n):
        raise ValueError(f"expected a CUDA float64 tensor of {n} entries")
    return v.contiguous().reshape(-1)


def kmeans(x, init_idx, max_iter=100, stream=None):
    """Lloyd's k-means (hdf_kmeans) from the centres x[init_idx]: (labels int32, centres, passes)."""
    import torch
    x = x.contiguous()
    init = np.ascontiguousarray(np.asarray(init_idx, dtype=np.int64))
    k = len(init)
    labels = torch.empty(x.shape[0], dtype=torch.int32, device=x.device)
    C = torch.empty((k, x.shape[1]), dtype=torch.float64, device=x.device)
    it = _c_int()
    _check(lib().hdf_kmeans(_vp(x.data_ptr()), x.shape[0], x.shape[1], k, init.ctypes.data_as(ctypes.POINTER(_c_i64)),
                            int(max_iter), _vp(labels.data_ptr()), _vp(C.data_ptr()), ctypes.byref(it),
                            _stream_handle(stream)))
    return labels, C, it.value


def kernel_matvec(xq, x, kernel, lengthscale, w, stream=None):
    """K(xq, x) w by direct evaluation (hdf_kernel_matvec)."""
    import torch
    xq, x = xq.contiguous(), x.contiguous()
    w = _f64_vec(w, x.shape[0])
    out = torch.empty(xq.shape[0], dtype=torch.float64, device=x.device)
    _check(lib().hdf_kernel_matvec(_vp(xq.data_ptr()), xq.shape[0], _vp(x.data_ptr()), x.shape[0], x.shape[1],
                                   KERNELS[kernel], float(lengthscale), _vp(w.data_ptr()), _vp(out.data_ptr()),
                                   _stream_handle(stream)))
    return out


class KRR:
    """(lambda I + K^) of Sec. 4.2 held by the library (hdf_krr_*)."""

    def __init__(self, x, labels, kernel, lengthscale, lam, tol, precision="fp64", p_max=None, eta=None,
                 stream=None):
        import torch
        x = x.contiguous()
        labels = labels.to(torch.int32).contiguous()
        self.n = x.shape[0]
        opt = HdfOptions(int(p_max or 0), float(eta or 0.0), 0)
        h = _vp()
        st = lib().hdf_krr_build(_vp(x.data_ptr()), x.shape[0], x.shape[1], _vp(labels.data_ptr()), KERNELS[kernel],
                                 float(lengthscale), float(lam), float(tol), PRECISIONS[precision], ctypes.byref(opt),
                                 _stream_handle(stream), ctypes.byref(h))
        _check(st, allow=(HDF_OK, HDF_ETOL_UNREACHABLE))
        self._h = h
        self.status = st

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.hdf_krr_free(h)
            self._h = None

    def free(self):
        h = getattr(self, "_h", None)
        if h is not None:
            lib().hdf_krr_free(h)
            self._h = None

    def apply(self, v, stream=None):
        import torch
        v = _f64_vec(v, self.n)
        out = torch.empty_like(v)
        _check(lib().hdf_krr_apply(self._h, _vp(v.data_ptr()), _vp(out.data_ptr()), _stream_handle(stream)))
        return out

    def precond(self, r, stream=None):
        import torch
        r = _f64_vec(r, self.n)
        out = torch.empty_like(r)
        _check(lib().hdf_krr_precond(self._h, _vp(r.data_ptr()), _vp(out.data_ptr()), _stream_handle(stream)))
        return out

    def solve(self, y, rtol=1e-8, max_iter=1000, stream=None):
        """(w, iterations, relative residual) of PCG for (lambda I + K^) w = y."""
        import torch
        y = _f64_vec(y, self.n)
        w = torch.empty_like(y)
        it, res = _c_int(), _c_dbl()
        st = lib().hdf_krr_solve(self._h, _vp(y.data_ptr()), float(rtol), int(max_iter), _vp(w.data_ptr()),
                                 ctypes.byref(it), ctypes.byref(res), _stream_handle(stream))
        _check(st, allow=(HDF_OK, HDF_ETOL_UNREACHABLE))
        return w, it.value, res.value

    def info(self):
        """(clusters, total rank of the diagonal blocks, (factorization ms, preconditioner ms))."""
        nc, rk = _c_int(), _c_i64()
        t = np.zeros(2)
        _check(lib().hdf_krr_info(self._h, ctypes.byref(nc), ctypes.byref(rk), _dptr(t)))
        return nc.value, rk.value, (float(t[0]), float(t[1]))

