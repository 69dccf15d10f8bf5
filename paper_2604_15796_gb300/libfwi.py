"""Thin ctypes binding of libfwi (include/libfwi.h).

The functions below carry the C names and only marshal arguments (integers,
doubles and device pointers); every computational step runs in the CUDA
kernels of libfwi.so.  There is no fallback: importing the binding without
the compiled library raises.

``Context`` is a convenience wrapper that owns a ``fwi_ctx`` and takes
torch tensors (device memory and the current CUDA stream come from torch).
"""
import ctypes
import json
import os
import time
from ctypes import POINTER, Structure, byref, c_double, c_float, c_int, c_size_t, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libfwi.so")

FWI_OK = 0
FWI_ERR_INVALID_ARG = 1
FWI_ERR_NOMEM = 2
FWI_ERR_CUDA = 3
FWI_ERR_NOT_CONVERGED = 4
FWI_ERR_BREAKDOWN = 5
FWI_ERR_NONFINITE = 6
FWI_ERR_CANCELLED = 7
FWI_ERR_UNSUPPORTED = 8
FWI_ERR_REDUCE = 9
FWI_MIXED = 0
FWI_FP64 = 1

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NOMEM", 3: "CUDA", 4: "NOT_CONVERGED",
                5: "BREAKDOWN", 6: "NONFINITE", 7: "CANCELLED", 8: "UNSUPPORTED", 9: "REDUCE"}


class fwi_problem_desc(Structure):
    _fields_ = [("dim", c_int), ("n", c_int * 3), ("h", c_double), ("c0", c_double),
                ("n_elem", c_int), ("elem_pos", POINTER(c_double)), ("n_freq", c_int),
                ("freq_hz", POINTER(c_double)), ("krylov_tol", c_double),
                ("krylov_max_it", c_int), ("precision", c_int), ("max_batch", c_int),
                ("n_tx", c_int), ("tx_angle", POINTER(c_double)), ("elem_length", c_double),
                ("inv_factor", c_int), ("alpha0", c_double), ("hybrid_born", c_int)]


class fwi_solve_info(Structure):
    _fields_ = [("n_rhs", c_int), ("iters", POINTER(c_int)), ("rel_resid", POINTER(c_double)),
                ("status", POINTER(c_int)), ("max_iters", c_int), ("max_rel_resid", c_double),
                ("n_not_converged", c_int), ("device_ms", c_float)]


class fwi_kernel_stat(Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("ms", c_double), ("launches", ctypes.c_longlong),
                ("bytes", c_double), ("flops", c_double)]


FWI_MAX_KERNEL_STATS = 24


class fwi_stats(Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("n_kernel_stats", c_int),
                ("kernels", fwi_kernel_stat * FWI_MAX_KERNEL_STATS)]


class fwi_tuning(Structure):
    _fields_ = [("row_fwd_variant", c_int), ("row_inv_variant", c_int), ("col_variant", c_int),
                ("col_y_variant", c_int), ("tuned", c_int), ("ms", (c_float * 4) * 4),
                ("jac_tensor_cores", c_int), ("overlap_halves", c_int),
                ("debug_stall_once", c_int), ("col_tma", c_int),
                ("col_spectrum_stage", c_int), ("jac_tma", c_int), ("row_l2_prefetch", c_int),
                ("row_stage", c_int), ("col_pairs", c_int)]


class fwi_admm_params(Structure):
    _fields_ = [("lambda_", c_double), ("rho", c_double), ("gamma", c_double),
                ("dual_step", c_double), ("n_cg", c_int), ("m_ref", c_void_p)]


class fwi_request(Structure):
    _fields_ = [("problem", fwi_problem_desc), ("sos0", POINTER(c_double)),
                ("d_obs", c_void_p), ("admm", fwi_admm_params), ("n_iter", c_int),
                ("refresh_every", c_int)]


class fwi_request_result(Structure):
    _fields_ = [("status", c_int), ("queue_ms", c_double), ("run_ms", c_double),
                ("latency_ms", c_double), ("misfit_first", c_double), ("misfit_last", c_double),
                ("rhs_solves", ctypes.c_longlong), ("bytes", c_size_t),
                ("krylov_iters_max", c_int), ("krylov_iters_mean", c_double),
                ("not_converged", ctypes.c_longlong)]


EXPORTS = {
    "fwi_workspace_bytes": (c_size_t, [POINTER(fwi_problem_desc)]),
    "fwi_create": (c_int, [POINTER(fwi_problem_desc), c_void_p, POINTER(c_void_p)]),
    "fwi_destroy": (c_int, [c_void_p]),
    "fwi_last_error": (ctypes.c_char_p, [c_void_p]),
    "fwi_cancel": (c_int, [c_void_p]),
    "fwi_contrast_from_sos": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "fwi_sos_attenuation_from_contrast": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "fwi_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p,
                            POINTER(fwi_solve_info)]),
    "fwi_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(fwi_solve_info)]),
    "fwi_gradient": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_double),
                             c_void_p, POINTER(fwi_solve_info), POINTER(fwi_solve_info)]),
    "fwi_admm_tv_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 POINTER(fwi_admm_params), c_void_p]),
    "fwi_admm_init": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "fwi_freeze_receiver_fields": (c_int, [c_void_p, c_int]),
    "fwi_set_reducer": (c_int, [c_void_p, c_void_p, c_void_p]),
    "fwi_apply_K": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "fwi_apply_A": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "fwi_apply_AH": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "fwi_jac_forward": (c_int, [c_void_p, c_void_p, c_void_p]),
    "fwi_jac_adjoint": (c_int, [c_void_p, c_void_p, c_void_p]),
    "fwi_contract_pixels_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int,
                                            ctypes.c_longlong, POINTER(c_double), c_void_p,
                                            c_void_p]),
    "fwi_server_create": (c_int, [c_size_t, c_int, POINTER(c_void_p)]),
    "fwi_server_submit": (c_int, [c_void_p, POINTER(fwi_request), POINTER(ctypes.c_longlong)]),
    "fwi_server_wait": (c_int, [c_void_p, ctypes.c_longlong, POINTER(c_double),
                                POINTER(fwi_request_result)]),
    "fwi_server_cancel": (c_int, [c_void_p, ctypes.c_longlong]),
    "fwi_server_stats": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_size_t)]),
    "fwi_server_destroy": (c_int, [c_void_p]),
    "fwi_get_tuning": (c_int, [c_void_p, POINTER(fwi_tuning)]),
    "fwi_set_tuning": (c_int, [c_void_p, POINTER(fwi_tuning)]),
    "fwi_set_profiling": (c_int, [c_void_p, c_int]),
    "fwi_get_stats": (c_int, [c_void_p, POINTER(fwi_stats)]),
    "fwi_reset_stats": (c_int, [c_void_p]),
    "fwi_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path=LIB_PATH):
    """Load libfwi.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError("libfwi.so not built: run paper_2604_15796_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _bind(name):
    def call(*args):
        return getattr(load(), name)(*args)
    call.__name__ = name
    return call


fwi_workspace_bytes = _bind("fwi_workspace_bytes")
fwi_create = _bind("fwi_create")
fwi_destroy = _bind("fwi_destroy")
fwi_last_error = _bind("fwi_last_error")
fwi_cancel = _bind("fwi_cancel")
fwi_contrast_from_sos = _bind("fwi_contrast_from_sos")
fwi_sos_attenuation_from_contrast = _bind("fwi_sos_attenuation_from_contrast")
fwi_forward = _bind("fwi_forward")
fwi_adjoint = _bind("fwi_adjoint")
fwi_gradient = _bind("fwi_gradient")
fwi_admm_tv_step = _bind("fwi_admm_tv_step")
fwi_admm_init = _bind("fwi_admm_init")
fwi_freeze_receiver_fields = _bind("fwi_freeze_receiver_fields")
fwi_set_reducer = _bind("fwi_set_reducer")

# int (*fwi_reduce_fn)(void* buf, size_t count, void* cuda_stream, void* user)
REDUCE_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_size_t, c_void_p, c_void_p)
fwi_apply_K = _bind("fwi_apply_K")
fwi_apply_A = _bind("fwi_apply_A")
fwi_apply_AH = _bind("fwi_apply_AH")
fwi_jac_forward = _bind("fwi_jac_forward")
fwi_jac_adjoint = _bind("fwi_jac_adjoint")
fwi_contract_pixels_noalloc = _bind("fwi_contract_pixels_noalloc")
fwi_server_create = _bind("fwi_server_create")
fwi_server_submit = _bind("fwi_server_submit")
fwi_server_wait = _bind("fwi_server_wait")
fwi_server_cancel = _bind("fwi_server_cancel")
fwi_server_stats = _bind("fwi_server_stats")
fwi_server_destroy = _bind("fwi_server_destroy")
fwi_get_tuning = _bind("fwi_get_tuning")
fwi_set_tuning = _bind("fwi_set_tuning")
fwi_set_profiling = _bind("fwi_set_profiling")
fwi_get_stats = _bind("fwi_get_stats")
fwi_reset_stats = _bind("fwi_reset_stats")
fwi_version = _bind("fwi_version")


def reduce_callback(fn):
    """C reducer (REDUCE_FN) that calls ``fn(ptr, count, stream)`` and
    returns 0, or 1 after printing the exception it raised."""
    def cb(buf, count, stream, user):
        try:
            fn(int(buf or 0), int(count), int(stream or 0))
            return 0
        except Exception:  # reported to the library as a failed reduction
            import traceback
            traceback.print_exc()
            return 1
    return REDUCE_FN(cb)


class FwiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libfwi {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def make_desc(shape, h, c0, elem, freqs, precision=FWI_MIXED, tol=1e-6, max_it=1000,
              max_batch=0, tx_angles=None, elem_length=0.0, inv_factor=1, alpha0=0.0,
              hybrid_born=False):
    """fwi_problem_desc from array-order ``shape`` ((Nz, Nx) or (Nz, Ny, Nx)).
    ``tx_angles``: steering angles [rad] of plane-wave transmits, or None for
    point transmits at every element.  ``elem_length``: 3-D line elements of
    that length along y [m] (0: point elements).  ``inv_factor``: inversion
    mesh of cells of inv_factor^d forward pixels (1: the forward mesh).
    ``alpha0``: attenuation of the background [Np/m/Hz] (0: lossless).
    Returns (desc, keepalive) -- keep the second item alive while desc is used."""
    dim = len(shape)
    elem = np.ascontiguousarray(elem, dtype=np.float64)
    freqs = np.ascontiguousarray(freqs, dtype=np.float64)
    d = fwi_problem_desc()
    d.dim = dim
    if dim == 2:
        d.n[0], d.n[1], d.n[2] = shape[1], 1, shape[0]
    else:
        d.n[0], d.n[1], d.n[2] = shape[2], shape[1], shape[0]
    d.h, d.c0 = h, c0
    d.n_elem = elem.shape[0]
    d.elem_pos = elem.ctypes.data_as(POINTER(c_double))
    d.n_freq = len(freqs)
    d.freq_hz = freqs.ctypes.data_as(POINTER(c_double))
    d.krylov_tol, d.krylov_max_it = tol, max_it
    d.precision, d.max_batch = precision, max_batch
    d.elem_length = float(elem_length)
    d.inv_factor = int(inv_factor)
    d.alpha0 = float(alpha0)
    d.hybrid_born = int(bool(hybrid_born))
    tx = None
    if tx_angles is not None and len(tx_angles) > 0:
        tx = np.ascontiguousarray(tx_angles, dtype=np.float64)
        d.n_tx = tx.shape[0]
        d.tx_angle = tx.ctypes.data_as(POINTER(c_double))
    return d, (elem, freqs, tx)


def _ptr(t):
    return None if t is None else c_void_p(t.data_ptr())


def _dev(t, dtype, numel, name, optional=False):
    """Pointer to a tensor argument after checking it against the layout the
    C ABI documents for `name`: a contiguous CUDA tensor of `dtype` with
    exactly `numel` elements (NULL for None when the argument is optional).
    A mismatch raises ValueError before anything reaches the library, which
    reads and writes the buffers by their documented sizes."""
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    if not (t.is_cuda and t.dtype == dtype and t.numel() == numel and t.is_contiguous()):
        raise ValueError(
            f"{name}: expected a contiguous CUDA {dtype} tensor of {numel} elements, got "
            f"{t.dtype} of shape {tuple(t.shape)} on {t.device}"
            + ("" if t.is_contiguous() else " (not contiguous)"))
    return c_void_p(t.data_ptr())


class SolveReport:
    """Host arrays of an fwi_solve_info."""

    def __init__(self, n_rhs):
        self.iters = np.zeros(n_rhs, dtype=np.int32)
        self.rel_resid = np.zeros(n_rhs, dtype=np.float64)
        self.status = np.zeros(n_rhs, dtype=np.int32)
        self.info = fwi_solve_info()
        self.info.n_rhs = n_rhs
        self.info.iters = self.iters.ctypes.data_as(POINTER(c_int))
        self.info.rel_resid = self.rel_resid.ctypes.data_as(POINTER(c_double))
        self.info.status = self.status.ctypes.data_as(POINTER(c_int))

    @property
    def device_ms(self):
        return float(self.info.device_ms)

    @property
    def max_iters(self):
        return int(self.info.max_iters)

    def record(self):
        """The report's summary for the call log."""
        return {"device_ms": self.device_ms, "max_iters": self.max_iters,
                "not_converged": int(self.info.n_not_converged),
                "max_rel_resid": float(self.info.max_rel_resid)}


_call_log = {"file": None, "owned": False}


def set_call_log(target):
    """Append one JSON line per solve, gradient and ADMM-TV call to
    ``target`` (a path, an open text file, or None to stop): the call, its
    status, wall time, the device time and Krylov iterations of each solve,
    the grid and the number of right-hand sides.  The environment variable
    FWI_CALL_LOG=<path> enables it at import."""
    if _call_log["owned"] and _call_log["file"] is not None:
        _call_log["file"].close()
    if target is None:
        _call_log.update(file=None, owned=False)
    elif isinstance(target, (str, os.PathLike)):
        _call_log.update(file=open(target, "a", buffering=1), owned=True)
    else:
        _call_log.update(file=target, owned=False)


def _log_call(call, ctx, status, wall_s, **reports):
    f = _call_log["file"]
    if f is None:
        return
    rec = {"call": call, "status": STATUS_NAMES.get(status, status), "wall_ms": 1e3 * wall_s,
           "grid": list(ctx.shape), "n_rhs": ctx.n_rhs}
    rec.update({k: r.record() for k, r in reports.items()})
    f.write(json.dumps(rec) + "\n")


if os.environ.get("FWI_CALL_LOG"):
    set_call_log(os.environ["FWI_CALL_LOG"])


class Context:
    """Owns one fwi_ctx.  Tensors are torch CUDA tensors (complex64 fields for
    FWI_MIXED, complex128 for FWI_FP64; m, grad, g, u always complex128).

    shape: grid in array order ((Nz, Nx) or (Nz, Ny, Nx)); h: pixel [m];
    c0: background SoS [m/s]; elem: element positions [N_E, d]; freqs [Hz];
    tol, max_it: BiCGSTAB stopping rule; max_batch: RHS per Krylov launch
    (0: all); stream: the torch stream the library enqueues on;
    tx_angles: plane-wave transmits [rad] instead of point transmits
    (data [n_freq][N_T][N_E]); elem_length: 3-D line elements [m];
    inv_factor: inversion mesh of inv_factor^d pixels per cell (m, grad,
    g, u, SoS on it: ``inv_shape``); alpha0: background attenuation
    [Np/m/Hz]; hybrid_born: keep a receiver-field snapshot for
    ``freeze_receiver_fields``."""

    def __init__(self, shape, h, c0, elem, freqs, precision=FWI_MIXED, tol=1e-6,
                 max_it=1000, max_batch=0, stream=None, tx_angles=None, elem_length=0.0,
                 inv_factor=1, alpha0=0.0, hybrid_born=False):
        import torch
        self.torch = torch
        self.shape = tuple(shape)
        # the model (m, gradient, TV variables, SoS) lives on the inversion mesh
        self.inv_factor = max(int(inv_factor), 1)
        self.inv_shape = tuple(s // self.inv_factor for s in self.shape)
        self.n_inv = int(np.prod(self.inv_shape))
        self.dim = len(shape)
        self.n = int(np.prod(shape))
        self.n_elem = int(np.asarray(elem).shape[0])
        self.n_freq = int(len(freqs))
        self.n_rhs = self.n_elem * self.n_freq
        # transmits N_T: plane waves (tx_angles) or one point source per element
        self.n_t = len(tx_angles) if tx_angles is not None and len(tx_angles) > 0 else self.n_elem
        self.precision = precision
        self.field_dtype = torch.complex128 if precision == FWI_FP64 else torch.complex64
        self.desc, self._keep = make_desc(shape, h, c0, elem, freqs, precision, tol, max_it,
                                          max_batch, tx_angles, elem_length, inv_factor,
                                          alpha0, hybrid_born)
        self.workspace_bytes = int(fwi_workspace_bytes(byref(self.desc)))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = c_void_p()
        st = fwi_create(byref(self.desc), c_void_p(stream.cuda_stream), byref(handle))
        if st != FWI_OK:
            raise FwiError(st, fwi_last_error(None).decode())
        self.handle = handle

    # -- helpers ---------------------------------------------------------
    def _check(self, st, ok=(FWI_OK,)):
        if st not in ok:
            raise FwiError(st, fwi_last_error(self.handle).decode())
        return st

    def _m(self, t, name="m", optional=False):
        return _dev(t, self.torch.complex128, self.n_inv, name, optional)

    def _fields(self, t, name, optional=False):
        return _dev(t, self.field_dtype, self.n_rhs * self.n, name, optional)

    def _data(self, t, name, optional=False):
        return _dev(t, self.field_dtype, self.n_freq * self.n_t * self.n_elem, name, optional)

    def empty_fields(self):
        return self.torch.empty((self.n_freq, self.n_elem) + self.shape,
                                dtype=self.field_dtype, device="cuda")

    def empty_data(self):
        """[n_freq][N_T][n_elem]: transmits x receivers per frequency."""
        return self.torch.empty((self.n_freq, self.n_t, self.n_elem),
                                dtype=self.field_dtype, device="cuda")

    def close(self):
        if getattr(self, "handle", None) is not None:
            fwi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls -----------------------------------------------------------
    def contrast_from_sos(self, sos, alpha=None):
        m = self.torch.empty(self.inv_shape, dtype=self.torch.complex128, device="cuda")
        f64 = self.torch.float64
        self._check(fwi_contrast_from_sos(self.handle, _dev(sos, f64, self.n_inv, "sos"),
                                          _dev(alpha, f64, self.n_inv, "alpha", True), _ptr(m)))
        return m

    def sos_attenuation_from_contrast(self, m):
        """(SoS [m/s], attenuation [Np/m/Hz]) of a contrast on the inversion
        mesh, the inverse of contrast_from_sos."""
        f64 = self.torch.float64
        sos = self.torch.empty(self.inv_shape, dtype=f64, device="cuda")
        alpha = self.torch.empty(self.inv_shape, dtype=f64, device="cuda")
        self._check(fwi_sos_attenuation_from_contrast(self.handle, self._m(m), _ptr(sos),
                                                      _ptr(alpha)))
        return sos, alpha

    def forward(self, m, fields=None, warm_start=False, data=None, allow_nonconverged=False):
        rep = SolveReport(self.n_rhs)
        ok = (FWI_OK, FWI_ERR_NOT_CONVERGED) if allow_nonconverged else (FWI_OK,)
        args = (self._m(m), self._fields(fields, "fields", True), int(warm_start),
                self._data(data, "data", True))
        t0 = time.perf_counter()
        st = fwi_forward(self.handle, *args, byref(rep.info))
        _log_call("forward", self, st, time.perf_counter() - t0, forward=rep)
        self._check(st, ok)
        rep.code = st
        return rep

    def adjoint(self, m, src, lam):
        rep = SolveReport(self.n_rhs)
        args = (self._m(m), self._fields(src, "src"), self._fields(lam, "lam"))
        t0 = time.perf_counter()
        st = fwi_adjoint(self.handle, *args, byref(rep.info))
        _log_call("adjoint", self, st, time.perf_counter() - t0, adjoint=rep)
        self._check(st)
        return rep

    def gradient(self, m, d_obs, grad, data=None):
        rf, ra = SolveReport(self.n_rhs), SolveReport(self.n_rhs)
        mis = c_double(0.0)
        args = (self._m(m), self._data(d_obs, "d_obs"), self._m(grad, "grad"))
        dp = self._data(data, "data", True)
        t0 = time.perf_counter()
        st = fwi_gradient(self.handle, *args, byref(mis), dp, byref(rf.info), byref(ra.info))
        _log_call("gradient", self, st, time.perf_counter() - t0, forward=rf, adjoint=ra)
        self._check(st)
        return float(mis.value), rf, ra

    def admm_init(self, m0):
        """(g, u) = (nabla m0, 0) on the device (Algorithm 1 initialisation)."""
        g = self.torch.empty((self.dim,) + self.inv_shape, dtype=self.torch.complex128,
                             device="cuda")
        u = self.torch.empty_like(g)
        self._check(fwi_admm_init(self.handle, self._m(m0, "m0"), _ptr(g), _ptr(u)))
        return g, u

    def admm_tv_step(self, m, g, u, grad, lam=1e-4, rho=1e-3, gamma=1e-5, n_cg=10,
                     dual_step=0.0, m_ref=None, sos=None):
        p = fwi_admm_params()
        p.lambda_, p.rho, p.gamma, p.dual_step, p.n_cg = lam, rho, gamma, dual_step, n_cg
        m_ref_p = self._m(m_ref, "m_ref", True)
        p.m_ref = None if m_ref_p is None else m_ref_p.value
        c128, dn = self.torch.complex128, self.dim * self.n_inv
        args = (self._m(m), _dev(g, c128, dn, "g"), _dev(u, c128, dn, "u"),
                self._m(grad, "grad"))
        sp = _dev(sos, self.torch.float64, self.n_inv, "sos", True)
        t0 = time.perf_counter()
        st = fwi_admm_tv_step(self.handle, *args, byref(p), sp)
        _log_call("admm_tv_step", self, st, time.perf_counter() - t0)
        self._check(st)

    def set_reducer(self, fn):
        """Frequency sharding (fwi_set_reducer): ``fn(ptr, count, stream)``
        replaces the ``count`` doubles at device address ``ptr`` by their
        sum over all ranks, ordered on the CUDA stream handle ``stream``
        (see ``sharding``); None removes it.  An exception in fn makes the
        library call fail with FWI_ERR_REDUCE."""
        self._reducer = None if fn is None else reduce_callback(fn)
        self._check(fwi_set_reducer(self.handle, self._reducer, None))

    def freeze_receiver_fields(self, freeze=True):
        """Hybrid Born schedule (Sec. IV-B): True snapshots the current
        forward fields as the Jacobian's receiver fields until the next call;
        False returns to the current fields."""
        self._check(fwi_freeze_receiver_fields(self.handle, int(bool(freeze))))

    def apply(self, kind, vin, freq, m=None):
        nb = vin.shape[0]
        vp = _dev(vin, self.field_dtype, nb * self.n, "in")
        out = self.torch.empty_like(vin)
        if kind == "K":
            st = fwi_apply_K(self.handle, freq, nb, vp, _ptr(out))
        elif kind == "A":
            st = fwi_apply_A(self.handle, self._m(m), freq, nb, vp, _ptr(out))
        else:
            st = fwi_apply_AH(self.handle, self._m(m), freq, nb, vp, _ptr(out))
        self._check(st)
        return out

    def tuning(self):
        t = fwi_tuning()
        self._check(fwi_get_tuning(self.handle, byref(t)))
        return {"row_fwd": t.row_fwd_variant, "row_inv": t.row_inv_variant,
                "col": t.col_variant, "col_y": t.col_y_variant, "tuned": t.tuned,
                "ms": [[t.ms[k][v] for v in range(4)] for k in range(4)],
                "jac_tensor_cores": t.jac_tensor_cores, "overlap_halves": t.overlap_halves,
                "col_tma": t.col_tma, "col_spectrum_stage": t.col_spectrum_stage,
                "jac_tma": t.jac_tma, "row_l2_prefetch": t.row_l2_prefetch,
                "row_stage": t.row_stage, "col_pairs": t.col_pairs}

    def set_tuning(self, row_fwd=None, row_inv=None, col=None, col_y=None,
                   jac_tensor_cores=None, overlap_halves=None):
        """Force tile variants (0 when not given) and, optionally, switch the
        tensor-core pixel contractions or the two-chain iteration on (1) or
        off (0); None keeps the current setting."""
        t = fwi_tuning()
        self._check(fwi_get_tuning(self.handle, byref(t)))
        t.row_fwd_variant, t.row_inv_variant, t.col_variant, t.col_y_variant = (
            row_fwd or 0, row_inv or 0, col or 0, col_y or 0)
        if jac_tensor_cores is not None:
            t.jac_tensor_cores = int(jac_tensor_cores)
        if overlap_halves is not None:
            t.overlap_halves = int(overlap_halves)
        self._check(fwi_set_tuning(self.handle, byref(t)))

    def set_overlap(self, on):
        """Iterate large batches as two chains (True) or one (False), keeping
        the tile variants."""
        t = fwi_tuning()
        self._check(fwi_get_tuning(self.handle, byref(t)))
        t.overlap_halves = int(bool(on))
        self._check(fwi_set_tuning(self.handle, byref(t)))

    def set_jac_tensor_cores(self, on):
        """Switch the FP32 pixel contractions between tensor cores (True) and
        CUDA cores (False), keeping the tile variants."""
        t = fwi_tuning()
        self._check(fwi_get_tuning(self.handle, byref(t)))
        t.jac_tensor_cores = int(bool(on))
        self._check(fwi_set_tuning(self.handle, byref(t)))

    def set_col_tma(self, on):
        """Stage the FP32 column passes' tiles in shared memory with TMA
        copies (True) or read them with plain loads (False); results agree
        to FP32 rounding."""
        t = fwi_tuning()
        self._check(fwi_get_tuning(self.handle, byref(t)))
        t.col_tma = int(bool(on))
        self._check(fwi_set_tuning(self.handle, byref(t)))

    def set_col_spectrum_stage(self, on):
        """With TMA staging, also stage the convolution's kernel-spectrum
        tiles (True) or read the spectrum from global memory (False)."""
        t = fwi_tuning()
        self._check(fwi_get_tuning(self.handle, byref(t)))
        t.col_spectrum_stage = int(bool(on))
        self._check(fwi_set_tuning(self.handle, byref(t)))

    def set_jac_tma(self, on):
        """Tensor-core contractions take their raw operand tiles by TMA
        (True) or by the producers' cp.async (False); same bits."""
        t = fwi_tuning()
        self._check(fwi_get_tuning(self.handle, byref(t)))
        t.jac_tma = int(bool(on))
        self._check(fwi_set_tuning(self.handle, byref(t)))

    def set_row_l2_prefetch(self, on):
        """Row passes prefetch their next work item's rows into L2 (True)
        or not (False); results are bitwise the same."""
        t = fwi_tuning()
        self._check(fwi_get_tuning(self.handle, byref(t)))
        t.row_l2_prefetch = int(bool(on))
        self._check(fwi_set_tuning(self.handle, byref(t)))

    def set_row_stage(self, on):
        """The FP32 forward row pass stages its rows in shared memory with
        bulk copies (True) or loads them from global memory (False); results
        agree to FP32 rounding."""
        t = fwi_tuning()
        self._check(fwi_get_tuning(self.handle, byref(t)))
        t.row_stage = int(bool(on))
        self._check(fwi_set_tuning(self.handle, byref(t)))

    def set_col_pairs(self, on):
        """The FP32 convolution pass computes two columns per thread with
        packed arithmetic (True) or one (False), where its transform length
        allows; results agree to FP32 rounding."""
        t = fwi_tuning()
        self._check(fwi_get_tuning(self.handle, byref(t)))
        t.col_pairs = int(bool(on))
        self._check(fwi_set_tuning(self.handle, byref(t)))

    def debug_stall_once(self):
        """Test of the failure path: the next tensor-core contraction
        withholds its first pipeline stage, so that its bounded waits give up
        (about 1 s) and the call raises FwiError (FWI_ERR_CUDA)."""
        t = fwi_tuning()
        self._check(fwi_get_tuning(self.handle, byref(t)))
        t.debug_stall_once = 1
        self._check(fwi_set_tuning(self.handle, byref(t)))

    def cancel(self):
        """Ask a running (or the next) solve on this context to stop at its
        next host check; that call raises FwiError (FWI_ERR_CANCELLED).
        Thread-safe."""
        self._check(fwi_cancel(self.handle))

    def set_profiling(self, on):
        self._check(fwi_set_profiling(self.handle, int(bool(on))))

    def stats(self):
        """(kernel launches so far, {class: dict(ms, launches, bytes, flops)})."""
        st = fwi_stats()
        self._check(fwi_get_stats(self.handle, byref(st)))
        ks = {}
        for i in range(st.n_kernel_stats):
            k = st.kernels[i]
            ks[k.name.decode()] = dict(ms=k.ms, launches=int(k.launches), bytes=k.bytes,
                                       flops=k.flops)
        return int(st.kernel_launches), ks

    def reset_stats(self):
        self._check(fwi_reset_stats(self.handle))

    def jac_forward(self, a):
        y = self.torch.empty((self.n_freq, self.n_t, self.n_elem),
                             dtype=self.torch.complex128, device="cuda")
        self._check(fwi_jac_forward(self.handle, self._m(a, "a"), _ptr(y)))
        return y

    def jac_adjoint(self, y):
        z = self.torch.empty(self.inv_shape, dtype=self.torch.complex128, device="cuda")
        self._check(fwi_jac_adjoint(self.handle,
                                    _dev(y, self.torch.complex128,
                                         self.n_freq * self.n_t * self.n_elem, "y"), _ptr(z)))
        return z


class Server:
    """Owns one fwi_server (continuous batching of reconstructions)."""

    def __init__(self, hbm_budget=0, max_active=4):
        h = c_void_p()
        st = fwi_server_create(c_size_t(int(hbm_budget)), int(max_active), byref(h))
        if st != FWI_OK:
            raise FwiError(st, fwi_last_error(None).decode())
        self.handle = h
        self._pending = {}

    def submit(self, shape, h, c0, elem, freqs, sos0, d_obs, n_iter=5, lam=1e-4, rho=1e-3,
               gamma=1e-5, n_cg=10, dual_step=0.0, precision=FWI_MIXED, tol=1e-6, max_it=1000,
               max_batch=0, tx_angles=None, elem_length=0.0, inv_factor=1, alpha0=0.0,
               refresh_every=1):
        """Queue a reconstruction; host numpy inputs (sos0 float64 of the inversion mesh,
        d_obs [n_freq][N_T][n_elem], complex64 for FWI_MIXED and complex128
        for FWI_FP64).  max_batch limits the right-hand sides per Krylov launch
        (0: all); tx_angles selects plane-wave transmits, elem_length 3-D line
        elements, inv_factor an inversion mesh (sos0 and the result on it),
        alpha0 an attenuating background, refresh_every > 1 the hybrid Born
        schedule of the receiver fields (refreshed every refresh_every
        iterations).
        Returns the request id."""
        req = fwi_request()
        desc, keep = make_desc(shape, h, c0, elem, freqs, precision, tol, max_it, max_batch,
                               tx_angles, elem_length, inv_factor, alpha0,
                               hybrid_born=refresh_every > 1)
        req.problem = desc
        sos0 = np.ascontiguousarray(sos0, dtype=np.float64)
        cdt = np.complex128 if precision == FWI_FP64 else np.complex64
        d_obs = np.ascontiguousarray(d_obs, dtype=cdt)
        n_elem, n_freq, n_t = int(np.asarray(elem).shape[0]), int(len(freqs)), int(desc.n_tx)
        n_t = n_t if n_t > 0 else n_elem
        rf = max(int(inv_factor), 1)
        inv_shape = tuple(s // rf for s in shape)
        if sos0.size != int(np.prod(inv_shape)) or d_obs.size != n_freq * n_t * n_elem:
            raise ValueError(f"sos0 must hold {int(np.prod(inv_shape))} values (inversion mesh) "
                             f"and d_obs {n_freq} x {n_t} x {n_elem}; got {sos0.shape}, "
                             f"{d_obs.shape}")
        req.sos0 = sos0.ctypes.data_as(POINTER(c_double))
        req.d_obs = d_obs.ctypes.data
        req.admm.lambda_, req.admm.rho, req.admm.gamma = lam, rho, gamma
        req.admm.dual_step, req.admm.n_cg, req.admm.m_ref = dual_step, n_cg, None
        req.n_iter = n_iter
        req.refresh_every = int(refresh_every)
        rid = ctypes.c_longlong()
        st = fwi_server_submit(self.handle, byref(req), byref(rid))
        if st != FWI_OK:
            raise FwiError(st, fwi_last_error(None).decode())
        self._pending[rid.value] = inv_shape
        del keep
        return rid.value

    def wait(self, rid):
        """Block until request ``rid`` completes: (sos ndarray or None, result
        dict with the reconstruction's fwi_status in "status")."""
        shape = self._pending.pop(rid)
        sos = np.full(shape, np.nan, dtype=np.float64)
        res = fwi_request_result()
        st = fwi_server_wait(self.handle, ctypes.c_longlong(rid),
                             sos.ctypes.data_as(POINTER(c_double)), byref(res))
        out = {k: getattr(res, k) for k, _ in fwi_request_result._fields_}
        if st == FWI_ERR_INVALID_ARG and res.status == FWI_OK:
            raise FwiError(st, fwi_last_error(None).decode())
        return (sos if out["status"] == FWI_OK else None), out

    def cancel(self, rid):
        """Cancel request ``rid`` (queued or running); its wait then returns
        (None, result with status FWI_ERR_CANCELLED)."""
        st = fwi_server_cancel(self.handle, ctypes.c_longlong(rid))
        if st != FWI_OK:
            raise FwiError(st, fwi_last_error(None).decode())

    def stats(self):
        a, q, b = c_int(), c_int(), c_size_t()
        fwi_server_stats(self.handle, byref(a), byref(q), byref(b))
        return a.value, q.value, b.value

    def close(self):
        if getattr(self, "handle", None) is not None:
            fwi_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
