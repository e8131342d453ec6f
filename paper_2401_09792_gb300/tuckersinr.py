"""Python binding of ``libtuckersinr.so`` (C ABI in ``include/tuckersinr.h``).

Argument marshalling only: every step of the SINR path runs in the CUDA
library.  Tensors are PyTorch CUDA tensors used as device memory; complex
arrays are ``torch.complex64`` (interleaved re/im, the ABI's ``ts_c64``).
Functions carry the C names (``ts_sinr_svd`` ...) and raise ``TsError`` on a
non-zero status.  There is no CPU fallback: if the library or a GPU is
missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtuckersinr.so")

TS_COEF_DENSE, TS_COEF_PATHS = 0, 1
TS_OK, TS_ERR_DIMS, TS_ERR_NULL, TS_ERR_ALIGN, TS_ERR_WORKSPACE = 0, 1, 2, 3, 4
TS_OP_SINR_SVD, TS_OP_SINR_MMSE, TS_OP_DENSE_SVD, TS_OP_DENSE_MMSE = 0, 1, 2, 3
TS_OP_SINR_SVD_ADJOINT, TS_OP_SINR_MMSE_ADJOINT, TS_OP_TUCKER_FIT = 4, 5, 6
TS_OP_SINR_SVD_TF32, TS_OP_SINR_SVD_BF16X2, TS_OP_SINR_SVD_TF32X3 = 7, 8, 14
TS_OP_TUCKER_FIT_SHARED, TS_OP_TUCKER_FIT_INDIVIDUAL, TS_OP_RECONSTRUCT = 9, 10, 11
TS_MODEL_GROUPWISE, TS_MODEL_SHARED, TS_MODEL_INDIVIDUAL = 0, 1, 2
TS_OP_SINR_SVD_MULTIUSER, TS_OP_DENSE_SVD_MULTIUSER = 12, 13
TS_PREC_FP32, TS_PREC_TF32, TS_PREC_BF16X2, TS_PREC_TF32X3 = 0, 1, 2, 3
TS_FLAG_NOT_PD, TS_FLAG_NONFINITE, TS_FLAG_RANK_DEFICIENT, TS_FLAG_EIG_UNCONVERGED = 1, 2, 4, 8
TS_FLAG_TIMEOUT = 16
TS_FLAG_REFINED = 32
TS_FLAG_PRECODER_REFINED = 64
# bits that report a problem (the two REFINED bits are informational)
TS_FLAG_ERRORS = 0xFF & ~(TS_FLAG_REFINED | TS_FLAG_PRECODER_REFINED)


class TsError(RuntimeError):
    """A tuckersinr call returned a non-zero status."""

    def __init__(self, fn: str, status: int, lib=None):
        msg = lib.ts_status_string(status).decode() if lib is not None else str(status)
        extra = ""
        if lib is not None and status == 5:
            extra = f" (cudaError {lib.ts_last_cuda_error()})"
        super().__init__(f"{fn}: status {status}: {msg}{extra}")
        self.status = status


class ts_dims(ctypes.Structure):
    _fields_ = [("J", ctypes.c_int32), ("M", ctypes.c_int32), ("N", ctypes.c_int32),
                ("P", ctypes.c_int32), ("m", ctypes.c_int32), ("n", ctypes.c_int32),
                ("p", ctypes.c_int32), ("K", ctypes.c_int32), ("L", ctypes.c_int32),
                ("delta_f_hz", ctypes.c_float)]


class ts_coef(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("c", ctypes.c_void_p), ("alpha", ctypes.c_void_p),
                ("tau_s", ctypes.c_void_p)]


class ts_instance(ctypes.Structure):
    _fields_ = [("d", ts_dims), ("op", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("coef", ts_coef), ("G", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("Pt", ctypes.c_void_p), ("sigma2", ctypes.c_void_p), ("sinr", ctypes.c_void_p),
                ("flags", ctypes.c_void_p)]


TS_BATCH_AUTOTUNE = 1

_P = ctypes.c_void_p
_SIG = {
    "ts_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ts_last_cuda_error": (ctypes.c_int, []),
    "ts_abi_version": (ctypes.c_int, []),
    "ts_set_timing_events": (None, [_P, _P]),
    "ts_set_phase_event": (None, [_P]),
    "ts_set_refinement": (None, [ctypes.c_float]),
    "ts_device_peaks": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), _P]),
    "ts_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(ts_dims), ctypes.c_int]),
    "ts_coefficients": (ctypes.c_int, [ctypes.POINTER(ts_dims), _P, _P, _P, _P]),
    "ts_project_precoder": (ctypes.c_int, [ctypes.POINTER(ts_dims), _P, _P, _P, _P]),
    "ts_sinr_mmse": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.POINTER(ts_coef), _P, _P, _P,
                                    _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "ts_sinr_svd": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.POINTER(ts_coef), _P, _P, _P,
                                   _P, _P, _P, ctypes.c_size_t, _P]),
    "ts_sinr_svd_range": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ts_coef), _P, _P, _P, ctypes.c_int, _P, _P,
                                         _P, ctypes.c_size_t, _P]),
    "ts_sinr_mmse_range": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ts_coef), _P, _P, _P, _P, _P, _P, _P,
                                          ctypes.c_size_t, _P]),
    "ts_dense_sinr_svd": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.POINTER(ts_coef), _P, _P,
                                         _P, _P, _P, ctypes.c_size_t, _P]),
    "ts_dense_sinr_mmse": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.POINTER(ts_coef), _P, _P,
                                          _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "ts_tucker_fit": (ctypes.c_int, [ctypes.POINTER(ts_dims), _P, ctypes.c_int, ctypes.c_int, _P, _P,
                                     _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "ts_sinr_svd_multiuser": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.c_int,
                                             ctypes.POINTER(ts_coef), _P, _P, _P, _P, _P, _P,
                                             ctypes.c_size_t, _P]),
    "ts_dense_sinr_svd_multiuser": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.c_int,
                                                   ctypes.POINTER(ts_coef), _P, _P, _P, _P, _P,
                                                   ctypes.c_size_t, _P]),
    "ts_set_fit_iterations": (None, [ctypes.c_int]),
    "ts_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, _P, _P]),
    "ts_tucker_fit_model": (ctypes.c_int, [ctypes.POINTER(ts_dims), _P, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "ts_tucker_reconstruct": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.c_int, _P, _P, _P, _P, _P,
                                             _P, ctypes.c_size_t, _P]),
    "ts_sinr_svd_adjoint": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.POINTER(ts_coef), _P, _P,
                                           _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "ts_sinr_mmse_adjoint": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.POINTER(ts_coef), _P, _P,
                                            _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "ts_project_precoder_adjoint": (ctypes.c_int, [ctypes.POINTER(ts_dims), _P, _P, _P, _P]),
    "ts_sinr_mmse_noalloc": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.POINTER(ts_coef), _P, _P,
                                            _P, _P, _P, _P, _P]),
    "ts_svd_precoders": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.POINTER(ts_coef), _P, _P,
                                        _P, ctypes.c_size_t, _P]),
    "ts_sinr_svd_from_precoders": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.POINTER(ts_coef),
                                                  _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "ts_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(ts_instance), ctypes.c_int]),
    "ts_batch_plan_create": (ctypes.c_int, [ctypes.POINTER(ts_instance), ctypes.c_int, _P, ctypes.c_size_t,
                                            ctypes.c_int, ctypes.POINTER(_P)]),
    "ts_batch_launch": (ctypes.c_int, [_P, _P]),
    "ts_batch_plan_destroy": (None, [_P]),
    "ts_autotune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "ts_autotune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "ts_sinr_svd_prec": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.POINTER(ts_coef), _P, _P, _P,
                                        ctypes.c_int, _P, _P, _P, ctypes.c_size_t, _P]),
    "ts_sinr_svd_from_precoders_prec": (ctypes.c_int, [ctypes.POINTER(ts_dims), ctypes.POINTER(ts_coef),
                                                       _P, _P, _P, ctypes.c_int, _P, _P, _P,
                                                       ctypes.c_size_t, _P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (once) and declare every exported signature."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it first (__graft_entry__.build())")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIG.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


@dataclass(frozen=True)
class Dims:
    """Sizes of one system (see ts_dims)."""

    J: int
    M: int
    N: int
    P: int
    m: int
    n: int
    p: int
    K: int
    L: int
    delta_f_hz: float = 15e3

    def c(self) -> ts_dims:
        return ts_dims(self.J, self.M, self.N, self.P, self.m, self.n, self.p, self.K, self.L,
                       self.delta_f_hz)

    @staticmethod
    def of(w) -> "Dims":
        return Dims(w.J, w.M, w.N, w.P, w.m, w.n, w.p, w.K, w.L, w.delta_f_hz)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int | None:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


def _check(fn: str, st: int):
    if st != 0:
        raise TsError(fn, st, _lib)


def ts_device_peaks(stream=None) -> dict:
    """Measured FP32 FMA, TF32 tensor-core and FP64 FMA throughput (TFLOP/s)."""
    f32, t32, f64 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check("ts_device_peaks", load().ts_device_peaks(ctypes.byref(f32), ctypes.byref(t32),
                                                     ctypes.byref(f64), _stream(stream)))
    return {"fp32_fma": f32.value, "tf32_mma": t32.value, "fp64_fma": f64.value}


def ts_set_refinement(threshold: float):
    """Sensitivity threshold above which a unit is re-evaluated from a
    double-float R with FP64-residual refinement (default 8, this thread);
    negative turns it off."""
    load().ts_set_refinement(float(threshold))


def ts_set_timing_events(start=None, stop=None):
    """Record two torch.cuda.Event objects around the dominant kernel of the
    following SINR calls on this thread (None, None: off)."""
    h = lambda e: None if e is None else e.cuda_event  # noqa: E731
    load().ts_set_timing_events(h(start), h(stop))


def ts_set_phase_event(event=None):
    """Record a torch.cuda.Event between the precoder and link phases of the
    following SVD-precoded SINR calls on this thread (None: off)."""
    load().ts_set_phase_event(None if event is None else event.cuda_event)


def ts_workspace_bytes(d: Dims, op: int) -> int:
    return load().ts_workspace_bytes(ctypes.byref(d.c()), op)


def workspace(d: Dims, op: int, device="cuda") -> torch.Tensor:
    """A device workspace buffer for `op` (PyTorch allocations are 256-byte aligned)."""
    nb = ts_workspace_bytes(d, op)
    if nb == 0:
        raise TsError("ts_workspace_bytes", 1, load())
    return torch.empty(nb, dtype=torch.uint8, device=device)


def make_coef(c=None, alpha=None, tau=None) -> tuple[ts_coef, tuple]:
    """Dense (c) or path-form (alpha, tau) coefficients; returns the struct and the
    tensors it points into (keep them alive for the call)."""
    if c is not None:
        return ts_coef(TS_COEF_DENSE, _ptr(c), None, None), (c,)
    return ts_coef(TS_COEF_PATHS, None, _ptr(alpha), _ptr(tau)), (alpha, tau)


def ts_coefficients(d: Dims, alpha, tau, c, stream=None):
    lib = load()
    _check("ts_coefficients", lib.ts_coefficients(ctypes.byref(d.c()), _ptr(alpha), _ptr(tau),
                                                  _ptr(c), _stream(stream)))


def ts_project_precoder(d: Dims, B, Pfull, Pt, stream=None):
    lib = load()
    _check("ts_project_precoder", lib.ts_project_precoder(ctypes.byref(d.c()), _ptr(B), _ptr(Pfull),
                                                          _ptr(Pt), _stream(stream)))


def ts_sinr_mmse(d: Dims, coef: ts_coef, G, C, Pt, sigma2, sinr, flags, ws, stream=None):
    lib = load()
    _check("ts_sinr_mmse", lib.ts_sinr_mmse(ctypes.byref(d.c()), ctypes.byref(coef), _ptr(G), _ptr(C),
                                            _ptr(Pt), _ptr(sigma2), _ptr(sinr), _ptr(flags),
                                            _ptr(ws), ws.numel(), _stream(stream)))


def ts_sinr_svd(d: Dims, coef: ts_coef, G, C, sigma2, sinr, flags, ws, stream=None):
    lib = load()
    _check("ts_sinr_svd", lib.ts_sinr_svd(ctypes.byref(d.c()), ctypes.byref(coef), _ptr(G), _ptr(C),
                                          _ptr(sigma2), _ptr(sinr), _ptr(flags), _ptr(ws),
                                          ws.numel(), _stream(stream)))


def ts_sinr_svd_prec(d: Dims, coef: ts_coef, G, C, sigma2, precision: int, sinr, flags, ws,
                     stream=None):
    lib = load()
    _check("ts_sinr_svd_prec",
           lib.ts_sinr_svd_prec(ctypes.byref(d.c()), ctypes.byref(coef), _ptr(G), _ptr(C), _ptr(sigma2),
                                int(precision), _ptr(sinr), _ptr(flags), _ptr(ws), ws.numel(),
                                _stream(stream)))


def ts_sinr_svd_range(d: Dims, kappa0: int, count: int, coef: ts_coef, G, C, sigma2, precision: int,
                      sinr, flags, ws, stream=None):
    lib = load()
    _check("ts_sinr_svd_range",
           lib.ts_sinr_svd_range(ctypes.byref(d.c()), int(kappa0), int(count), ctypes.byref(coef), _ptr(G),
                                 _ptr(C), _ptr(sigma2), int(precision), _ptr(sinr), _ptr(flags), _ptr(ws),
                                 ws.numel(), _stream(stream)))


def ts_sinr_mmse_range(d: Dims, kappa0: int, count: int, coef: ts_coef, G, C, Pt, sigma2, sinr, flags,
                       ws, stream=None):
    lib = load()
    _check("ts_sinr_mmse_range",
           lib.ts_sinr_mmse_range(ctypes.byref(d.c()), int(kappa0), int(count), ctypes.byref(coef), _ptr(G),
                                  _ptr(C), _ptr(Pt), _ptr(sigma2), _ptr(sinr), _ptr(flags), _ptr(ws),
                                  ws.numel(), _stream(stream)))


def ts_sinr_svd_from_precoders_prec(d: Dims, coef: ts_coef, G, C, sigma2, precision: int, sinr, flags,
                                    ws, stream=None):
    lib = load()
    _check("ts_sinr_svd_from_precoders_prec",
           lib.ts_sinr_svd_from_precoders_prec(ctypes.byref(d.c()), ctypes.byref(coef), _ptr(G), _ptr(C),
                                               _ptr(sigma2), int(precision), _ptr(sinr), _ptr(flags),
                                               _ptr(ws), ws.numel(), _stream(stream)))


def instance(d: Dims, op: int, coef: ts_coef, G, C, sigma2, sinr, flags=None, Pt=None,
             precision: int = TS_PREC_FP32) -> ts_instance:
    """One system of a batch (device tensors in the library's layouts)."""
    return ts_instance(d.c(), op, precision, coef, _ptr(G), _ptr(C), _ptr(Pt), _ptr(sigma2), _ptr(sinr),
                       _ptr(flags))


class BatchPlan:
    """ts_batch_plan_create / ts_batch_launch / ts_batch_plan_destroy."""

    def __init__(self, instances, ws, autotune: bool = False):
        lib = load()
        self._arr = (ts_instance * len(instances))(*instances)
        self._ws = ws
        h = _P()
        _check("ts_batch_plan_create",
               lib.ts_batch_plan_create(self._arr, len(instances), _ptr(ws), ws.numel(),
                                        TS_BATCH_AUTOTUNE if autotune else 0, ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check("ts_batch_launch", load().ts_batch_launch(self._h, _stream(stream)))

    def close(self):
        if self._h:
            load().ts_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_workspace(instances, device="cuda") -> torch.Tensor:
    arr = (ts_instance * len(instances))(*instances)
    nb = load().ts_batch_workspace_bytes(arr, len(instances))
    if nb == 0:
        raise TsError("ts_batch_workspace_bytes", 1, load())
    return torch.empty(nb, dtype=torch.uint8, device=device)


def ts_tucker_fit(d: Dims, X, S, init, A, B, C, G, g_hist, ws, stream=None):
    lib = load()
    _check("ts_tucker_fit", lib.ts_tucker_fit(ctypes.byref(d.c()), _ptr(X), S, init, _ptr(A), _ptr(B),
                                              _ptr(C), _ptr(G), _ptr(g_hist), _ptr(ws), ws.numel(),
                                              _stream(stream)))


def ts_sinr_svd_multiuser(d: Dims, U, coef: ts_coef, G, C, sigma2, sinr, flags, ws, stream=None):
    lib = load()
    _check("ts_sinr_svd_multiuser",
           lib.ts_sinr_svd_multiuser(ctypes.byref(d.c()), U, ctypes.byref(coef), _ptr(G), _ptr(C),
                                     _ptr(sigma2), _ptr(sinr), _ptr(flags), _ptr(ws), ws.numel(),
                                     _stream(stream)))


def ts_dense_sinr_svd_multiuser(d: Dims, U, coef: ts_coef, X, sigma2, sinr, flags, ws, stream=None):
    lib = load()
    _check("ts_dense_sinr_svd_multiuser",
           lib.ts_dense_sinr_svd_multiuser(ctypes.byref(d.c()), U, ctypes.byref(coef), _ptr(X),
                                           _ptr(sigma2), _ptr(sinr), _ptr(flags), _ptr(ws),
                                           ws.numel(), _stream(stream)))


def ts_selftest_bounded_wait(limit: int, arrive: bool, out, stream=None):
    _check("ts_selftest_bounded_wait",
           load().ts_selftest_bounded_wait(int(limit), 1 if arrive else 0, _ptr(out), _stream(stream)))


def ts_set_fit_iterations(iterations: int):
    load().ts_set_fit_iterations(int(iterations))


def ts_tucker_fit_model(d: Dims, X, S, init, model, A, B, C, G, g_hist, ws, stream=None):
    lib = load()
    _check("ts_tucker_fit_model",
           lib.ts_tucker_fit_model(ctypes.byref(d.c()), _ptr(X), S, init, model, _ptr(A), _ptr(B), _ptr(C),
                                   _ptr(G), _ptr(g_hist), _ptr(ws), ws.numel(), _stream(stream)))


def ts_tucker_reconstruct(d: Dims, model, A, B, C, G, Xhat, ws, stream=None):
    lib = load()
    _check("ts_tucker_reconstruct",
           lib.ts_tucker_reconstruct(ctypes.byref(d.c()), model, _ptr(A), _ptr(B), _ptr(C), _ptr(G),
                                     _ptr(Xhat), _ptr(ws), ws.numel(), _stream(stream)))


def ts_sinr_svd_adjoint(d: Dims, coef: ts_coef, G, C, sigma2, dsinr, dG, dC, sinr, ws, stream=None):
    lib = load()
    _check("ts_sinr_svd_adjoint",
           lib.ts_sinr_svd_adjoint(ctypes.byref(d.c()), ctypes.byref(coef), _ptr(G), _ptr(C),
                                   _ptr(sigma2), _ptr(dsinr), _ptr(dG), _ptr(dC), _ptr(sinr),
                                   _ptr(ws), ws.numel(), _stream(stream)))


def ts_sinr_mmse_adjoint(d: Dims, coef: ts_coef, G, C, Pt, sigma2, dsinr, dG, dC, dPt, sinr, ws,
                         stream=None):
    lib = load()
    _check("ts_sinr_mmse_adjoint",
           lib.ts_sinr_mmse_adjoint(ctypes.byref(d.c()), ctypes.byref(coef), _ptr(G), _ptr(C),
                                    _ptr(Pt), _ptr(sigma2), _ptr(dsinr), _ptr(dG), _ptr(dC),
                                    _ptr(dPt), _ptr(sinr), _ptr(ws), ws.numel(), _stream(stream)))


def ts_project_precoder_adjoint(d: Dims, Pfull, dPt, dB, stream=None):
    lib = load()
    _check("ts_project_precoder_adjoint",
           lib.ts_project_precoder_adjoint(ctypes.byref(d.c()), _ptr(Pfull), _ptr(dPt), _ptr(dB),
                                           _stream(stream)))


TS_NOALLOC_SCRATCH_BYTES = 16 << 20


def ts_sinr_mmse_noalloc(d: Dims, coef: ts_coef, G, C, Pt, sigma2, sinr, flags, stream=None):
    """ts_sinr_mmse without a workspace argument: the library's own fixed
    device scratch is used (for callers that cannot allocate at call time)."""
    lib = load()
    _check("ts_sinr_mmse_noalloc",
           lib.ts_sinr_mmse_noalloc(ctypes.byref(d.c()), ctypes.byref(coef), _ptr(G), _ptr(C),
                                    _ptr(Pt), _ptr(sigma2), _ptr(sinr), _ptr(flags),
                                    _stream(stream)))


def ts_svd_precoders(d: Dims, coef: ts_coef, G, C, ws, stream=None):
    lib = load()
    _check("ts_svd_precoders", lib.ts_svd_precoders(ctypes.byref(d.c()), ctypes.byref(coef), _ptr(G),
                                                    _ptr(C), _ptr(ws), ws.numel(), _stream(stream)))


def ts_sinr_svd_from_precoders(d: Dims, coef: ts_coef, G, C, sigma2, sinr, flags, ws, stream=None):
    lib = load()
    _check("ts_sinr_svd_from_precoders",
           lib.ts_sinr_svd_from_precoders(ctypes.byref(d.c()), ctypes.byref(coef), _ptr(G), _ptr(C),
                                          _ptr(sigma2), _ptr(sinr), _ptr(flags), _ptr(ws),
                                          ws.numel(), _stream(stream)))


def ts_dense_sinr_svd(d: Dims, coef: ts_coef, X, sigma2, sinr, flags, ws, stream=None):
    lib = load()
    _check("ts_dense_sinr_svd", lib.ts_dense_sinr_svd(ctypes.byref(d.c()), ctypes.byref(coef), _ptr(X),
                                                      _ptr(sigma2), _ptr(sinr), _ptr(flags), _ptr(ws),
                                                      ws.numel(), _stream(stream)))


def ts_dense_sinr_mmse(d: Dims, coef: ts_coef, X, Pfull, sigma2, sinr, flags, ws, stream=None):
    lib = load()
    _check("ts_dense_sinr_mmse", lib.ts_dense_sinr_mmse(ctypes.byref(d.c()), ctypes.byref(coef),
                                                        _ptr(X), _ptr(Pfull), _ptr(sigma2), _ptr(sinr),
                                                        _ptr(flags), _ptr(ws), ws.numel(),
                                                        _stream(stream)))


def channels_to_device(X, device="cuda") -> torch.Tensor:
    """(J, J, M, N, P) complex -> device [J*J][P][M][N] complex64."""
    import numpy as np
    J, _, M, N, P = X.shape
    a = np.ascontiguousarray(np.transpose(X, (0, 1, 4, 2, 3)).reshape(J * J, P, M, N))
    return torch.from_numpy(a.astype(np.complex64)).to(device)


# ----------------------------------------------------------- layout marshalling
def core_to_device(G, device="cuda") -> torch.Tensor:
    """(J, J, m, n, p) complex -> device [J*J][p][m][n] complex64."""
    import numpy as np
    J, _, m, n, p = G.shape
    a = np.ascontiguousarray(np.transpose(G, (0, 1, 4, 2, 3)).reshape(J * J, p, m, n))
    return torch.from_numpy(a.astype(np.complex64)).to(device)


def factor_to_device(X, device="cuda") -> torch.Tensor:
    """Any complex array -> contiguous complex64 device tensor, leading link axes merged
    when the first two axes are (J, J)."""
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(X).astype(np.complex64)).to(device)


def real_to_device(x, device="cuda") -> torch.Tensor:
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(x).astype(np.float32)).to(device)
