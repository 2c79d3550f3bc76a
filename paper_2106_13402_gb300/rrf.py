"""Thin Python binding of the C ABI in include/rrf.h (argument marshalling only).

Matrices are torch float64 CUDA tensors in column-major storage: a tensor X of shape (rows, cols)
with X.stride(0) == 1 and X.stride(1) == ld >= rows (make one with ``fortran_empty`` or convert with
``as_fortran``).  Every computation runs in the CUDA library; if it is not built or cannot be loaded
the calls raise, there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "librrf.so")
_lock = threading.Lock()
_lib = None

RRF_OK, RRF_INVALID_ARG, RRF_CUDA_ERROR, RRF_NOT_CONVERGED, RRF_TIMEOUT, RRF_NUMERICAL, RRF_UNSUPPORTED, \
    RRF_WORKSPACE_TOO_SMALL = range(8)
SKETCH_FP64, SKETCH_BF16 = 0, 1

EXPORTED = [
    "rrf_randutv_workspace", "rrf_randutv", "rrf_powerurv_workspace", "rrf_powerurv", "rrf_randutv_host",
    "rrf_powerurv_host", "rrf_randn", "rrf_gemm_workspace", "rrf_gemm", "rrf_panel_qr_workspace", "rrf_panel_qr",
    "rrf_jacobi_svd_workspace", "rrf_jacobi_svd", "rrf_workspace_status", "rrf_status_string",
    "rrf_last_arg_error", "rrf_version", "rrf_launch_count", "rrf_gemm_profile_begin", "rrf_gemm_profile_end",
    "rrf_gemm_bf16_workspace", "rrf_gemm_bf16", "rrf_batch_plan_create", "rrf_batch_plan_workspace",
    "rrf_batch_plan_tiles", "rrf_batch_plan_destroy", "rrf_powerurv_batched_f32", "rrf_mlp_param_count",
    "rrf_mlp_train_workspace", "rrf_mlp_forward", "rrf_mlp_grad", "rrf_mlp_adam", "rrf_gemm_emulated_workspace",
    "rrf_gemm_emulated", "rrf_gemm_profile_emulated", "rrf_low_rank_workspace", "rrf_low_rank",
    "rrf_gemm_profile_bf16", "rrf_test_inject", "rrf_gemm_profile_emulated_bytes", "rrf_gemm_profile_panel",
]


class RrfError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        name = lib().rrf_status_string(status).decode() if _lib is not None else str(status)
        arg = lib().rrf_last_arg_error() if _lib is not None else 0
        super().__init__(f"{what}: {name}" + (f" (argument {arg})" if arg else ""))


class Opts(ctypes.Structure):
    _fields_ = [("sketch_prec", ctypes.c_int), ("reorth", ctypes.c_int),
                ("q_per_block", ctypes.POINTER(ctypes.c_int)), ("q_policy", ctypes.c_int),
                ("mlp_params", ctypes.c_void_p), ("q_used_out", ctypes.POINTER(ctypes.c_int)),
                ("features_out", ctypes.POINTER(ctypes.c_float)), ("gemm_mode", ctypes.c_int),
                ("oversample", ctypes.c_int), ("frob_tol", ctypes.c_double),
                ("frob_out", ctypes.POINTER(ctypes.c_double)), ("steps_out", ctypes.POINTER(ctypes.c_int)),
                ("resume_steps", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


Q_FIXED, Q_LEARNED = 0, 1
GEMM_AUTO, GEMM_NATIVE, GEMM_EMULATED = 0, 1, 2
INJECT_NONE, INJECT_PANEL_STALL, INJECT_GEMM_STALL, INJECT_JACOBI_CAP = 0, 1, 2, 3


_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Load librrf.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"CUDA library {_LIB_PATH} is not built; run __graft_entry__.build()")
            L = ctypes.CDLL(_LIB_PATH)
            fact = [_i64, _i64, _vp, _i64, _i64, ctypes.c_int, _vp, _i64, _vp, _i64, _vp, _i64, ctypes.c_uint64,
                    _vp, _sz, ctypes.POINTER(Opts), _vp]
            for name in ("rrf_randutv", "rrf_powerurv"):
                getattr(L, name).argtypes = fact
                getattr(L, name).restype = ctypes.c_int
            hostf = [_i64, _i64, _vp, _i64, _i64, ctypes.c_int, _vp, _i64, _vp, _i64, _vp, _i64, ctypes.c_uint64,
                     ctypes.POINTER(Opts), _vp]
            for name in ("rrf_randutv_host", "rrf_powerurv_host"):
                getattr(L, name).argtypes = hostf
                getattr(L, name).restype = ctypes.c_int
            for name in ("rrf_randutv_workspace", "rrf_powerurv_workspace"):
                getattr(L, name).argtypes = [_i64, _i64, _i64, ctypes.POINTER(Opts)]
                getattr(L, name).restype = _sz
            L.rrf_randn.argtypes = [_i64, _i64, _vp, _i64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _vp]
            L.rrf_randn.restype = ctypes.c_int
            L.rrf_gemm_workspace.argtypes = [_i64, _i64, _i64]
            L.rrf_gemm_workspace.restype = _sz
            L.rrf_gemm.argtypes = [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, ctypes.c_double, _vp, _i64, _vp,
                                   _i64, ctypes.c_double, _vp, _i64, _vp, _sz, _vp]
            L.rrf_gemm.restype = ctypes.c_int
            L.rrf_panel_qr_workspace.argtypes = [_i64, _i64]
            L.rrf_panel_qr_workspace.restype = _sz
            L.rrf_panel_qr.argtypes = [_i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, _vp, _sz, _vp]
            L.rrf_panel_qr.restype = ctypes.c_int
            L.rrf_jacobi_svd_workspace.argtypes = [_i64]
            L.rrf_jacobi_svd_workspace.restype = _sz
            L.rrf_jacobi_svd.argtypes = [_i64, _vp, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _sz, _vp]
            L.rrf_jacobi_svd.restype = ctypes.c_int
            L.rrf_workspace_status.argtypes = [_vp, _vp]
            L.rrf_workspace_status.restype = ctypes.c_int
            L.rrf_status_string.argtypes = [ctypes.c_int]
            L.rrf_status_string.restype = ctypes.c_char_p
            L.rrf_last_arg_error.restype = ctypes.c_int
            L.rrf_version.restype = ctypes.c_char_p
            L.rrf_launch_count.restype = ctypes.c_int64
            L.rrf_gemm_bf16_workspace.argtypes = [_i64, _i64, _i64]
            L.rrf_gemm_bf16_workspace.restype = _sz
            L.rrf_gemm_bf16.argtypes = [_i64, _i64, _i64, ctypes.c_double, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _sz,
                                        _vp]
            L.rrf_gemm_bf16.restype = ctypes.c_int
            L.rrf_gemm_emulated_workspace.argtypes = [_i64, _i64, _i64]
            L.rrf_gemm_emulated_workspace.restype = _sz
            L.rrf_gemm_emulated.argtypes = L.rrf_gemm.argtypes
            L.rrf_gemm_emulated.restype = ctypes.c_int
            L.rrf_mlp_param_count.restype = ctypes.c_int
            L.rrf_mlp_train_workspace.argtypes = [ctypes.c_int]
            L.rrf_mlp_train_workspace.restype = _sz
            L.rrf_mlp_forward.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp]
            L.rrf_mlp_forward.restype = ctypes.c_int
            L.rrf_mlp_grad.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _sz, _vp]
            L.rrf_mlp_grad.restype = ctypes.c_int
            L.rrf_mlp_adam.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_float, _vp]
            L.rrf_mlp_adam.restype = ctypes.c_int
            L.rrf_batch_plan_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_i64),
                                                ctypes.POINTER(_i64), _i64, ctypes.c_int]
            L.rrf_batch_plan_create.restype = ctypes.c_int
            L.rrf_batch_plan_workspace.argtypes = [_vp]
            L.rrf_batch_plan_workspace.restype = _sz
            L.rrf_batch_plan_tiles.argtypes = [_vp, ctypes.c_int]
            L.rrf_batch_plan_tiles.restype = ctypes.c_int
            L.rrf_batch_plan_destroy.argtypes = [_vp]
            L.rrf_batch_plan_destroy.restype = ctypes.c_int
            pp = ctypes.POINTER(_vp)
            L.rrf_powerurv_batched_f32.argtypes = [_vp, pp, ctypes.POINTER(_i64), pp, ctypes.POINTER(_i64), pp,
                                                   ctypes.POINTER(_i64), pp, ctypes.POINTER(_i64), ctypes.c_uint64,
                                                   _vp, _sz, _vp]
            L.rrf_powerurv_batched_f32.restype = ctypes.c_int
            L.rrf_gemm_profile_begin.argtypes = [ctypes.c_int]
            L.rrf_gemm_profile_begin.restype = ctypes.c_int
            L.rrf_gemm_profile_end.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_int64)]
            L.rrf_gemm_profile_end.restype = ctypes.c_int
            L.rrf_gemm_profile_emulated.argtypes = [ctypes.POINTER(ctypes.c_double)] * 3 + [
                ctypes.POINTER(ctypes.c_int64)]
            L.rrf_gemm_profile_emulated.restype = ctypes.c_int
            L.rrf_gemm_profile_bf16.argtypes = [ctypes.POINTER(ctypes.c_double)] * 3 + [ctypes.POINTER(ctypes.c_int64)]
            L.rrf_gemm_profile_bf16.restype = ctypes.c_int
            L.rrf_low_rank_workspace.argtypes = [_i64, _i64, _i64]
            L.rrf_low_rank_workspace.restype = _sz
            L.rrf_low_rank.argtypes = [_i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _sz, _vp]
            L.rrf_low_rank.restype = ctypes.c_int
            L.rrf_gemm_profile_panel.argtypes = [ctypes.POINTER(ctypes.c_double)] * 3 + [ctypes.POINTER(ctypes.c_int64)]
            L.rrf_gemm_profile_panel.restype = ctypes.c_int
            L.rrf_gemm_profile_emulated_bytes.argtypes = [ctypes.POINTER(ctypes.c_double)]
            L.rrf_gemm_profile_emulated_bytes.restype = ctypes.c_int
            L.rrf_test_inject.argtypes = [ctypes.c_int, ctypes.c_longlong]
            L.rrf_test_inject.restype = ctypes.c_int
            _lib = L
    return _lib


# ------------------------------------------------------------------------------------------------ helpers
def _torch():
    import torch
    return torch


def fortran_empty(rows: int, cols: int, device="cuda", dtype=None):
    torch = _torch()
    dtype = dtype or torch.float64
    return torch.empty((cols, rows), device=device, dtype=dtype).t()


def as_fortran(x):
    if x.dim() == 2 and x.numel() == 0:
        return fortran_empty(x.shape[0], x.shape[1], x.device, x.dtype)
    if x.dim() == 2 and x.stride(0) == 1 and x.stride(1) >= max(1, x.shape[0]):
        return x
    return x.t().contiguous().t()


def _ld(x) -> int:
    assert x.dim() == 2, "matrix expected"
    if x.numel() == 0:
        return max(int(x.shape[0]), 1)
    assert x.stride(0) == 1 and x.stride(1) >= x.shape[0], "column-major (stride (1, ld)) tensor expected"
    return max(int(x.stride(1)), int(x.shape[0]), 1)


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(st: int, what: str):
    if st != RRF_OK:
        raise RrfError(st, what)


def make_opts(sketch_prec: int = SKETCH_FP64, reorth: bool = False, q_per_block=None, q_policy: int = Q_FIXED,
              mlp_params=None, steps: int = 0, gemm_mode: int = GEMM_AUTO, oversample: int = 0,
              frob_tol: float = 0.0, track_frob: bool = False, resume_steps: int = 0):
    """rrf_opts.  With q_policy=Q_LEARNED, pass `steps` (= ceil(n/b)) to receive per-step q and features in
    opts.q_used / opts.features after the call; mlp_params is a CUDA float16 tensor of rrf_mlp_param_count
    values (None: features only, q stays fixed).  oversample = p > 0 selects randUTV_boosted (Algorithm 2).
    frob_tol > 0 stops at the first step whose trailing Frobenius norm e_i <= frob_tol (Sec. 4.1);
    with track_frob (needs `steps`) opts_frob(o) returns e_0 .. e_done and opts_steps_done(o) the count.
    resume_steps = s0 > 0 continues a factorization stopped after s0 steps (U, T, V passed as `out`)."""
    o = Opts()
    o.sketch_prec = int(sketch_prec)
    o.reorth = 1 if reorth else 0
    o.q_policy = int(q_policy)
    o.gemm_mode = int(gemm_mode)
    o.oversample = int(oversample)
    o.frob_tol = float(frob_tol)
    o.resume_steps = int(resume_steps)
    keep = []
    if track_frob or frob_tol > 0:
        sd = ctypes.c_int(-1)
        o.steps_out = ctypes.pointer(sd)
        keep.append(sd)
        o._steps_done = sd
    if track_frob:
        if steps <= 0:
            raise ValueError("track_frob needs steps = ceil(n / b)")
        fr = (ctypes.c_double * (steps + 1))()
        o.frob_out = ctypes.cast(fr, ctypes.POINTER(ctypes.c_double))
        keep.append(fr)
        o._frob = fr
    if q_per_block is not None:
        qa = (ctypes.c_int * len(q_per_block))(*[int(v) for v in q_per_block])
        o.q_per_block = ctypes.cast(qa, ctypes.POINTER(ctypes.c_int))
        keep.append(qa)
    if mlp_params is not None:
        o.mlp_params = mlp_params.data_ptr()
        keep.append(mlp_params)
    if steps > 0:
        qu = (ctypes.c_int * steps)()
        fo = (ctypes.c_float * (16 * steps))()
        o.q_used_out = ctypes.cast(qu, ctypes.POINTER(ctypes.c_int))
        o.features_out = ctypes.cast(fo, ctypes.POINTER(ctypes.c_float))
        keep += [qu, fo]
        o._qu, o._fo, o._steps = qu, fo, steps
    o._keep = keep
    return o


def opts_steps_done(o) -> int:
    """Number of randUTV steps the last call with these options performed."""
    return int(o._steps_done.value)


def opts_frob(o):
    """e_0 = ||A||_F, e_1, ..., e_done of the Frobenius recurrence (Sec. 4.1) from the last call."""
    return [float(o._frob[j]) for j in range(opts_steps_done(o) + 1)]


def opts_q_used(o):
    return [int(v) for v in o._qu]


def opts_features(o):
    return np.array(o._fo[:], dtype=np.float32).reshape(o._steps, 16)


def workspace(nbytes: int, device="cuda"):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# --------------------------------------------------------------------------------------- factorizations
def _factor(name: str, A, b: int, q: int, seed: int, opts=None, ws=None, out=None, stream=None,
            check_status: bool = True):
    L = lib()
    m, n = A.shape
    A = as_fortran(A)
    if out is None:
        U = fortran_empty(m, m, A.device)
        T = fortran_empty(m, n, A.device)
        V = fortran_empty(n, n, A.device)
    else:
        U, T, V = out
    optp = ctypes.byref(opts) if opts is not None else None
    need = getattr(L, name + "_workspace")(m, n, b, optp)
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    st = getattr(L, name)(m, n, _vp(A.data_ptr()), _ld(A), b, q, _vp(U.data_ptr()), _ld(U), _vp(T.data_ptr()),
                          _ld(T), _vp(V.data_ptr()), _ld(V), seed, _vp(ws.data_ptr()), ws.numel(), optp,
                          _stream(stream))
    _check(st, name)
    if check_status:
        _check(L.rrf_workspace_status(_vp(ws.data_ptr()), _stream(stream)), name + " (device status)")
    return U, T, V


def randutv(A, b: int, q: int, seed: int, opts=None, ws=None, out=None, stream=None, check_status=True):
    """rrf_randutv: randUTV_basic (Algorithm 3), or with opts randUTV_boosted (Algorithm 2), early termination
    or resume (Sec. 4.1); m < n goes through A^T.  Returns (U, T, V) as column-major CUDA tensors; out=(U, A, V)
    factors in place."""
    return _factor("rrf_randutv", A, b, q, seed, opts, ws, out, stream, check_status)


def powerurv(A, b: int, q: int, seed: int, opts=None, ws=None, out=None, stream=None, check_status=True):
    """powerURV (Algorithm 1) through rrf_powerurv: returns (U, R, V); b is the QR panel width."""
    return _factor("rrf_powerurv", A, b, q, seed, opts, ws, out, stream, check_status)


def randutv_workspace_bytes(m: int, n: int, b: int, opts=None) -> int:
    return int(lib().rrf_randutv_workspace(m, n, b, ctypes.byref(opts) if opts is not None else None))


def powerurv_workspace_bytes(m: int, n: int, b: int, opts=None) -> int:
    return int(lib().rrf_powerurv_workspace(m, n, b, ctypes.byref(opts) if opts is not None else None))


def _host_factor(name: str, A: np.ndarray, b: int, q: int, seed: int, opts=None, out=None, stream=None):
    L = lib()
    A = np.asfortranarray(A, dtype=np.float64)
    m, n = A.shape
    if out is None:
        U = np.empty((m, m), order="F")
        T = np.empty((m, n), order="F")
        V = np.empty((n, n), order="F")
    else:
        U, T, V = out
    optp = ctypes.byref(opts) if opts is not None else None
    sp = _stream(stream) if stream is not None else None

    def p(x):
        return _vp(x.ctypes.data)

    st = getattr(L, name)(m, n, p(A), m, b, q, p(U), m, p(T), m, p(V), n, seed, optp, sp)
    _check(st, name)
    return U, T, V


def randutv_host(A, b: int, q: int, seed: int, opts=None, out=None, stream=None):
    """rrf_randutv_host: numpy (host) in and out, device buffers managed by the library."""
    return _host_factor("rrf_randutv_host", A, b, q, seed, opts, out, stream)


def powerurv_host(A, b: int, q: int, seed: int, opts=None, out=None, stream=None):
    return _host_factor("rrf_powerurv_host", A, b, q, seed, opts, out, stream)


# ---------------------------------------------------------------------------------------- building blocks
def randn(rows: int, cols: int, seed: int, step: int, tag: int, device="cuda", stream=None):
    G = fortran_empty(rows, cols, device)
    _check(lib().rrf_randn(rows, cols, _vp(G.data_ptr()), max(rows, 1), seed, step, tag, _stream(stream)),
           "rrf_randn")
    return G


def gemm(transa: str, transb: str, A, B, alpha: float = 1.0, beta: float = 0.0, C=None, stream=None,
         emulated: bool = False):
    """C = alpha op(A) op(B) + beta C in FP64: the DFMA kernel (rrf_gemm) or the emulation on the BF16
    tensor cores (rrf_gemm_emulated)."""
    L = lib()
    A = as_fortran(A)
    B = as_fortran(B)
    m = A.shape[1] if transa == "T" else A.shape[0]
    k = A.shape[0] if transa == "T" else A.shape[1]
    n = B.shape[0] if transb == "T" else B.shape[1]
    if C is None:
        C = fortran_empty(m, n, A.device)
        C.zero_()
    need = L.rrf_gemm_emulated_workspace(m, n, k) if emulated else L.rrf_gemm_workspace(m, n, k)
    ws = workspace(need, A.device) if need else None
    fn = L.rrf_gemm_emulated if emulated else L.rrf_gemm
    st = fn(transa.encode(), transb.encode(), m, n, k, alpha, _vp(A.data_ptr()), _ld(A),
                    _vp(B.data_ptr()), _ld(B), beta, _vp(C.data_ptr()), _ld(C),
                    _vp(ws.data_ptr()) if ws is not None else None, ws.numel() if ws is not None else 0,
                    _stream(stream))
    _check(st, "rrf_gemm_emulated" if emulated else "rrf_gemm")
    if emulated:
        _check(L.rrf_workspace_status(_vp(ws.data_ptr()), _stream(stream)), "rrf_gemm_emulated (device status)")
    return C


def low_rank(U, T, V, k: int, stream=None):
    """rrf_low_rank: the rank-k approximation A_k = U(:, :k) (T(:k, :) V^T) of a (partial) randUTV
    factorization (Sec. 4.1); ||A - A_k|| equals ||T(k:, k:)|| in the 2- and Frobenius norms."""
    L = lib()
    m, n = T.shape
    U, T, V = as_fortran(U), as_fortran(T), as_fortran(V)
    Ak = fortran_empty(m, n, T.device)
    ws = workspace(L.rrf_low_rank_workspace(m, n, k), T.device)
    st = L.rrf_low_rank(m, n, k, _vp(U.data_ptr()), _ld(U), _vp(T.data_ptr()), _ld(T), _vp(V.data_ptr()), _ld(V),
                        _vp(Ak.data_ptr()), _ld(Ak), _vp(ws.data_ptr()), ws.numel(), _stream(stream))
    _check(st, "rrf_low_rank")
    return Ak


def gemm_bf16(A, B, alpha: float = 1.0, stream=None):
    """D = alpha A B^T (FP64, column-major) from BF16 tensors A (m x k) and B (n x k) with contiguous rows
    (row stride a multiple of 8 elements), FP32 accumulation on the tensor cores."""
    torch = _torch()
    L = lib()
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16
    assert A.stride(1) == 1 and B.stride(1) == 1
    m, k = A.shape
    n = B.shape[0]
    D = fortran_empty(m, n, A.device)
    ws = workspace(L.rrf_gemm_bf16_workspace(m, n, k), A.device)
    st = L.rrf_gemm_bf16(m, n, k, alpha, _vp(A.data_ptr()), A.stride(0), _vp(B.data_ptr()), B.stride(0),
                         _vp(D.data_ptr()), _ld(D), _vp(ws.data_ptr()), ws.numel(), _stream(stream))
    _check(st, "rrf_gemm_bf16")
    _check(L.rrf_workspace_status(_vp(ws.data_ptr()), _stream(stream)), "rrf_gemm_bf16 (device status)")
    return D


def panel_qr(P, want_tf: bool = True, stream=None):
    """Householder QR of a panel (in place): returns (P, tau, Y, Tf)."""
    torch = _torch()
    L = lib()
    P = as_fortran(P)
    r, w = P.shape
    tau = torch.empty(w, dtype=torch.float64, device=P.device)
    Y = fortran_empty(r, w, P.device)
    Tf = fortran_empty(w, w, P.device) if want_tf else None
    need = L.rrf_panel_qr_workspace(r, w)
    ws = workspace(need, P.device)
    st = L.rrf_panel_qr(r, w, _vp(P.data_ptr()), _ld(P), _vp(tau.data_ptr()), _vp(Y.data_ptr()), _ld(Y),
                        _vp(Tf.data_ptr()) if Tf is not None else None, w, _vp(ws.data_ptr()), ws.numel(),
                        _stream(stream))
    _check(st, "rrf_panel_qr")
    _check(L.rrf_workspace_status(_vp(ws.data_ptr()), _stream(stream)), "rrf_panel_qr (device status)")
    return P, tau, Y, Tf


def jacobi_svd(M, stream=None, check_status=True):
    """One-sided Jacobi SVD of a c x c block: returns (Us, s, Vs, status)."""
    torch = _torch()
    L = lib()
    M = as_fortran(M)
    c = M.shape[0]
    Us = fortran_empty(c, c, M.device)
    Vs = fortran_empty(c, c, M.device)
    s = torch.empty(c, dtype=torch.float64, device=M.device)
    ws = workspace(L.rrf_jacobi_svd_workspace(c), M.device)
    st = L.rrf_jacobi_svd(c, _vp(M.data_ptr()), _ld(M), _vp(Us.data_ptr()), c, _vp(s.data_ptr()),
                          _vp(Vs.data_ptr()), c, _vp(ws.data_ptr()), ws.numel(), _stream(stream))
    _check(st, "rrf_jacobi_svd")
    dev = L.rrf_workspace_status(_vp(ws.data_ptr()), _stream(stream))
    if check_status:
        _check(dev, "rrf_jacobi_svd (device status)")
    return Us, s, Vs, dev


def launch_count() -> int:
    """Kernels the library has launched in this process (diagnostics)."""
    return int(lib().rrf_launch_count())


def gemm_profile_begin(max_launches: int = 100000):
    if lib().rrf_gemm_profile_begin(int(max_launches)) != 0:
        raise RuntimeError("rrf_gemm_profile_begin failed")


def gemm_profile_end():
    """Returns (total GEMM device ms, algorithmic flops, launches) since gemm_profile_begin."""
    ms, fl, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    if lib().rrf_gemm_profile_end(ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(n)) != 0:
        raise RuntimeError("rrf_gemm_profile_end failed")
    return ms.value, fl.value, n.value


def gemm_profile_emulated():
    """After gemm_profile_end: (device ms, FP64-equivalent flops, tensor flops, launches) of the emulated
    GEMM's tensor-core kernel."""
    ms, fl, tf, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    if lib().rrf_gemm_profile_emulated(ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(tf), ctypes.byref(n)) != 0:
        raise RuntimeError("rrf_gemm_profile_emulated failed")
    return ms.value, fl.value, tf.value, n.value


def gemm_profile_emulated_bytes() -> float:
    """After gemm_profile_end: algorithmic DRAM bytes of the emulated GEMM's timed tensor-core launches."""
    b = ctypes.c_double()
    if lib().rrf_gemm_profile_emulated_bytes(ctypes.byref(b)) != 0:
        raise RuntimeError("rrf_gemm_profile_emulated_bytes failed")
    return b.value


def gemm_profile_panel():
    """After gemm_profile_end: (device ms, HQR flops, algorithmic bytes, launches) of the panel kernel."""
    ms, fl, by, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    if lib().rrf_gemm_profile_panel(ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(by), ctypes.byref(n)) != 0:
        raise RuntimeError("rrf_gemm_profile_panel failed")
    return ms.value, fl.value, by.value, n.value


def gemm_profile_bf16():
    """After gemm_profile_end: (device ms, flops, algorithmic bytes, launches) of the BF16 sketch GEMM's
    tensor-core kernel."""
    ms, fl, by, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    if lib().rrf_gemm_profile_bf16(ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(by), ctypes.byref(n)) != 0:
        raise RuntimeError("rrf_gemm_profile_bf16 failed")
    return ms.value, fl.value, by.value, n.value


def test_inject(kind: int, value: int = 1):
    """rrf_test_inject: drive a bounded wait or the Jacobi sweep cap into its failure path (tests only);
    INJECT_NONE restores normal operation."""
    _check(lib().rrf_test_inject(int(kind), int(value)), "rrf_test_inject")


class injected:
    """Context manager: failure injection `kind` with `value` inside the block, normal operation after."""

    def __init__(self, kind: int, value: int):
        self.kind, self.value = kind, value

    def __enter__(self):
        test_inject(self.kind, self.value)
        return self

    def __exit__(self, *exc):
        test_inject(INJECT_NONE, 0)
        return False


def mlp_param_count() -> int:
    return int(lib().rrf_mlp_param_count())


def mlp_forward(params, X, stream=None):
    """Logits (N x 4, FP32) of the policy MLP for features X (N x 16, FP32, CUDA)."""
    torch = _torch()
    X = X.contiguous().float()
    N = X.shape[0]
    out = torch.empty(N, 4, dtype=torch.float32, device=X.device)
    _check(lib().rrf_mlp_forward(_vp(params.data_ptr()), _vp(X.data_ptr()), N, _vp(out.data_ptr()), _stream(stream)),
           "rrf_mlp_forward")
    return out


def mlp_grad(params, X, labels, ws=None, stream=None):
    """(gradient packed like the parameters, mean loss) of softmax cross-entropy over the samples."""
    torch = _torch()
    L = lib()
    X = X.contiguous().float()
    labels = labels.contiguous().to(torch.int32)
    N = X.shape[0]
    grad = torch.empty(mlp_param_count(), dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    need = L.rrf_mlp_train_workspace(N)
    if ws is None or ws.numel() < need:
        ws = workspace(need, X.device)
    _check(L.rrf_mlp_grad(_vp(params.data_ptr()), _vp(X.data_ptr()), _vp(labels.data_ptr()), N, _vp(grad.data_ptr()),
                          _vp(loss.data_ptr()), _vp(ws.data_ptr()), ws.numel(), _stream(stream)), "rrf_mlp_grad")
    return grad, loss


def mlp_adam(master, m, v, grad, params, step: int, lr: float, stream=None):
    _check(lib().rrf_mlp_adam(_vp(master.data_ptr()), _vp(m.data_ptr()), _vp(v.data_ptr()), _vp(grad.data_ptr()),
                              _vp(params.data_ptr()), step, lr, _stream(stream)), "rrf_mlp_adam")


class BatchPlan:
    """Batched FP32 powerURV over matrices of uneven shape (rrf_batch_plan_* / rrf_powerurv_batched_f32).
    The first run autotunes, captures a CUDA graph and launches it; later runs with the same buffers replay
    the graph."""

    def __init__(self, shapes, b: int = 64, q: int = 1):
        L = lib()
        self.shapes = [(int(m), int(n)) for m, n in shapes]
        cnt = len(self.shapes)
        ms = (_i64 * cnt)(*[m for m, _ in self.shapes])
        ns = (_i64 * cnt)(*[n for _, n in self.shapes])
        h = _vp()
        _check(L.rrf_batch_plan_create(ctypes.byref(h), cnt, ms, ns, b, q), "rrf_batch_plan_create")
        self._h = h
        self.b, self.q = b, q

    def workspace_bytes(self) -> int:
        return int(lib().rrf_batch_plan_workspace(self._h))

    def tiles(self):
        L = lib()
        return L.rrf_batch_plan_tiles(self._h, 0), L.rrf_batch_plan_tiles(self._h, 1)

    def allocate(self, device="cuda"):
        torch = _torch()
        U = [fortran_empty(m, m, device, torch.float32) for m, n in self.shapes]
        T = [fortran_empty(m, n, device, torch.float32) for m, n in self.shapes]
        V = [fortran_empty(n, n, device, torch.float32) for m, n in self.shapes]
        return U, T, V

    def run(self, As, out, seed: int, ws, stream=None):
        L = lib()
        U, T, V = out
        cnt = len(self.shapes)

        def ptrs(xs):
            return (_vp * cnt)(*[x.data_ptr() for x in xs])

        def lds(xs):
            return (_i64 * cnt)(*[_ld(x) for x in xs])

        self._keep = [ptrs(As), lds(As), ptrs(U), lds(U), ptrs(T), lds(T), ptrs(V), lds(V)]
        k = self._keep
        st = L.rrf_powerurv_batched_f32(self._h, k[0], k[1], k[2], k[3], k[4], k[5], k[6], k[7], seed,
                                        _vp(ws.data_ptr()), ws.numel(), _stream(stream))
        _check(st, "rrf_powerurv_batched_f32")
        return U, T, V

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None and _lib is not None:
                _lib.rrf_batch_plan_destroy(self._h)
        except Exception:
            pass


def version() -> str:
    return lib().rrf_version().decode()
