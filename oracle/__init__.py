"""FP64 CPU oracle for randUTV (Algorithm 3) and powerURV (Algorithm 1) -- ctypes binding.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain reference that the CUDA path is checked
against.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA path: the C sources here are compiled by
gcc into their own library and nothing under the CUDA package imports them.

Every matrix crossing this boundary is a Fortran-ordered (column-major) float64 numpy array.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rrf_oracle.c")
_HDR = os.path.join(_HERE, "rrf_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + OpenMP, strict IEEE: no contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_randn.argtypes = [_i64, _i64, _dp, _i64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
            L.orc_gemm.argtypes = [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, ctypes.c_double, _dp, _i64,
                                   _dp, _i64, ctypes.c_double, _dp, _i64]
            L.orc_hqr.argtypes = [_i64, _i64, _dp, _i64, _dp]
            L.orc_larft.argtypes = [_i64, _i64, _dp, _i64, _dp, _dp, _i64]
            L.orc_apply_q.argtypes = [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, _dp, _i64, _dp, _dp, _i64]
            L.orc_form_q.argtypes = [_i64, _i64, _i64, _dp, _i64, _dp, _dp, _i64]
            L.orc_jacobi_svd.argtypes = [_i64, _i64, _dp, _i64, _dp, _i64, _dp, _dp, _i64,
                                         ctypes.POINTER(ctypes.c_int)]
            L.orc_jacobi_svd.restype = ctypes.c_int
            L.orc_randutv.argtypes = [_i64, _i64, _dp, _i64, _i64, ctypes.c_int, ctypes.c_uint64, _dp, _i64,
                                      _dp, _i64, _dp, _i64, ctypes.c_int]
            L.orc_randutv.restype = ctypes.c_int
            L.orc_randutv_reorth.argtypes = L.orc_randutv.argtypes
            L.orc_randutv_reorth.restype = ctypes.c_int
            L.orc_randutv_boosted.argtypes = [_i64, _i64, _dp, _i64, _i64, ctypes.c_int, _i64, ctypes.c_uint64,
                                              _dp, _i64, _dp, _i64, _dp, _i64, ctypes.c_int]
            L.orc_randutv_boosted.restype = ctypes.c_int
            L.orc_powerurv.argtypes = [_i64, _i64, _dp, _i64, ctypes.c_int, ctypes.c_uint64, _dp, _i64, _dp,
                                       _i64, _dp, _i64]
            L.orc_powerurv.restype = ctypes.c_int
            L.orc_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def randn(rows: int, cols: int, seed: int, step: int, tag: int) -> np.ndarray:
    G = np.zeros((rows, cols), dtype=np.float64, order="F")
    if rows * cols:
        lib().orc_randn(rows, cols, _p(G), max(rows, 1), seed, step, tag)
    return G


def gemm(ta: str, tb: str, A, B, alpha: float = 1.0, beta: float = 0.0, C=None) -> np.ndarray:
    A = _f64(A)
    B = _f64(B)
    m = A.shape[1] if ta == "T" else A.shape[0]
    k = A.shape[0] if ta == "T" else A.shape[1]
    n = B.shape[0] if tb == "T" else B.shape[1]
    C = np.zeros((m, n), order="F") if C is None else _f64(C).copy(order="F")
    lib().orc_gemm(ta.encode(), tb.encode(), m, n, k, alpha, _p(A), max(A.shape[0], 1), _p(B),
                   max(B.shape[0], 1), beta, _p(C), max(m, 1))
    return C


def hqr(A):
    A = _f64(A).copy(order="F")
    m, n = A.shape
    tau = np.zeros(max(min(m, n), 1))
    lib().orc_hqr(m, n, _p(A), m, _p(tau))
    return A, tau[: min(m, n)]


def larft(Y, tau) -> np.ndarray:
    Y = _f64(Y)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    m, k = Y.shape[0], len(tau)
    Tf = np.zeros((k, k), order="F")
    lib().orc_larft(m, k, _p(Y), m, _p(tau), _p(Tf), max(k, 1))
    return Tf


def apply_q(side: str, trans: str, Y, tau, C) -> np.ndarray:
    Y = _f64(Y)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    C = _f64(C).copy(order="F")
    m, n = C.shape
    lib().orc_apply_q(side.encode(), trans.encode(), m, n, len(tau), _p(Y), Y.shape[0], _p(tau), _p(C), m)
    return C


def form_q(Y, tau, ncols: int) -> np.ndarray:
    Y = _f64(Y)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    m = Y.shape[0]
    Q = np.zeros((m, ncols), order="F")
    lib().orc_form_q(m, ncols, len(tau), _p(Y), m, _p(tau), _p(Q), m)
    return Q


def jacobi_svd(M):
    M = _f64(M)
    r, c = M.shape
    U = np.zeros((r, c), order="F")
    s = np.zeros(max(c, 1))
    V = np.zeros((c, c), order="F")
    sw = ctypes.c_int(0)
    st = lib().orc_jacobi_svd(r, c, _p(M), r, _p(U), r, _p(s), _p(V), c, ctypes.byref(sw))
    return U, s[:c], V, int(st), int(sw.value)


def randutv(A, b: int, q: int, seed: int, max_steps: int = 0):
    """randUTV_basic (Algorithm 3): returns (U, T, V, status)."""
    A = _f64(A)
    m, n = A.shape
    U = np.zeros((m, m), order="F")
    T = np.zeros((m, n), order="F")
    V = np.zeros((n, n), order="F")
    st = lib().orc_randutv(m, n, _p(A), m, b, q, seed, _p(U), m, _p(T), m, _p(V), n, max_steps)
    return U, T, V, int(st)


def randutv_reorth(A, b: int, q: int, seed: int, max_steps: int = 0):
    """randUTV_basic with the re-orthonormalized power iteration (Sec. 2.5 (ii)): returns (U, T, V, status)."""
    A = _f64(A)
    m, n = A.shape
    U = np.zeros((m, m), order="F")
    T = np.zeros((m, n), order="F")
    V = np.zeros((n, n), order="F")
    st = lib().orc_randutv_reorth(m, n, _p(A), m, b, q, seed, _p(U), m, _p(T), m, _p(V), n, max_steps)
    return U, T, V, int(st)


def randutv_boosted(A, b: int, q: int, p: int, seed: int, max_steps: int = 0):
    """randUTV_boosted (Algorithm 2, oversampling p, recycled samples): returns (U, T, V, status)."""
    A = _f64(A)
    m, n = A.shape
    U = np.zeros((m, m), order="F")
    T = np.zeros((m, n), order="F")
    V = np.zeros((n, n), order="F")
    st = lib().orc_randutv_boosted(m, n, _p(A), m, b, q, p, seed, _p(U), m, _p(T), m, _p(V), n, max_steps)
    return U, T, V, int(st)


def powerurv(A, q: int, seed: int):
    """powerURV (Algorithm 1): returns (U, R, V, status)."""
    A = _f64(A)
    m, n = A.shape
    U = np.zeros((m, m), order="F")
    R = np.zeros((m, n), order="F")
    V = np.zeros((n, n), order="F")
    st = lib().orc_powerurv(m, n, _p(A), m, q, seed, _p(U), m, _p(R), m, _p(V), n)
    return U, R, V, int(st)


# ---------------------------------------------------------------------------------------------------------
# Policy MLP reference (FP64 numpy): 16 -> 64 (ReLU) -> 64 (ReLU) -> 4, softmax cross-entropy.
# Packing: [W1 (64 x 16, row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (4 x 64), b3 (4)].
MLP_SIZES = ((64, 16), (64,), (64, 64), (64,), (4, 64), (4,))


def mlp_unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = [], 0
    for shp in MLP_SIZES:
        k = int(np.prod(shp))
        out.append(p[o:o + k].reshape(shp))
        o += k
    return out


def mlp_forward(p, X):
    """Logits and activations: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(p)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3.T + b3
    return z, (X, a1, h1, a2, h2)


def mlp_loss_grad(p, X, labels):
    """Mean softmax cross-entropy and its gradient by the chain rule (backpropagation), packed like p."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(p)
    z, (X, a1, h1, a2, h2) = mlp_forward(p, X)
    labels = np.asarray(labels)
    N = X.shape[0]
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    P = e / e.sum(axis=1, keepdims=True)
    loss = float(np.mean(-np.log(P[np.arange(N), labels])))
    dz = P.copy()
    dz[np.arange(N), labels] -= 1.0
    dz /= N
    gW3 = dz.T @ h2
    gb3 = dz.sum(axis=0)
    dh2 = (dz @ W3) * (a2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
