"""Seeded synthetic test matrices A = Q1 diag(s) Q2^T (Sec. 6.2's construction) and Gaussian inputs.

This module holds none of the factorization's arithmetic: it only draws seeded inputs that both the
CUDA path and the CPU oracle consume.  Q1 (m x n, orthonormal) and Q2 (n x n, orthogonal) are Haar
distributed: the Q factor of a seeded standard Gaussian matrix with its columns signed by
sign(diag R) (Mezzadri 2007).  The paper's "fast decay" matrices use the same construction without
the sign fix (Sec. 6.2); the sign fix only makes the distribution exactly Haar.

Small inputs are drawn on the CPU with numpy's PCG64 stream; large inputs (``device="cuda"``) are
drawn with torch's CUDA generator and factored by the library QR there.  Either way the matrix is
produced once, off any timed region, and handed unchanged to both sides.
"""
from __future__ import annotations

import math

import numpy as np

PROFILES = ("exp100", "c2", "poly", "fast", "sshape", "step", "exp8", "gaussian", "rank")


def singular_values(n: int, profile: str, rank: int | None = None) -> np.ndarray:
    """Prescribed singular values s_0 >= s_1 >= ... (index base 0, s_0 = 1).

    exp100 : s_j = exp(-j/100)                           (1024^2 configuration)
    c2     : s_j = 10^(-8j/n) for j < n/2, then 1e-4       (8192^2 configurations)
    poly   : s_j = 1/(1+j)                                (16384^2 BF16-sketch configuration)
    fast   : s_j = beta^(j/(n-1)), beta = 1e-5            (Sec. 6.2 "fast decay")
    sshape : s_j = 1e-2 + (1 - 1e-2)/(1 + exp((j - n/4)/(n/50)))   (Sec. 6.2 "S-shaped", our reading)
    step   : s_j = 1 for j < n/4, else 1e-3
    exp8   : s_j = exp(-8j/n)
    rank   : s_j = 1/(1+j) for j < rank, else exactly 0
    """
    j = np.arange(n, dtype=np.float64)
    if profile == "exp100":
        s = np.exp(-j / 100.0)
    elif profile == "c2":
        s = np.where(j < n / 2, 10.0 ** (-8.0 * j / n), 1e-4)
    elif profile == "poly":
        s = 1.0 / (1.0 + j)
    elif profile == "fast":
        s = (1e-5) ** (j / max(n - 1, 1))
    elif profile == "sshape":
        s = 1e-2 + (1.0 - 1e-2) / (1.0 + np.exp((j - n / 4.0) / (n / 50.0)))
    elif profile == "step":
        s = np.where(j < n / 4, 1.0, 1e-3)
    elif profile == "exp8":
        s = np.exp(-8.0 * j / n)
    elif profile == "rank":
        if rank is None:
            raise ValueError("profile 'rank' needs rank=")
        s = np.where(j < rank, 1.0 / (1.0 + j), 0.0)
    else:
        raise ValueError(f"unknown profile {profile!r}")
    return s


def _haar_np(rows: int, cols: int, seed: int) -> np.ndarray:
    g = np.random.default_rng(seed).standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def make_matrix(m: int, n: int, profile: str, seed1: int, seed2: int, rank: int | None = None,
                device: str = "cpu"):
    """Return (A, s): A = Q1 diag(s) Q2^T (m x n, m >= n), or a standard Gaussian A (s = None).

    device="cpu" returns a Fortran-ordered numpy float64 array.  device="cuda" returns a torch
    float64 CUDA tensor of shape (m, n) in column-major storage (stride (1, m)).
    """
    if m < n:
        raise ValueError("m >= n required")
    if device == "cpu":
        if profile == "gaussian":
            A = np.random.default_rng(seed1).standard_normal((m, n))
            return np.asfortranarray(A), None
        s = singular_values(n, profile, rank)
        q1 = _haar_np(m, n, seed1)
        q2 = _haar_np(n, n, seed2)
        A = (q1 * s) @ q2.T
        return np.asfortranarray(A), s
    import torch

    dev = torch.device(device)

    def haar_t(rows, cols, seed):
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed)
        g = torch.randn(cols, rows, generator=gen, device=dev, dtype=torch.float64).t()
        q, r = torch.linalg.qr(g)
        d = torch.sign(torch.diagonal(r))
        d[d == 0] = 1.0
        return q * d

    if profile == "gaussian":
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed1)
        A = torch.randn(n, m, generator=gen, device=dev, dtype=torch.float64).t()
        return A, None
    s = singular_values(n, profile, rank)
    st = torch.as_tensor(s, device=dev)
    q1 = haar_t(m, n, seed1)
    q2 = haar_t(n, n, seed2)
    A = (q1 * st) @ q2.t()
    A = A.t().contiguous().t()  # column-major storage
    del q1, q2
    return A, s


POLICY_DECAY_CLASSES = ("exp", "poly", "sshape", "step")


def policy_spectrum(n: int, rng: np.random.Generator) -> np.ndarray:
    """Training and held-out spectra of the learned q policy: one of four decay classes with random rates
    (exponential, polynomial, S-shaped, step), drawn from `rng`."""
    j = np.arange(n, dtype=np.float64)
    cls = POLICY_DECAY_CLASSES[rng.integers(len(POLICY_DECAY_CLASSES))]
    if cls == "exp":
        s = np.exp(-rng.uniform(2.0, 40.0) * j / n)
    elif cls == "poly":
        s = (1.0 + j) ** (-rng.uniform(0.3, 3.0))
    elif cls == "sshape":
        c, w, lo = rng.uniform(0.05, 0.7) * n, rng.uniform(0.005, 0.1) * n, 10.0 ** rng.uniform(-5, -1)
        s = lo + (1.0 - lo) / (1.0 + np.exp((j - c) / w))
    else:
        k, lo = int(rng.uniform(0.05, 0.8) * n), 10.0 ** rng.uniform(-6, -1)
        s = np.where(j < k, 1.0, lo)
    return np.sort(s)[::-1].copy()


def policy_matrix(n: int, seed: int):
    """(A, s): an n x n training matrix of the learned q policy, A = Q1 diag(s) Q2^T with s from
    policy_spectrum(numpy PCG64(seed)) and Haar Q1, Q2 from numpy seeds 2 seed + 1, 2 seed + 2
    (Fortran-ordered float64; the same on every machine)."""
    rng = np.random.default_rng(seed)
    s = policy_spectrum(n, rng)
    q1 = _haar_np(n, n, 2 * seed + 1)
    q2 = _haar_np(n, n, 2 * seed + 2)
    return np.asfortranarray((q1 * s) @ q2.T), s


def batch_shapes(count: int, seed: int, m_lo: int = 256, m_hi: int = 2048, n_lo: int = 128):
    """Uneven batch shapes: m ~ U[m_lo, m_hi], n ~ U[n_lo, m] (uniform integers), seeded."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=count)
    ns = np.array([rng.integers(n_lo, int(mm) + 1) for mm in ms])
    return [(int(a), int(b)) for a, b in zip(ms, ns)]


def flops_randutv(m: int, n: int, b: int, q: int, max_steps: int = 0) -> float:
    """Algorithmic flop count of randUTV_basic (Algorithm 3), FP64-equivalent.

    Per step i < s (r = m - b(i-1), c = n - b(i-1)): sketch (2+4q) r c b, HQR of Y 2cb^2,
    V-application 4mcb + 4ncb, panel HQR 2rb^2, U-application 4mrb + 4r(c-b)b, small updates
    2mb^2 + 2nb^2 + 2b^2(c-b) + 2(i-1)b^3; final block 2rc^2 + 4mrc + 2nc^2 + 2(i-1)bc^2.
    max_steps > 0 counts only the first max_steps steps (a partial factorization).
    """
    steps = min(math.ceil(m / b), math.ceil(n / b))
    if max_steps > 0:
        steps = min(steps, max_steps)
    f = 0.0
    for i in range(1, steps + 1):
        o = b * (i - 1)
        r, c = m - o, n - o
        if b * i < m and b * i < n:
            f += (2 + 4 * q) * r * c * b + 2 * c * b * b + 4 * m * c * b + 4 * n * c * b + 2 * r * b * b
            f += 4 * m * r * b + 4 * r * (c - b) * b
            f += 2 * m * b * b + 2 * n * b * b + 2 * b * b * (c - b) + 2 * o * b * b
        else:
            f += 2 * r * c * c + 4 * m * r * c + 2 * n * c * c + 2 * o * c * c
    return float(f)


def flops_powerurv(m: int, n: int, q: int) -> float:
    """Algorithmic flop count of powerURV (Algorithm 1): GEMMs 2mn^2 per product, HQR of an r x c
    matrix 2rc^2 - 2c^3/3, the same again for forming its thin Q (r x c), and
    4 m^2 n - 4 m n^2 + 4n^3/3 for forming the full m x m U from n reflectors."""
    def hqr(r, c):
        return 2.0 * r * c * c - 2.0 * c ** 3 / 3.0
    f = 0.0
    if q == 0:
        f += 2 * hqr(n, n)
    for _ in range(q):
        f += 2.0 * m * n * n + 2 * hqr(m, n)   # Yh = A V, HQR_thin(Yh) + form Q
        f += 2.0 * m * n * n + 2 * hqr(n, n)   # Y = A^T Vh, HQR_thin(Y) + form Q
    f += 2.0 * m * n * n                       # Ah = A V
    f += hqr(m, n) + 4.0 * m * m * n - 4.0 * m * n * n + 4.0 * n ** 3 / 3.0
    return float(f)
