"""Learned per-step power-iteration count for randUTV (the policy behind rrf_opts.q_policy = LEARNED).

Training data comes from the method itself: each training matrix A = Q1 diag(s) Q2^T (seeded Haar factors,
a random decay class) is factored with q = 0 (recording the 16 features of every step through the C ABI)
and with fixed q = 1, 2, 3; the criterion is the rank-k error e_k = ||T(k:, k:)||_2 at every block boundary
k (Sec. 4.1).  A q is acceptable at a boundary when its e_k meets the quality target 1.1 sigma_{k+1}, or
else comes within 5 % of the best of q = 2 (the fallback) and q = 3; the label is the cheapest acceptable
q.  The MLP is trained on the GPU with the library's FP16 forward/backward kernels and Adam; at run time
the step takes the smallest q whose cumulative softmax probability reaches 0.8.  Without parameters the
method falls back to q = 2.

    python -m paper_2106_13402_gb300.qpolicy --count 1000 --n 1024     # writes qpolicy_fp16.npy
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np

from . import rrf

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "qpolicy_fp16.npy")
FALLBACK_Q = 2
DECAY_CLASSES = ("exp", "poly", "sshape", "step")


def random_spectrum(n: int, rng: np.random.Generator) -> np.ndarray:
    """One of four decay classes with random rates (exponential, polynomial, S-shaped, step)."""
    j = np.arange(n, dtype=np.float64)
    cls = DECAY_CLASSES[rng.integers(len(DECAY_CLASSES))]
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


def make_matrix(n: int, seed: int, device: str = "cuda"):
    import torch
    rng = np.random.default_rng(seed)
    s = random_spectrum(n, rng)
    dev = torch.device(device)

    def haar(sd):
        g = torch.Generator(device=dev)
        g.manual_seed(sd)
        q, r = torch.linalg.qr(torch.randn(n, n, generator=g, device=dev, dtype=torch.float64))
        d = torch.sign(torch.diagonal(r))
        d[d == 0] = 1
        return q * d

    q1, q2 = haar(2 * seed + 1), haar(2 * seed + 2)
    A = (q1 * torch.as_tensor(s, device=dev)) @ q2.t()
    return rrf.as_fortran(A.t().contiguous().t()), s


def spectral_norm(torch, M, iters: int = 40) -> float:
    g = torch.Generator(device=M.device)
    g.manual_seed(7)
    x = torch.randn(M.shape[1], 1, generator=g, device=M.device, dtype=M.dtype)
    x /= torch.linalg.norm(x)
    s = 0.0
    for _ in range(iters):
        y = M.t() @ (M @ x)
        nrm = torch.linalg.norm(y)
        if float(nrm) == 0.0:
            return 0.0
        x = y / nrm
        s = nrm
    return float(math.sqrt(float(s)))


def acceptable(errs: np.ndarray, sig: np.ndarray, target: float = 1.1, slack: float = 1.05) -> np.ndarray:
    """errs: (4, k) e_k for q = 0..3; sig: (k,) sigma_{k+1}.  True where q meets target * sigma_{k+1} or
    comes within `slack` of min(e(q=2), e(q=3))."""
    ref = np.minimum(errs[2], errs[3])
    return errs <= np.maximum(target * sig, slack * ref)[None, :]


def label_matrix(A, s, b: int, seed: int):
    """Features of each step (q = 0 run), e_k for q = 0..3, and labels: the cheapest acceptable q."""
    import torch
    n = A.shape[1]
    steps = math.ceil(n / b)
    ws = rrf.workspace(rrf.randutv_workspace_bytes(n, n, b))
    opts = rrf.make_opts(q_policy=rrf.Q_LEARNED, steps=steps)
    _, T0, _ = rrf.randutv(A, b, 0, seed, opts=opts, ws=ws)
    feats = rrf.opts_features(opts)[: steps - 1]
    errs = np.zeros((4, steps - 1))
    for q in range(4):
        T = T0 if q == 0 else rrf.randutv(A, b, q, seed, ws=ws)[1]
        for i in range(1, steps):
            errs[q, i - 1] = spectral_norm(torch, T[i * b:, i * b:])
    sig = np.asarray(s)[b * np.arange(1, steps)]
    labels = np.argmax(acceptable(errs, sig), axis=0)
    return feats, labels, errs


def decide(logits: np.ndarray, confidence: float = 0.8) -> np.ndarray:
    """The run-time rule: smallest q whose cumulative softmax probability reaches `confidence`."""
    z = logits - logits.max(axis=1, keepdims=True)
    p = np.exp(z)
    p /= p.sum(axis=1, keepdims=True)
    return np.argmax(np.cumsum(p, axis=1) >= confidence, axis=1)


def generate(count: int, n: int, b: int, seed0: int = 1000, log=None):
    """Features, labels, e_k for q = 0..3 and sigma_{k+1} of every step of `count` seeded matrices."""
    X, y, E, S = [], [], [], []
    t0 = time.time()
    for t in range(count):
        A, sv = make_matrix(n, seed0 + t)
        f, lab, errs = label_matrix(A, sv, b, seed0 + t)
        X.append(f)
        y.append(lab)
        E.append(errs.T)
        S.append(np.asarray(sv)[b * np.arange(1, f.shape[0] + 1)])
        if log and (t + 1) % 25 == 0:
            log(f"  {t + 1}/{count} matrices labelled, {time.time() - t0:.0f} s")
    return (np.concatenate(X).astype(np.float32), np.concatenate(y).astype(np.int32), np.concatenate(E),
            np.concatenate(S))


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases, packed like the kernels expect."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((64, 16), (64, 64), (4, 64)):
        parts.append(rng.standard_normal((fan_out, fan_in)).ravel() * math.sqrt(2.0 / fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def train(X: np.ndarray, y: np.ndarray, epochs: int = 60, batch: int = 1024, lr: float = 3e-3, seed: int = 0,
          log=None):
    """Adam on mini-batches with the library's FP16 kernels; returns the FP16 parameters (CUDA tensor)."""
    import torch
    dev = torch.device("cuda")
    master = torch.from_numpy(init_params(seed)).to(dev)
    params = master.half()
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    Xd = torch.from_numpy(X).to(dev)
    yd = torch.from_numpy(y).to(dev)
    N = Xd.shape[0]
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(N, generator=g).to(dev)
        for s0 in range(0, N, batch):
            idx = perm[s0:s0 + batch]
            grad, loss = rrf.mlp_grad(params, Xd[idx], yd[idx])
            step += 1
            rrf.mlp_adam(master, m, v, grad, params, step, lr)
        if log and (ep + 1) % 10 == 0:
            _, loss = rrf.mlp_grad(params, Xd, yd)
            acc = float((rrf.mlp_forward(params, Xd).argmax(1) == yd).float().mean())
            log(f"  epoch {ep + 1}: loss {float(loss):.4f} accuracy {acc:.3f}")
    return params


def save(params, path: str = WEIGHTS):
    np.save(path, params.detach().cpu().numpy().astype(np.float16))


def load(device="cuda", path: str = WEIGHTS):
    """Packaged FP16 parameters as a CUDA tensor, or None (the method then falls back to q = 2)."""
    import torch
    if not os.path.exists(path):
        return None
    return torch.from_numpy(np.load(path).astype(np.float16)).to(device)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=1000)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--b", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=100)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--data-only", action="store_true")
    a = ap.parse_args()
    print(f"labelling {a.count} matrices of {a.n}^2 (b = {a.b})", flush=True)
    X, y, E, S = generate(a.count, a.n, a.b, log=lambda s: print(s, flush=True))
    print("label histogram q=0..3:", np.bincount(y, minlength=4).tolist(), flush=True)
    np.savez(os.path.splitext(a.out)[0] + "_data.npz", X=X, y=y, E=E, S=S)
    if a.data_only:
        return
    params = train(X, y, epochs=a.epochs, log=lambda s: print(s, flush=True))
    save(params, a.out)
    print("saved", a.out, flush=True)


if __name__ == "__main__":
    main()
