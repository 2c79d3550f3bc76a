"""Learned per-step power-iteration count for randUTV (the policy behind rrf_opts.q_policy = LEARNED).

Training data: each training matrix A = Q1 diag(s) Q2^T (testmats.policy_matrix: seeded Haar factors, a
random decay class) is factored on the GPU with q = 0, recording the 16 features of every step through the
C ABI.  The judge of each step's q is the FP64 oracle: for the same matrix and Gaussian stream it factors A
with q = 0, 1, 2, 3 and records the rank-k error e_k = ||T(k:, k:)||_2 at every block boundary k (Sec. 4.1);
those e_k ship with the package (qpolicy_labels_1024.npz, written by the oracle's label script).  A q is
acceptable at a boundary when its e_k meets the quality target 1.1 sigma_{k+1} wherever q = 2 (the
fallback) or q = 3 meets it, and otherwise when it comes within 5 % of the better of those two; the label
is the cheapest acceptable q.  The MLP is trained on
the GPU with the library's FP16 forward/backward kernels and Adam; at run time the step takes the smallest
q whose cumulative softmax probability reaches 0.8.  Without parameters the method falls back to q = 2.

    python -m paper_2106_13402_gb300.qpolicy            # features on the GPU, writes qpolicy_fp16.npy
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
LABELS = os.path.join(HERE, "qpolicy_labels_1024.npz")


def make_matrix(n: int, seed: int, device: str = "cuda"):
    """testmats.policy_matrix(n, seed) on the device (column-major), with its spectrum."""
    import torch
    from . import testmats
    A, s = testmats.policy_matrix(n, seed)
    return rrf.as_fortran(torch.from_numpy(A).to(device)), s


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
    """errs: (4, k) e_k for q = 0..3; sig: (k,) sigma_{k+1}.  Where q = 2 or q = 3 meets the quality target
    target * sigma_{k+1}, a q is acceptable only if it meets it too; where neither does, a q is acceptable
    if it comes within `slack` of min(e(q=2), e(q=3))."""
    ref = np.minimum(errs[2], errs[3])
    bound = np.where(ref <= target * sig, target * sig, slack * ref)
    return errs <= bound[None, :]


def step_features(A, b: int, seed: int) -> np.ndarray:
    """The 16 features of every step of the q = 0 factorization (the policy's run-time inputs), from the GPU."""
    n = A.shape[1]
    steps = math.ceil(n / b)
    ws = rrf.workspace(rrf.randutv_workspace_bytes(n, n, b))
    opts = rrf.make_opts(q_policy=rrf.Q_LEARNED, steps=steps)
    rrf.randutv(A, b, 0, seed, opts=opts, ws=ws)
    return rrf.opts_features(opts)[: steps - 1]


def labels_from_errors(E: np.ndarray, S: np.ndarray) -> np.ndarray:
    """E: (boundaries, 4) e_k for q = 0..3 (the oracle's), S: sigma_{k+1}; the cheapest acceptable q."""
    return np.argmax(acceptable(E.T, S), axis=0)


def decide(logits: np.ndarray, confidence: float = 0.8) -> np.ndarray:
    """The run-time rule: smallest q whose cumulative softmax probability reaches `confidence`."""
    z = logits - logits.max(axis=1, keepdims=True)
    p = np.exp(z)
    p /= p.sum(axis=1, keepdims=True)
    return np.argmax(np.cumsum(p, axis=1) >= confidence, axis=1)


def generate(labels_path: str = LABELS, count: int = 0, log=None):
    """Features (GPU, q = 0 run) and labels (the oracle's e_k) of the labelled training matrices."""
    d = np.load(labels_path)
    seeds, E, S = d["seeds"], d["E"], d["S"]
    n, b = int(d["n"]), int(d["b"])
    if count > 0:
        seeds, E, S = seeds[:count], E[:count], S[:count]
    X, y = [], []
    t0 = time.time()
    for t, seed in enumerate(seeds):
        A, sv = make_matrix(n, int(seed))
        X.append(step_features(A, b, int(seed)))
        y.append(labels_from_errors(E[t], S[t]))
        if log and (t + 1) % 100 == 0:
            log(f"  {t + 1}/{len(seeds)} matrices, {time.time() - t0:.0f} s")
    return np.concatenate(X).astype(np.float32), np.concatenate(y).astype(np.int32)


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
    ap.add_argument("--labels", default=LABELS)
    ap.add_argument("--count", type=int, default=0, help="use the first COUNT labelled matrices (0: all)")
    ap.add_argument("--epochs", type=int, default=100)
    ap.add_argument("--out", default=WEIGHTS)
    a = ap.parse_args()
    X, y = generate(a.labels, a.count, log=lambda s: print(s, flush=True))
    print(f"{X.shape[0]} labelled steps; label histogram q=0..3:", np.bincount(y, minlength=4).tolist(), flush=True)
    params = train(X, y, epochs=a.epochs, log=lambda s: print(s, flush=True))
    save(params, a.out)
    print("saved", a.out, flush=True)


if __name__ == "__main__":
    main()
