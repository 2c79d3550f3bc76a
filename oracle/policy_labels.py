"""Quality labels for the learned power-iteration policy, computed by the oracle.

TEST INFRASTRUCTURE ONLY (run offline; the library never imports this): for each training matrix
testmats.policy_matrix(n, seed) the oracle factors A with randUTV_basic (Algorithm 3) for q = 0, 1, 2, 3
with the same Gaussian stream (seed) and records, at every block boundary k = b, 2b, ..., the rank-k error
e_k = ||T(k:, k:)||_2 (Sec. 4.1; the trailing block's spectral norm, by numpy's SVD) and sigma_{k+1}.  The
policy is then trained on the GPU with these e_k as the judge of each step's q.

    python -m oracle.policy_labels --count 1000 --n 1024 --b 128 --out oracle/policy_labels_1024.npz
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2106_13402_gb300 import testmats  # noqa: E402


def label_errors(A: np.ndarray, s: np.ndarray, b: int, seed: int, qmax: int = 3):
    """(E, S): E[i, q] = e_k at boundary k = (i + 1) b for q = 0 .. qmax; S[i] = sigma_{k+1}."""
    n = A.shape[1]
    steps = -(-n // b)
    E = np.zeros((steps - 1, qmax + 1))
    for q in range(qmax + 1):
        _, T, _, st = oracle.randutv(A, b, q, seed)
        if st != 0:
            raise RuntimeError(f"oracle status {st}")
        for i in range(1, steps):
            E[i - 1, q] = np.linalg.norm(T[i * b:, i * b:], 2)
    return E, np.asarray(s)[b * np.arange(1, steps)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=1000)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--b", type=int, default=128)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "policy_labels_1024.npz"))
    a = ap.parse_args()
    oracle.build()
    seeds, Es, Ss = [], [], []
    if os.path.exists(a.out):  # continue an interrupted run
        d = np.load(a.out)
        seeds, Es, Ss = list(d["seeds"]), list(d["E"]), list(d["S"])
    t0 = time.time()
    for t in range(len(seeds), a.count):
        seed = a.seed0 + t
        A, s = testmats.policy_matrix(a.n, seed)
        E, S = label_errors(A, s, a.b, seed)
        seeds.append(seed)
        Es.append(E)
        Ss.append(S)
        if (t + 1) % 10 == 0 or t + 1 == a.count:
            np.savez(a.out, seeds=np.array(seeds), E=np.array(Es), S=np.array(Ss), n=a.n, b=a.b)
            print(f"{t + 1}/{a.count} matrices, {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
