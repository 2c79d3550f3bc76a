"""Writes c2_oracle_ek_8192.txt: the FP64 oracle's rank-k errors on the 8192 x 8192 matrix of the default
bench configuration, generated on the CPU.

A = Q1 diag(s) Q2^T with s_j = 10^(-8j/n) for j < n/2, then 1e-4 (testmats.make_matrix(8192, 8192, "c2",
11, 12), numpy Haar factors); randUTV_basic (Algorithm 3) with b = 128, q = 1 and the Gaussian stream of
seed 17, run by the oracle.  For every block boundary k = 128, 256, ..., 8064 the file holds k, the
rank-k error e_k = ||T(k+1:n, k+1:n)||_2 (Sec. 4.1: with U and V orthogonal this is ||A - A_k||_2 for the
factorization's own rank-k approximation), sigma_{k+1} and their ratio.  The 2-norms are computed with
ARPACK (scipy.sparse.linalg.svds, relative tolerance 1e-12) on the oracle's T.

    python tests/golden/make_c2_oracle_ek.py        # about 10 minutes on 8 cores
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2106_13402_gb300 import testmats  # noqa: E402

N, B, Q, SEED = 8192, 128, 1, 17
OUT = os.path.join(HERE, "c2_oracle_ek_8192.txt")


def spectral_norm(M: np.ndarray) -> float:
    from scipy.sparse.linalg import svds
    return float(svds(M, k=1, tol=1e-12, return_singular_vectors=False, random_state=0)[0])


def main():
    t0 = time.time()
    A, s = testmats.make_matrix(N, N, "c2", 11, 12)
    print(f"matrix {time.time() - t0:.0f} s", flush=True)
    U, T, V, st = oracle.randutv(A, B, Q, SEED)
    assert st == 0, st
    print(f"oracle randUTV {time.time() - t0:.0f} s, {oracle.num_threads()} threads", flush=True)
    rows = []
    for k in range(B, N, B):
        ek = spectral_norm(np.ascontiguousarray(T[k:, k:]))
        rows.append((k, ek, s[k], ek / s[k]))
    res = np.linalg.norm(A - U @ T @ V.T) / np.linalg.norm(A)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle randUTV_basic (Algorithm 3), 8192^2 'c2' matrix (numpy Haar seeds 11, 12), b = 128,\n")
        f.write("# q = 1, Gaussian seed 17; written by tests/golden/make_c2_oracle_ek.py.\n")
        f.write(f"# residual ||A - U T V^T||_F / ||A||_F = {res:.3e}\n")
        f.write("# k  e_k  sigma_{k+1}  e_k/sigma_{k+1}\n")
        for k, ek, sk, r in rows:
            f.write(f"{k} {ek:.17e} {sk:.17e} {r:.12f}\n")
    print(f"wrote {OUT} ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main()
