"""FP64 GEMM emulated on the BF16 tensor cores, and both factorizations running on it.

The emulation splits each row of op(A) / column of op(B) into 7 exact 8-bit digits below a power-of-two
scale (remainder < 2^-55 of the row / column maximum), accumulates the digit products exactly (FP32 on the
tensor cores per 32-wide K chunk, then int64) and drops only the digit products of diagonals 7..12 (at most
2^-51.4 of the row / column scale per k).  Against an extended-precision reference (numpy longdouble) each
entry is held to 2^-51 (|alpha op(A) op(B)| + |beta C|)_ij for the final FP64 roundings plus the worst case
2^-50 K max_k|a_ik| max_k|b_kj| of the dropped digits; a second check holds the typical error (random
digits, about 2^-55 sqrt(K) of the scale) to 2^-51 sqrt(K) max|a_i.| max|b_.j|, which an accumulation that
rounds at 2^-48 per chunk fails.  The factorizations keep every FP64 tolerance of the native path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2106_13402_gb300 import rrf, testmats

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")


def dev(x):
    return rrf.as_fortran(torch.from_numpy(np.asfortranarray(x)).cuda())


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("m,n,k,graded", [(128, 64, 32, False), (300, 100, 1000, False), (513, 200, 77, True),
                                          (64, 300, 500, False), (600, 256, 2048, True),
                                          (1024, 640, 96, False), (256, 64, 8192, False)])
def test_emulated_gemm_accuracy(ta, tb, m, n, k, graded):
    rng = np.random.default_rng(m + 3 * n + 7 * k)
    A = rng.standard_normal((k, m) if ta == "T" else (m, k))
    B = rng.standard_normal((n, k) if tb == "T" else (k, n))
    if graded:  # wide dynamic range inside rows and columns
        A = A * 10.0 ** rng.uniform(-6, 0, A.shape)
        B = B * 10.0 ** rng.uniform(-6, 0, B.shape)
    C0 = rng.standard_normal((m, n))
    opA, opB = (A.T if ta == "T" else A), (B.T if tb == "T" else B)
    C = rrf.gemm(ta, tb, dev(A), dev(B), alpha=-0.75, beta=0.5, C=dev(C0), emulated=True).cpu().numpy()
    L = np.longdouble
    ref = (-0.75 * (opA.astype(L) @ opB.astype(L)) + 0.5 * C0.astype(L)).astype(np.float64)
    absA, absB = np.abs(opA), np.abs(opB)
    scale = np.outer(absA.max(axis=1), absB.max(axis=0))
    prod = np.abs((opA.astype(L) @ opB.astype(L)).astype(np.float64))
    rnd = 2.0 ** -51 * (0.75 * prod + 0.5 * np.abs(C0))
    err = np.abs(C - ref)
    bound = rnd + 0.75 * 2.0 ** -50 * k * scale + 1e-300
    assert np.all(err <= bound), float((err / bound).max())
    typical = rnd + 0.75 * 2.0 ** -51 * np.sqrt(k) * scale + 1e-300
    assert np.all(err <= typical), float((err / typical).max())


@pytest.mark.parametrize("m,n,b,q,prof", [(512, 384, 64, 1, "poly"), (300, 250, 64, 2, "fast"),
                                          (700, 300, 64, 1, "sshape")])
def test_randutv_on_emulated_gemm(m, n, b, q, prof):
    A, s = testmats.make_matrix(m, n, prof, 3, 4)
    opts = rrf.make_opts(gemm_mode=rrf.GEMM_EMULATED)
    U, T, V = (x.cpu().numpy() for x in rrf.randutv(dev(A), b, q, seed=99, opts=opts))
    res = np.linalg.norm(A - U @ T @ V.T) / np.linalg.norm(A)
    assert res <= 1e-12
    assert np.abs(U.T @ U - np.eye(m)).max() <= 1e-12
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
    assert np.all(np.tril(T, -1) == 0.0)
    Uo, To, Vo, st = oracle.randutv(A, b, q, seed=99)
    do, dg = np.abs(np.diag(To)), np.abs(np.diag(T))
    np.testing.assert_allclose(dg, do, rtol=1e-10, atol=1e-11 * do[0])


@pytest.mark.parametrize("m,n,b,q", [(512, 384, 64, 1), (400, 400, 128, 0)])
def test_powerurv_on_emulated_gemm(m, n, b, q):
    A, s = testmats.make_matrix(m, n, "gaussian", 8, 9)
    opts = rrf.make_opts(gemm_mode=rrf.GEMM_EMULATED)
    U, T, V = (x.cpu().numpy() for x in rrf.powerurv(dev(A), b, q, seed=21, opts=opts))
    assert np.linalg.norm(A - U @ T @ V.T) / np.linalg.norm(A) <= 1e-12
    assert np.abs(U.T @ U - np.eye(m)).max() <= 1e-12
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
    assert np.all(np.tril(T, -1) == 0.0)
    Uo, Ro, Vo, st = oracle.powerurv(A, q, seed=21)
    np.testing.assert_allclose(T, Ro, atol=1e-10 * np.abs(Ro).max())


@pytest.mark.slow
def test_randutv_1024_emulated_matches_oracle():
    A, s = testmats.make_matrix(1024, 1024, "exp100", 1, 2)
    opts = rrf.make_opts(gemm_mode=rrf.GEMM_EMULATED)
    U, T, V = (x.cpu().numpy() for x in rrf.randutv(dev(A), 64, 1, seed=7, opts=opts))
    assert np.linalg.norm(A - U @ T @ V.T) / np.linalg.norm(A) <= 1e-12
    assert np.abs(U.T @ U - np.eye(1024)).max() <= 1e-12
    Uo, To, Vo, st = oracle.randutv(A, 64, 1, seed=7)
    np.testing.assert_allclose(np.diag(T), np.diag(To), rtol=1e-10)
