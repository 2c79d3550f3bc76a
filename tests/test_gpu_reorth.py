"""GPU randUTV with the re-orthonormalized power iteration (Sec. 2.5 (ii); opts.reorth = 1) against the
oracle's orc_randutv_reorth, and the BF16 sketch (which always re-orthonormalizes) at b = 256.

FP64 tolerances are those of randUTV_basic: residual and orthogonality <= 1e-12, exact zeros, e_k within
1 % of the oracle's, and each block's |diag T| within max(1e-10, 50 x the oracle's own change when A moves
by one ulp) relative (+1e-11 ||A||_2): where a block boundary falls on a flat stretch of the spectrum the
split of the sample is ill conditioned and rounding alone moves those entries.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2106_13402_gb300 import rrf, testmats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    rrf.lib()


def dev(x):
    return rrf.as_fortran(torch.from_numpy(np.asfortranarray(x)).cuda())


def host(x):
    torch.cuda.synchronize()
    return x.cpu().numpy()


def check_factorization(A, U, T, V, b, tol=1e-12):
    m, n = A.shape
    assert np.linalg.norm(A - U @ T @ V.T) <= tol * np.linalg.norm(A)
    assert np.abs(U.T @ U - np.eye(m)).max() <= tol
    assert np.abs(V.T @ V - np.eye(n)).max() <= tol
    assert np.all(np.tril(T, -1) == 0.0)
    for o in range(0, n, b):
        blk = T[o:o + b, o:o + b]
        assert np.all(blk * (1.0 - np.eye(*blk.shape)) == 0.0)


def ek(T, k):
    return np.linalg.norm(T[k:, k:], 2) if k < min(T.shape) else 0.0


def oracle_sensitivity(A, b, q, seed, do, draws=2):
    n = A.shape[1]
    rng = np.random.default_rng(54321)
    sens = np.zeros(-(-n // b))
    for _ in range(draws):
        Ap = np.asfortranarray(A * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=A.shape)))
        _, Tp, _, st = oracle.randutv_reorth(Ap, b, q, seed)
        rel = np.abs(np.abs(np.diag(Tp)) - do) / np.maximum(do, 1e-300)
        for i, o in enumerate(range(0, n, b)):
            sens[i] = max(sens[i], rel[o:o + b].max())
    return sens


REORTH_CASES = [
    (200, 160, 32, 1, "exp8"),
    (300, 250, 64, 2, "fast"),     # ragged last block
    (257, 129, 64, 1, "poly"),     # tall, ragged
    (500, 100, 32, 2, "sshape"),   # tall final block through HQR; flat floor
    (130, 130, 13, 3, "step"),     # flat stretches
    (64, 64, 16, 0, "gaussian"),   # q = 0: nothing to orthonormalize
]


@pytest.mark.parametrize("m,n,b,q,prof", REORTH_CASES)
def test_reorth_matches_oracle(m, n, b, q, prof):
    A, s = testmats.make_matrix(m, n, prof, 3, 4)
    opts = rrf.make_opts(reorth=True)
    U, T, V = (host(x) for x in rrf.randutv(dev(A), b, q, seed=99, opts=opts))
    check_factorization(A, U, T, V, b)
    Uo, To, Vo, st = oracle.randutv_reorth(A, b, q, 99)
    assert st == 0
    do, dg = np.abs(np.diag(To)), np.abs(np.diag(T))
    sens = oracle_sensitivity(A, b, q, 99, do)
    for i, o in enumerate(range(0, n, b)):
        np.testing.assert_allclose(dg[o:o + b], do[o:o + b], rtol=max(1e-10, 50.0 * sens[i]), atol=1e-11 * do[0],
                                   err_msg=f"block {i}, oracle sensitivity {sens[i]:.2e}")
    for k in range(b, n, b):
        eo, eg = ek(To, k), ek(T, k)
        assert abs(eg - eo) <= 1e-2 * eo + 1e-13 * do[0], (k, eg, eo)


def test_reorth_entrywise_on_well_separated_spectrum():
    A, s = testmats.make_matrix(192, 160, "fast", 5, 6)
    opts = rrf.make_opts(reorth=True)
    U, T, V = (host(x) for x in rrf.randutv(dev(A), 32, 2, seed=5, opts=opts))
    Uo, To, Vo, st = oracle.randutv_reorth(A, 32, 2, 5)
    np.testing.assert_allclose(T, To, atol=1e-10 * np.abs(To).max())
    np.testing.assert_allclose(V[:, :32], Vo[:, :32], atol=1e-9)


def test_reorth_keeps_the_small_directions_of_a_wide_block():
    """The oracle pin's input (a first block spanning 10^8.4, then a flat tail): the GPU's re-orthonormalized
    sketch reaches e_b within 1 % of sigma_{b+1}, like the oracle's, where the plain sketch does not."""
    n, b = 96, 8
    rng = np.random.default_rng(0)
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    j = np.arange(n)
    sv = np.where(j < b, 10.0 ** (-1.2 * j), 10.0 ** (-1.2 * (b - 1)) * 0.5 * np.exp(-(j - b) / 200.0))
    A = np.asfortranarray((Q1 * sv) @ Q2.T)
    U, T, V = (host(x) for x in rrf.randutv(dev(A), b, 2, seed=7, opts=rrf.make_opts(reorth=True)))
    check_factorization(A, U, T, V, b)
    assert ek(T, b) / sv[b] <= 1.01
    _, Tp, _ = (host(x) for x in rrf.randutv(dev(A), b, 2, seed=7))
    assert ek(Tp, b) / sv[b] >= 5.0


@pytest.mark.slow
def test_bf16_sketch_b256_against_fp64_oracle():
    """The precision form at the BF16 configuration's block size and spectrum, reduced to 2048^2:
    s_j = 1/(1+j), b = 256, q = 2, BF16 sketch (FP32 accumulate), FP64 everything else.  Exact
    factorization in FP64; at every block boundary e_k within 5 % of the FP64 re-orthonormalized
    oracle's (same Gaussian), and e_k >= sigma_{k+1} (Eckart-Young)."""
    n, b, q = 2048, 256, 2
    A, s = testmats.make_matrix(n, n, "poly", 21, 22)
    opts = rrf.make_opts(rrf.SKETCH_BF16)
    U, T, V = (host(x) for x in rrf.randutv(dev(A), b, q, seed=17, opts=opts))
    check_factorization(A, U, T, V, b)
    Uo, To, Vo, st = oracle.randutv_reorth(A, b, q, 17)
    assert st == 0
    for k in range(b, n, b):
        eg, eo = ek(T, k), ek(To, k)
        assert eg >= s[k] * (1 - 1e-10)
        assert eg <= eo * 1.05, (k, eg / s[k], eo / s[k])
