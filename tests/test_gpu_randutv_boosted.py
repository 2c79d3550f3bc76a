"""GPU randUTV_boosted (Algorithm 2: opts.oversample = p > 0) through the C ABI against the FP64 oracle's
orc_randutv_boosted on the same inputs and Gaussian stream.

Tolerances are those of randUTV_basic (residual and orthogonality <= 1e-12, exact zeros below the diagonal
and off the diagonal of each b x b block, e_k within 1 % of the oracle's) and |diag T| within 1e-10
relative (+1e-11 ||A||_2) where the split of the b + p sample into its leading b directions is well
conditioned.  Where the spectrum has a flat stretch (the step profile, the S-shaped floor, the plateau of
the 8192^2 spectrum's shape) the sample's singular values there are close, its leading-b subspace moves
with rounding, and so do the diagonal entries of the blocks on either side of that split: the oracle itself,
run on A with every entry moved by one unit in the last place, changes them by up to ~1e-8 (S-shaped,
500 x 100, b = p = 32).  Each block's diagonal is therefore held to max(1e-10, 50 x that measured
sensitivity of the oracle) relative.
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
    res = np.linalg.norm(A - U @ T @ V.T) / max(np.linalg.norm(A), 1e-300)
    assert res <= tol, res
    assert np.abs(U.T @ U - np.eye(m)).max() <= tol
    assert np.abs(V.T @ V - np.eye(n)).max() <= tol
    assert np.all(np.tril(T, -1) == 0.0)
    for o in range(0, n, b):
        blk = T[o:o + b, o:o + b]
        assert np.all(blk * (1.0 - np.eye(*blk.shape)) == 0.0)


def ek(T, k):
    return np.linalg.norm(T[k:, k:], 2) if k < min(T.shape) else 0.0


def boosted(A, b, q, p, seed, gemm_mode=rrf.GEMM_AUTO):
    opts = rrf.make_opts(oversample=p, gemm_mode=gemm_mode)
    return tuple(host(x) for x in rrf.randutv(dev(A), b, q, seed=seed, opts=opts))


BOOSTED_CASES = [
    # m, n, b, q, p, profile, compare |diag T|
    (64, 64, 16, 1, 16, "gaussian", True),
    (200, 160, 32, 1, 32, "exp8", True),
    (300, 250, 64, 2, 64, "fast", True),        # ragged last block
    (257, 129, 32, 1, 16, "poly", True),        # tall, ragged
    (500, 100, 32, 2, 32, "sshape", True),      # tall: the last block goes through HQR first
    (96, 96, 16, 0, 16, "gaussian", True),      # q = 0
    (100, 90, 32, 1, 200, "exp8", True),        # p capped by c - b at every step
    (40, 40, 1, 1, 3, "gaussian", True),        # b = 1
    (130, 130, 13, 3, 7, "step", False),        # flat stretch
    (512, 512, 32, 2, 32, "c2", False),         # the 8192^2 spectrum's shape, plateau
]


def oracle_diag_sensitivity(A, b, q, p, seed, do, draws=2):
    """Per-block relative change of the oracle's |diag T| when every entry of A moves by one ulp."""
    n = A.shape[1]
    rng = np.random.default_rng(12345)
    sens = np.zeros(-(-n // b))
    for _ in range(draws):
        Ap = np.asfortranarray(A * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=A.shape)))
        _, Tp, _, st = oracle.randutv_boosted(Ap, b, q, p, seed)
        assert st == 0
        rel = np.abs(np.abs(np.diag(Tp)) - do) / np.maximum(do, 1e-300)
        for i, o in enumerate(range(0, n, b)):
            sens[i] = max(sens[i], rel[o:o + b].max())
    return sens


@pytest.mark.parametrize("m,n,b,q,p,prof,diag", BOOSTED_CASES)
def test_boosted_matches_oracle(m, n, b, q, p, prof, diag):
    A, s = testmats.make_matrix(m, n, prof, 3, 4)
    U, T, V = boosted(A, b, q, p, 99)
    check_factorization(A, U, T, V, b)
    Uo, To, Vo, st = oracle.randutv_boosted(A, b, q, p, 99)
    assert st == 0
    do, dg = np.abs(np.diag(To)), np.abs(np.diag(T))
    if diag:
        sens = oracle_diag_sensitivity(A, b, q, p, 99, do)
        for i, o in enumerate(range(0, n, b)):
            rtol = max(1e-10, 50.0 * sens[i])
            np.testing.assert_allclose(dg[o:o + b], do[o:o + b], rtol=rtol, atol=1e-11 * do[0],
                                       err_msg=f"block {i}, oracle sensitivity {sens[i]:.2e}")
    for k in range(b, n, b):
        eo, eg = ek(To, k), ek(T, k)
        assert abs(eg - eo) <= 1e-2 * eo + 1e-13 * do[0], (k, eg, eo)
    if s is not None:
        assert all(ek(T, k) >= s[k] * (1 - 1e-10) for k in range(b, n, b))   # Eckart-Young


def test_boosted_native_fp64_products_match_oracle():
    """The plain FP64 (DFMA-only) products give the same factorization."""
    A, s = testmats.make_matrix(300, 250, "fast", 3, 4)
    U, T, V = boosted(A, 64, 2, 64, 99, gemm_mode=rrf.GEMM_NATIVE)
    check_factorization(A, U, T, V, 64)
    Uo, To, Vo, st = oracle.randutv_boosted(A, 64, 2, 64, 99)
    np.testing.assert_allclose(np.abs(np.diag(T)), np.abs(np.diag(To)), rtol=1e-10, atol=1e-11 * To[0, 0])


def test_boosted_is_repeatable_bitwise():
    A, _ = testmats.make_matrix(300, 300, "poly", 1, 2)
    r1 = boosted(A, 32, 2, 32, 5)
    r2 = boosted(A, 32, 2, 32, 5)
    for x, y in zip(r1, r2):
        assert np.array_equal(x, y)


def test_boosted_exact_rank_input():
    """Exact rank 64 = 2 b: the trailing block after two steps is zero to rounding (Sec. 4.2)."""
    A, s = testmats.make_matrix(256, 192, "rank", 3, 4, rank=64)
    U, T, V = boosted(A, 32, 1, 32, 3)
    check_factorization(A, U, T, V, 32)
    assert ek(T, 64) <= 1e-13 * s[0]


@pytest.mark.slow
def test_boosted_1024_meets_boundary_target_like_oracle():
    """1024^2, s_j = exp(-j/100), b = 64, q = 2, p = b (emulated FP64 products for the large GEMMs): the GPU
    and the oracle agree on every e_k to 1 %, and both keep e_k <= 1.1 sigma_{k+1} at every boundary."""
    A, s = testmats.make_matrix(1024, 1024, "exp100", 1, 2)
    U, T, V = boosted(A, 64, 2, 64, 7)
    check_factorization(A, U, T, V, 64)
    Uo, To, Vo, st = oracle.randutv_boosted(A, 64, 2, 64, 7)
    np.testing.assert_allclose(np.abs(np.diag(T)), np.abs(np.diag(To)), rtol=1e-10, atol=1e-11 * s[0])
    for k in range(64, 1024, 64):
        rg, ro = ek(T, k) / s[k], ek(To, k) / s[k]
        assert abs(rg - ro) <= 1e-2 * ro
        assert ro <= 1.1 and rg <= 1.1, (k, rg, ro)
