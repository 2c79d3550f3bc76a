"""GPU parity: every kernel and both factorizations, called through the C ABI, against the FP64 oracle.

Tolerances (FP64 throughout):
  - Gaussian stream: the Philox words are bit-exact; the Box-Muller normals use CUDA's and libm's
    log/cos/sin, each within a few ulp, so |z_gpu - z_cpu| <= 1e-14 max(1, |z|).
  - GEMM: |C - C_ref| <= 2 K eps (|A||B|)_ij, the standard bound for any summation order.
  - Householder panel: R, tau, Y, Tf agree with the oracle to 1e-12 relative (same reflector rule).
  - Factorizations: ||A - U T V^T||_F / ||A||_F <= 1e-12, ||U^T U - I||, ||V^T V - I|| <= 1e-12,
    entries below the diagonal (and off-diagonal entries of the b x b diagonal blocks) exactly 0,
    |diag T| within 1e-10 relative of the oracle, e_k / sigma_{k+1} within 1% of the oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2106_13402_gb300 import rrf, testmats

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


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


# ------------------------------------------------------------------------------------------ randn --
@pytest.mark.parametrize("rows,cols,step,tag", [(1, 1, 0, 2), (37, 5, 3, 1), (1000, 129, 1, 1), (256, 256, 0, 2)])
def test_randn_matches_oracle(rows, cols, step, tag):
    seed = 0x1234_5678_9ABC
    g = host(rrf.randn(rows, cols, seed, step, tag))
    o = oracle.randn(rows, cols, seed, step, tag)
    assert np.all(np.abs(g - o) <= 1e-14 * np.maximum(1.0, np.abs(o)))
    # the integer stream is exact: signs and magnitudes agree to the last few ulp everywhere
    assert np.array_equal(np.sign(g), np.sign(o))


# ------------------------------------------------------------------------------------------- GEMM --
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (70, 33, 130), (130, 64, 5000), (513, 200, 17), (64, 64, 0)])
def test_gemm_matches_bound(ta, tb, m, n, k):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((k, m) if ta == "T" else (m, k))
    B = rng.standard_normal((n, k) if tb == "T" else (k, n))
    C0 = rng.standard_normal((m, n))
    opA, opB = (A.T if ta == "T" else A), (B.T if tb == "T" else B)
    C = host(rrf.gemm(ta, tb, dev(A), dev(B), alpha=-0.75, beta=0.5, C=dev(C0)))
    ref = -0.75 * (opA @ opB) + 0.5 * C0
    bound = 2 * max(k, 1) * EPS * (0.75 * np.abs(opA) @ np.abs(opB) + 0.5 * np.abs(C0)) + 1e-300
    assert np.all(np.abs(C - ref) <= bound)


def test_gemm_beta_zero_ignores_nan_in_c():
    A = np.ones((8, 4))
    B = np.ones((4, 8))
    C0 = np.full((8, 8), np.nan)
    C = host(rrf.gemm("N", "N", dev(A), dev(B), beta=0.0, C=dev(C0)))
    assert np.all(C == 4.0)


# ---------------------------------------------------------------------------------- Householder --
@pytest.mark.parametrize("r,w", [(1, 1), (5, 5), (100, 7), (777, 64), (3000, 128), (4100, 256)])
def test_panel_qr_matches_oracle(r, w):
    rng = np.random.default_rng(r + w)
    P = rng.standard_normal((r, w))
    Pg, tau, Y, Tf = rrf.panel_qr(dev(P))
    Pg, tau, Y, Tf = host(Pg), host(tau), host(Y), host(Tf)
    F, tau_o = oracle.hqr(P)
    np.testing.assert_allclose(np.triu(Pg[:w]), np.triu(F[:w]), rtol=0, atol=1e-12 * np.abs(F).max())
    np.testing.assert_allclose(tau, tau_o, rtol=1e-12, atol=1e-14)
    Yo = np.tril(F, -1)[:, :w] + np.eye(r, w)
    np.testing.assert_allclose(Y, Yo, rtol=0, atol=1e-11)
    np.testing.assert_allclose(np.tril(Pg, -1), np.tril(F, -1), rtol=0, atol=1e-11)
    np.testing.assert_allclose(Tf, oracle.larft(Yo, tau_o), rtol=0, atol=1e-11)
    assert np.all(np.tril(Tf, -1) == 0.0)


def test_panel_qr_zero_column_and_rank_deficient():
    rng = np.random.default_rng(9)
    P = rng.standard_normal((300, 3)) @ rng.standard_normal((3, 12))
    P[:, 0] = 0.0
    P[0, 0] = -2.0          # x(1:) == 0 and alpha < 0: identity reflector
    Pg, tau, Y, Tf = rrf.panel_qr(dev(P))
    tau = host(tau)
    F, tau_o = oracle.hqr(P)
    assert tau[0] == 0.0 and tau_o[0] == 0.0
    R = np.triu(host(Pg)[:12])
    Ro = np.triu(F[:12])
    np.testing.assert_allclose(R[:4, :], Ro[:4, :], atol=1e-11)
    assert np.abs(R[4:, 4:]).max() < 1e-12 * np.abs(R).max()   # rank 4 revealed (Sec. 2.4)


# --------------------------------------------------------------------------------------- Jacobi --
@pytest.mark.parametrize("c,kind", [(1, "gaussian"), (2, "gaussian"), (7, "gaussian"), (64, "upper"), (128, "upper"),
                                    (200, "gaussian"), (256, "graded")])
def test_jacobi_matches_oracle(c, kind):
    rng = np.random.default_rng(c)
    M = rng.standard_normal((c, c))
    if kind == "upper":
        M = np.triu(M)
    if kind == "graded":
        M = np.triu(M) * np.logspace(0, -6, c)
    Us, s, Vs, st = rrf.jacobi_svd(dev(M))
    Us, s, Vs = host(Us), host(s), host(Vs)
    assert st == 0
    Uo, so, Vo, sto, _ = oracle.jacobi_svd(M)
    np.testing.assert_allclose(s, so, rtol=1e-12, atol=1e-14 * so[0])
    np.testing.assert_allclose(Us @ np.diag(s) @ Vs.T, M, atol=1e-13 * np.abs(M).max())
    np.testing.assert_allclose(Vs.T @ Vs, np.eye(c), atol=1e-13)
    np.testing.assert_allclose(Us.T @ Us, np.eye(c), atol=1e-13)
    # same sign convention -> singular vectors agree where the spectrum is well separated
    gap = np.min(np.abs(np.diff(so))) / so[0] if c > 1 else 1.0
    if gap > 1e-6:
        np.testing.assert_allclose(Vs, Vo, atol=1e-13 / gap)


@pytest.mark.parametrize("c", [32, 64, 128, 200])
@pytest.mark.parametrize("spread", [1e-6, 1e-9, 1e-12])
def test_jacobi_clustered_core_is_orthogonal(c, spread):
    # A core close to a multiple of an orthogonal matrix (a flat stretch of the spectrum): its columns
    # are nearly orthogonal from the start, but alpha ~ beta makes every rotation large, so a stop on
    # |gamma| alone leaves u_k = m_k / sigma_k non-orthogonal at the level of gamma (Hestenes' rule
    # with tolerance c 2^-53 does not).
    rng = np.random.default_rng(c + int(-np.log10(spread)))
    Q1, _ = np.linalg.qr(rng.standard_normal((c, c)))
    Q2, _ = np.linalg.qr(rng.standard_normal((c, c)))
    s_true = 1e-2 * (1.0 + spread * np.arange(c))[::-1]
    M = (Q1 * s_true) @ Q2.T
    Us, s, Vs, st = rrf.jacobi_svd(dev(M))
    Us, s, Vs = host(Us), host(s), host(Vs)
    assert st == 0
    np.testing.assert_allclose(s, s_true, rtol=1e-13)
    np.testing.assert_allclose(Us @ np.diag(s) @ Vs.T, M, atol=1e-13 * np.abs(M).max())
    assert np.abs(Us.T @ Us - np.eye(c)).max() <= 1e-13
    assert np.abs(Vs.T @ Vs - np.eye(c)).max() <= 1e-13


def test_jacobi_zero_and_diagonal_inputs():
    Us, s, Vs, st = rrf.jacobi_svd(dev(np.zeros((16, 16))))
    Us, s = host(Us), host(s)
    assert np.all(s == 0.0)
    np.testing.assert_allclose(Us.T @ Us, np.eye(16), atol=1e-15)
    D = np.diag(np.arange(1.0, 33.0)[::-1] * np.where(np.arange(32) % 2, -1, 1))
    Us, s, Vs, st = rrf.jacobi_svd(dev(D))
    np.testing.assert_array_equal(host(s), np.arange(32.0, 0.0, -1.0))


# ------------------------------------------------------------------------------- factorizations --
def check_factorization(A, U, T, V, b=None, tol=1e-12):
    m, n = A.shape
    res = np.linalg.norm(A - U @ T @ V.T) / max(np.linalg.norm(A), 1e-300)
    assert res <= tol, res
    assert np.abs(U.T @ U - np.eye(m)).max() <= tol
    assert np.abs(V.T @ V - np.eye(n)).max() <= tol
    assert np.all(np.tril(T, -1) == 0.0)
    if b is not None:
        for o in range(0, n, b):
            blk = T[o:o + b, o:o + b]
            assert np.all(blk * (1.0 - np.eye(*blk.shape)) == 0.0)


def ek(T, k):
    return np.linalg.norm(T[k:, k:], 2) if k < min(T.shape) else 0.0


RANDUTV_CASES = [
    (64, 64, 16, 0, "gaussian"),
    (200, 160, 32, 1, "exp8"),
    (300, 250, 64, 2, "fast"),     # ragged last block
    (257, 129, 64, 1, "poly"),     # tall, ragged
    (500, 100, 32, 1, "sshape"),   # tall final block goes through HQR first
    (90, 70, 128, 1, "gaussian"),     # b >= n: single SVD
    (40, 40, 1, 0, "gaussian"),       # b = 1
    (130, 130, 13, 3, "step"),
]


@pytest.mark.parametrize("m,n,b,q,prof", RANDUTV_CASES)
def test_randutv_matches_oracle(m, n, b, q, prof):
    A, s = testmats.make_matrix(m, n, prof, 3, 4)
    U, T, V = (host(x) for x in rrf.randutv(dev(A), b, q, seed=99))
    check_factorization(A, U, T, V, b)
    Uo, To, Vo, st = oracle.randutv(A, b, q, seed=99)
    do, dg = np.abs(np.diag(To)), np.abs(np.diag(T))
    # Singular values are perfectly conditioned (Weyl): |d sigma_k| <= ||dT||, so the absolute part of
    # the bound is relative to ||A||; the sketch's conditioning (sigma ratios within a block raised to
    # 2q+1) amplifies rounding differences in the sampled subspace up to ~1e-11 ||A||.
    np.testing.assert_allclose(dg, do, rtol=1e-10, atol=1e-11 * do[0])
    for k in range(b, n, b):
        eo, eg = ek(To, k), ek(T, k)
        assert abs(eg - eo) <= 1e-2 * eo + 1e-13 * do[0]


def test_randutv_entrywise_on_well_separated_spectrum():
    """With distinct, well separated singular values and the shared sign convention, T, U, V agree
    with the oracle entry by entry, not only in sign-invariant quantities."""
    A, s = testmats.make_matrix(192, 160, "fast", 5, 6)
    U, T, V = (host(x) for x in rrf.randutv(dev(A), 32, 2, seed=5))
    Uo, To, Vo, st = oracle.randutv(A, 32, 2, seed=5)
    np.testing.assert_allclose(T, To, atol=1e-10 * np.abs(To).max())
    np.testing.assert_allclose(V[:, :32], Vo[:, :32], atol=1e-9)


@pytest.mark.parametrize("m,n,b,q", [(64, 64, 16, 0), (200, 160, 32, 1), (300, 250, 64, 2), (257, 129, 128, 1)])
def test_powerurv_matches_oracle(m, n, b, q):
    A, s = testmats.make_matrix(m, n, "gaussian", 8, 9)
    U, T, V = (host(x) for x in rrf.powerurv(dev(A), b, q, seed=21))
    check_factorization(A, U, T, V)
    Uo, Ro, Vo, st = oracle.powerurv(A, q, seed=21)
    # Householder QR with the shared sign rule is unique: U, R, V agree entrywise.
    np.testing.assert_allclose(np.abs(np.diag(T)), np.abs(np.diag(Ro)), rtol=1e-10)
    np.testing.assert_allclose(T, Ro, atol=1e-10 * np.abs(Ro).max())
    np.testing.assert_allclose(V, Vo, atol=1e-10)
    np.testing.assert_allclose(U[:, :n], Uo[:, :n], atol=1e-10)


def test_host_buffer_entry_points_match_device():
    A, _ = testmats.make_matrix(150, 120, "exp8", 1, 2)
    Ud, Td, Vd = (host(x) for x in rrf.randutv(dev(A), 32, 1, seed=3))
    Uh, Th, Vh = rrf.randutv_host(A, 32, 1, seed=3)
    np.testing.assert_array_equal(Td, Th)
    np.testing.assert_array_equal(Ud, Uh)
    Ud, Td, Vd = (host(x) for x in rrf.powerurv(dev(A), 32, 1, seed=3))
    Uh, Th, Vh = rrf.powerurv_host(A, 32, 1, seed=3)
    np.testing.assert_array_equal(Td, Th)


def test_repeatable_bitwise():
    A, _ = testmats.make_matrix(300, 300, "poly", 1, 2)
    T1 = host(rrf.randutv(dev(A), 64, 1, seed=4)[1])
    T2 = host(rrf.randutv(dev(A), 64, 1, seed=4)[1])
    np.testing.assert_array_equal(T1, T2)


def test_non_finite_input_reports_numerical():
    A = np.random.default_rng(0).standard_normal((64, 48))
    A[5, 7] = np.nan
    with pytest.raises(rrf.RrfError) as ei:
        rrf.randutv(dev(A), 16, 1, seed=1)
    assert ei.value.status == rrf.RRF_NUMERICAL


def test_zero_and_rank_deficient_inputs():
    Z = np.zeros((96, 80))
    U, T, V = (host(x) for x in rrf.randutv(dev(Z), 16, 1, seed=2))
    assert np.all(T == 0.0)
    np.testing.assert_allclose(U.T @ U, np.eye(96), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(80), atol=1e-12)
    A, s = testmats.make_matrix(128, 96, "rank", 3, 4, rank=32)
    U, T, V = (host(x) for x in rrf.randutv(dev(A), 16, 1, seed=2))
    check_factorization(A, U, T, V, 16)
    assert ek(T, 32) <= 1e-13 * s[0]


@pytest.mark.slow
def test_randutv_1024_matches_oracle_and_tracks_sigma():
    """1024^2, s_j = exp(-j/100), b = 64, q = 1 (the small configuration), full parity."""
    A, s = testmats.make_matrix(1024, 1024, "exp100", 1, 2)
    U, T, V = (host(x) for x in rrf.randutv(dev(A), 64, 1, seed=7))
    check_factorization(A, U, T, V, 64)
    Uo, To, Vo, st = oracle.randutv(A, 64, 1, seed=7)
    np.testing.assert_allclose(np.diag(T), np.diag(To), rtol=1e-10)
    for k in range(64, 1024, 64):
        rg, ro = ek(T, k) / s[k], ek(To, k) / s[k]
        assert rg >= 1 - 1e-10
        assert abs(rg - ro) <= 1e-2 * ro


@pytest.mark.slow
def test_powerurv_1024_matches_oracle():
    A, s = testmats.make_matrix(1024, 1024, "exp100", 1, 2)
    U, T, V = (host(x) for x in rrf.powerurv(dev(A), 64, 1, seed=7))
    check_factorization(A, U, T, V)
    Uo, Ro, Vo, st = oracle.powerurv(A, 1, seed=7)
    np.testing.assert_allclose(np.abs(np.diag(T)), np.abs(np.diag(Ro)), rtol=1e-8)
