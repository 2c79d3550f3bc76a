"""Pins for the FP64 CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test checks the oracle against something other than itself: published known-answer vectors,
an independent library implementation, closed forms, invariants stated in the paper, or brute
force on tiny inputs.  A plausible slip in the oracle (dropped term, wrong sign or index,
transposed operand) breaks at least one of them.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle
from paper_2106_13402_gb300 import testmats

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


# ---------------------------------------------------------------- Philox-4x32-10 (G stream) --
@pytest.mark.parametrize("ctr,key,expected", _kat_rows())
def test_philox_known_answers(ctr, key, expected):
    assert oracle.philox4x32_10(ctr, key) == expected


def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/x86_64-linux/lib",
                  "/usr/local/cuda/targets/sbsa-linux/lib", ""):
            p = os.path.join(d, name) if d else name
            try:
                return ctypes.CDLL(p)
            except OSError:
                continue
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host Philox4_32_10 generator with seed 0 emits block t = Philox(ctr=(0,0,t,0), key=0)."""
    L = _curand()
    if L is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    st = L.curandCreateGeneratorHost(ctypes.byref(gen), ctypes.c_int(161))  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    if st != 0:
        pytest.skip(f"curandCreateGeneratorHost failed ({st})")
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(0)) == 0
        n = 64
        buf = (ctypes.c_uint32 * n)()
        assert L.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
        for t in range(n // 4):
            assert oracle.philox4x32_10([0, 0, t, 0], [0, 0]) == list(buf[4 * t: 4 * t + 4])
    finally:
        L.curandDestroyGenerator(gen)


def test_randn_layout_and_blocks():
    """Element (i, j) of randn(rows, cols) is flat element i + j*rows of the stream; blocks pair up."""
    flat = oracle.randn(1, 2 * 21, seed=5, step=3, tag=1)[0]
    G = oracle.randn(6, 7, seed=5, step=3, tag=1)
    np.testing.assert_array_equal(G.flatten(order="F"), flat)
    odd = oracle.randn(5, 3, seed=5, step=3, tag=1)      # 15 elements: last block half used
    np.testing.assert_array_equal(odd.flatten(order="F"), flat[:15])
    # different step / tag / seed give different streams
    assert not np.array_equal(oracle.randn(6, 7, seed=5, step=4, tag=1), G)
    assert not np.array_equal(oracle.randn(6, 7, seed=5, step=3, tag=2), G)
    assert not np.array_equal(oracle.randn(6, 7, seed=6, step=3, tag=1), G)


def test_randn_is_standard_normal():
    from scipy import stats
    z = oracle.randn(400, 500, seed=123, step=1, tag=1).ravel()
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert abs(stats.skew(z)) < 0.02
    assert abs(stats.kurtosis(z)) < 0.04
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the two normals of one block are independent: correlation of even/odd elements ~ 0
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 0.01


# ------------------------------------------------------------------------------- GEMM --
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_gemm_matches_numpy(ta, tb):
    rng = np.random.default_rng(1)
    m, n, k = 13, 9, 17
    A = rng.standard_normal((k, m) if ta == "T" else (m, k))
    B = rng.standard_normal((n, k) if tb == "T" else (k, n))
    C0 = rng.standard_normal((m, n))
    opA = A.T if ta == "T" else A
    opB = B.T if tb == "T" else B
    C = oracle.gemm(ta, tb, A, B, alpha=0.5, beta=-2.0, C=C0)
    np.testing.assert_allclose(C, 0.5 * opA @ opB - 2.0 * C0, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------------------ Householder QR --
def test_hqr_reconstructs_and_matches_lapack_diag():
    rng = np.random.default_rng(2)
    m, n = 40, 17
    A = rng.standard_normal((m, n))
    F, tau = oracle.hqr(A)
    R = np.triu(F[:n, :])
    Q = oracle.form_q(F, tau, m)
    np.testing.assert_allclose(Q.T @ Q, np.eye(m), atol=1e-14)
    np.testing.assert_allclose(Q[:, :n] @ R, A, atol=1e-13)
    # LAPACK (dgeqrf) uses the same reflector convention: R agrees entrywise, not only |diag R|.
    r_np = np.linalg.qr(A, mode="r")
    np.testing.assert_allclose(R, r_np, atol=1e-13)
    # tau in [1, 2] for nontrivial reflectors of this convention
    assert np.all((tau >= 1.0) & (tau <= 2.0))


def test_hqr_detects_rank():
    """Sec. 2.4: rank-k input with independent first k columns gives R(k:, k:) = 0 (exact arithmetic)."""
    rng = np.random.default_rng(3)
    m, n, k = 50, 20, 7
    A = rng.standard_normal((m, k)) @ rng.standard_normal((k, n))
    F, tau = oracle.hqr(A)
    R = np.triu(F[:n, :])
    assert np.abs(R[k:, k:]).max() < 1e-13 * np.abs(R).max()
    assert np.abs(np.diag(R)[:k]).min() > 1e-3


def test_hqr_identity_reflector_for_zero_subcolumn():
    A = np.array([[-3.0, 1.0], [0.0, 2.0], [0.0, 5.0]])
    F, tau = oracle.hqr(A)
    assert tau[0] == 0.0 and F[0, 0] == -3.0
    R = np.triu(F[:2])
    Q = oracle.form_q(F, tau, 3)
    np.testing.assert_allclose(Q[:, :2] @ R, A, atol=1e-14)


def test_larft_compact_wy_equals_product_of_reflectors():
    """Sec. 2.4: H_0 ... H_{k-1} = I - Y T Y^T with T upper triangular."""
    rng = np.random.default_rng(4)
    m, k = 30, 9
    F, tau = oracle.hqr(rng.standard_normal((m, k)))
    Y = np.tril(F, -1)[:, :k] + np.eye(m, k)
    Tf = oracle.larft(Y, tau)
    assert np.allclose(Tf, np.triu(Tf))
    prod = np.eye(m)
    for j in range(k):
        v = Y[:, j]
        prod = prod @ (np.eye(m) - tau[j] * np.outer(v, v))
    np.testing.assert_allclose(np.eye(m) - Y @ Tf @ Y.T, prod, atol=1e-14)
    np.testing.assert_allclose(oracle.form_q(F, tau, m), prod, atol=1e-14)


@pytest.mark.parametrize("side,trans", [("L", "N"), ("L", "T"), ("R", "N"), ("R", "T")])
def test_apply_q_all_sides(side, trans):
    rng = np.random.default_rng(5)
    m, k = 23, 6
    F, tau = oracle.hqr(rng.standard_normal((m, k)))
    Y = np.tril(F, -1)[:, :k] + np.eye(m, k)
    Q = np.eye(m)
    for j in range(k):
        Q = Q @ (np.eye(m) - tau[j] * np.outer(Y[:, j], Y[:, j]))
    opQ = Q.T if trans == "T" else Q
    C = rng.standard_normal((m, 11)) if side == "L" else rng.standard_normal((11, m))
    out = oracle.apply_q(side, trans, F, tau, C)
    ref = opQ @ C if side == "L" else C @ opQ
    np.testing.assert_allclose(out, ref, atol=1e-13)


# --------------------------------------------------------------------- one-sided Jacobi --
def _check_svd(M, U, s, V, tol=1e-13):
    r, c = M.shape
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, M, atol=tol * max(1.0, np.abs(M).max()))
    np.testing.assert_allclose(V.T @ V, np.eye(c), atol=tol)
    np.testing.assert_allclose(U.T @ U, np.eye(c), atol=tol)
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)


def test_jacobi_matches_numpy_svd():
    rng = np.random.default_rng(6)
    M = rng.standard_normal((24, 24))
    U, s, V, st, sw = oracle.jacobi_svd(M)
    assert st == 0 and 2 <= sw <= 15
    _check_svd(M, U, s, V)
    np.testing.assert_allclose(s, np.linalg.svd(M, compute_uv=False), rtol=1e-13)
    # sign convention: largest-magnitude entry of every v_k is positive
    for k in range(24):
        assert V[np.argmax(np.abs(V[:, k])), k] > 0


def test_jacobi_upper_triangular_tall_and_graded():
    rng = np.random.default_rng(7)
    R = np.triu(rng.standard_normal((16, 16))) * np.logspace(0, -9, 16)
    U, s, V, st, _ = oracle.jacobi_svd(R)
    assert st == 0
    _check_svd(R, U, s, V)
    # one-sided Jacobi is relatively accurate on column-graded input
    np.testing.assert_allclose(s, np.linalg.svd(R, compute_uv=False), rtol=1e-11)
    T = rng.standard_normal((30, 12))
    U, s, V, st, _ = oracle.jacobi_svd(T)
    _check_svd(T, U, s, V)


def test_jacobi_closed_forms():
    D = np.diag([0.5, -3.0, 2.0, 0.0])
    U, s, V, st, sw = oracle.jacobi_svd(D)
    assert st == 0 and sw == 1
    np.testing.assert_array_equal(s, [3.0, 2.0, 0.5, 0.0])
    _check_svd(D, U, s, V)
    u = np.array([1.0, 2.0, 2.0])
    v = np.array([3.0, 0.0, 4.0])
    U, s, V, st, _ = oracle.jacobi_svd(np.outer(u, v))
    np.testing.assert_allclose(s, [15.0, 0.0, 0.0], atol=1e-14)
    np.testing.assert_allclose(np.abs(V[:, 0]), np.abs(v) / 5.0, atol=1e-14)
    # 2x2: [[1, 1], [0, 1]] has singular values golden ratio phi and 1/phi
    phi = (1 + 5 ** 0.5) / 2
    _, s, _, _, _ = oracle.jacobi_svd(np.array([[1.0, 1.0], [0.0, 1.0]]))
    np.testing.assert_allclose(s, [phi, 1 / phi], rtol=1e-15)


def test_jacobi_zero_matrix_completes_u():
    U, s, V, st, _ = oracle.jacobi_svd(np.zeros((5, 5)))
    assert st == 0
    np.testing.assert_array_equal(s, np.zeros(5))
    np.testing.assert_allclose(U.T @ U, np.eye(5), atol=1e-15)


# ------------------------------------------------------------------------------- randUTV --
def ek_spectral(T, k):
    """e_k = ||T(k:, k:)||_2 (Eq. for the rank-k error in Sec. 4.1)."""
    if k >= min(T.shape):
        return 0.0
    return np.linalg.norm(T[k:, k:], 2)


def check_utv(A, U, T, V, b, tol=1e-12):
    m, n = A.shape
    nrmA = np.linalg.norm(A)
    assert np.linalg.norm(A - U @ T @ V.T) <= tol * nrmA
    np.testing.assert_allclose(U.T @ U, np.eye(m), atol=tol)
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=tol)
    assert np.all(np.tril(T, -1) == 0.0), "T must be exactly upper trapezoidal"
    for o in range(0, n, b):
        blk = T[o:o + b, o:o + b]
        off = blk * (1.0 - np.eye(*blk.shape))
        assert np.all(off == 0.0), "diagonal b x b blocks must be diagonal"
        assert np.all(np.diag(blk) >= 0) and np.all(np.diff(np.diag(blk)) <= 0)


@pytest.mark.parametrize("m,n,b,q", [(8, 8, 3, 0), (8, 8, 3, 1), (8, 6, 2, 2), (7, 7, 7, 1), (6, 5, 8, 0)])
def test_randutv_tiny_brute_force(m, n, b, q):
    """Every e_k is at least the optimal sigma_{k+1} (Eckart-Young, Sec. 2.2) and T reveals it."""
    rng = np.random.default_rng(100 + m + n + b + q)
    A = rng.standard_normal((m, n))
    U, T, V, st = oracle.randutv(A, b, q, seed=11)
    assert st == 0
    check_utv(A, U, T, V, b)
    sv = np.linalg.svd(A, compute_uv=False)
    for k in range(1, n):
        e = ek_spectral(T, k)
        e_direct = np.linalg.norm(A - U[:, :k] @ T[:k, :] @ V.T, 2)   # Eq. (1) definition
        assert abs(e - e_direct) <= 1e-12 * sv[0]
        assert e >= sv[k] * (1 - 1e-12)


def test_randutv_single_block_is_svd():
    """b >= n: the first step takes the else-branch, T = diag(singular values)."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((12, 9))
    U, T, V, st = oracle.randutv(A, 16, 1, seed=3)
    check_utv(A, U, T, V, 16)
    np.testing.assert_allclose(np.diag(T), np.linalg.svd(A, compute_uv=False), rtol=1e-13)


def test_randutv_step1_equals_randomized_range():
    """Step 1: U(:, :b) spans (A A^T)^(q+1) G (Sec. 4.1), so e_b = ||(I - Q Q^T) A||_2 with
    Q = orth((A A^T)^(q+1) G), G the step-1 Gaussian -- an independent route through numpy."""
    A, s = testmats.make_matrix(60, 50, "exp100", 1, 2)
    A = A * np.exp(-np.arange(50) / 8.0)  # steeper decay so the comparison is well conditioned
    b, q, seed = 8, 1, 21
    U, T, V, st = oracle.randutv(A, b, q, seed)
    G = oracle.randn(60, b, seed, 1, 1)
    W = G.copy()
    for _ in range(q + 1):
        W = A @ (A.T @ W)
    Q, _ = np.linalg.qr(W)
    e_route = np.linalg.norm(A - Q @ (Q.T @ A), 2)
    assert abs(ek_spectral(T, b) - e_route) <= 1e-10 * e_route
    # and the projectors agree
    np.testing.assert_allclose(U[:, :b] @ U[:, :b].T, Q @ Q.T, atol=1e-9)


def test_randutv_exact_rank():
    """Rank-r input with r a multiple of b: e_r ~ 0 (Theorems in the appendix: sketches keep rank)."""
    A, _ = testmats.make_matrix(48, 40, "rank", 5, 6, rank=16)
    U, T, V, st = oracle.randutv(A, 8, 1, seed=9)
    check_utv(A, U, T, V, 8)
    assert ek_spectral(T, 16) <= 1e-13 * np.linalg.norm(A, 2)
    assert ek_spectral(T, 15) > 1e-3 * np.linalg.norm(A, 2)


def test_randutv_frobenius_recurrence():
    """Sec. 4.1: e_0 = ||A||_F, e_i^2 = e_{i-1}^2 - ||T(I2, J2 u J3)||_F^2 equals ||T22||_F^2."""
    A, _ = testmats.make_matrix(40, 33, "fast", 3, 4)
    b = 6
    U, T, V, st = oracle.randutv(A, b, 2, seed=5)
    e2 = np.linalg.norm(A) ** 2
    for i in range(1, (33 + b - 1) // b):
        o = b * (i - 1)
        e2 -= np.linalg.norm(T[o:o + b, o:]) ** 2
        direct = np.linalg.norm(T[b * i:, b * i:]) ** 2
        assert abs(e2 - direct) <= 1e-12 * np.linalg.norm(A) ** 2


def test_randutv_partial_steps_keep_factorization():
    A, _ = testmats.make_matrix(30, 30, "poly", 7, 8)
    U, T, V, st = oracle.randutv(A, 5, 1, seed=1, max_steps=2)
    assert np.linalg.norm(A - U @ T @ V.T) <= 1e-13 * np.linalg.norm(A)
    assert np.all(np.tril(T[:, :10], -1) == 0)


def test_randutv_ragged_and_tall_final_block():
    A, _ = testmats.make_matrix(70, 29, "exp8", 1, 2)
    U, T, V, st = oracle.randutv(A, 8, 1, seed=2)
    check_utv(A, U, T, V, 8)
    sv = np.linalg.svd(A, compute_uv=False)
    for k in (8, 16, 24):
        assert ek_spectral(T, k) >= sv[k] * (1 - 1e-12)


@pytest.mark.slow
def test_randutv_tracks_sigma_1024():
    """1024^2, s_j = exp(-j/100), b = 64: residual, orthogonality, sparsity, and e_k/sigma_{k+1} at the
    block boundaries.  Without oversampling the ratio degrades at multiples of b (Sec. 6.2, third
    observation), and power iteration drives it toward 1 (Sec. 2.5, Corollary 10.10 bound)."""
    A, s = testmats.make_matrix(1024, 1024, "exp100", 1, 2)
    worst = []
    for q in (0, 1, 2):
        U, T, V, st = oracle.randutv(A, 64, q, seed=7)
        assert st == 0
        check_utv(A, U, T, V, 64)
        ratios = [ek_spectral(T, k) / s[k] for k in range(64, 1024, 64)]
        assert min(ratios) >= 1 - 1e-10
        mid = [ek_spectral(T, k) / s[k] for k in range(32, 1024, 64)]
        assert max(mid) < max(ratios)          # boundaries are the worst points
        worst.append(max(ratios))
    assert worst[0] > worst[1] > worst[2]
    assert worst[1] < 1.3 and worst[2] < 1.2, worst


# ------------------------------------------------------------------------------ powerURV --
@pytest.mark.parametrize("q", [0, 1, 2])
def test_powerurv_factorization(q):
    A, s = testmats.make_matrix(40, 30, "fast", 11, 12)
    U, R, V, st = oracle.powerurv(A, q, seed=13)
    assert st == 0
    assert np.linalg.norm(A - U @ R @ V.T) <= 1e-13 * np.linalg.norm(A)
    np.testing.assert_allclose(U.T @ U, np.eye(40), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(30), atol=1e-13)
    assert np.all(np.tril(R, -1) == 0.0)


def test_powerurv_q0_is_rurv():
    """q = 0: V is the Q factor of HQR_full(G) (Sec. 3.1); LAPACK's Householder QR gives the same Q."""
    A, _ = testmats.make_matrix(20, 15, "poly", 1, 2)
    U, R, V, st = oracle.powerurv(A, 0, seed=4)
    G = oracle.randn(15, 15, 4, 0, 2)
    Qn, _ = np.linalg.qr(G)
    np.testing.assert_allclose(V, Qn, atol=1e-13)


@pytest.mark.parametrize("q", [1, 2])
def test_powerurv_theorem1_projectors(q):
    """Theorem 1: U(:, :l) U(:, :l)^T A = Q_l Q_l^T A, Q_l = orth((A A^T)^q A G(:, :l)), every l."""
    A, _ = testmats.make_matrix(36, 24, "exp8", 3, 4)
    seed = 17
    U, R, V, st = oracle.powerurv(A, q, seed)
    G = oracle.randn(24, 24, seed, 0, 2)
    for ell in (1, 3, 8, 16):
        W = A @ G[:, :ell]
        for _ in range(q):
            W = A @ (A.T @ W)
        Q, _ = np.linalg.qr(W)
        P1 = U[:, :ell] @ (U[:, :ell].T @ A)
        P2 = Q @ (Q.T @ A)
        # The numpy route forms (A A^T)^q A G without re-orthonormalization, so its own rounding
        # error grows like eps * cond(W) (Sec. 3.2); the tolerance follows that bound.
        tol = max(1e-13, 100 * np.finfo(float).eps * np.linalg.cond(W))
        np.testing.assert_allclose(P1, P2, atol=tol * np.linalg.norm(A, 2))


# ------------------------------------------------------------------------- policy MLP (FP64) --
def _mlp_params(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(5508) * scale


def test_mlp_gradient_matches_finite_differences():
    """Backpropagation pinned by central differences of the loss (independent of the chain rule)."""
    rng = np.random.default_rng(1)
    p = _mlp_params(1)
    X = rng.standard_normal((7, 16))
    y = rng.integers(0, 4, 7)
    loss, g = oracle.mlp_loss_grad(p, X, y)
    idx = rng.choice(5508, 60, replace=False)
    idx = np.concatenate([idx, [5504, 5507, 1024, 1087]])  # include biases
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(pp, X, y)[0] - oracle.mlp_loss_grad(pm, X, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_mlp_zero_network_closed_form():
    """All-zero parameters: logits 0, loss log 4, only the output bias gets gradient mean(1/4 - onehot)."""
    X = np.random.default_rng(2).standard_normal((8, 16))
    y = np.array([0, 1, 2, 3, 0, 0, 1, 3])
    loss, g = oracle.mlp_loss_grad(np.zeros(5508), X, y)
    assert abs(loss - np.log(4.0)) < 1e-15
    expect = np.array([0.25 - np.mean(y == k) for k in range(4)])
    np.testing.assert_allclose(g[-4:], expect, atol=1e-15)
    assert np.all(g[:-4] == 0.0)


# ----------------------------------------------------------------------- randUTV_boosted --
@pytest.mark.parametrize("m,n,b,q,p", [(96, 96, 16, 0, 16), (96, 96, 16, 1, 8), (100, 90, 16, 2, 16),
                                       (70, 70, 16, 1, 40), (64, 50, 8, 2, 0)])
def test_boosted_factorization_is_exact(m, n, b, q, p):
    """Alg. 2 keeps A = U T V^T with U, V orthogonal and the block-diagonal structure of T, for ragged
    sizes, tall inputs, p from 0 to more than the trailing width."""
    A, _ = testmats.make_matrix(m, n, "exp8", 3, 4)
    U, T, V, st = oracle.randutv_boosted(A, b, q, p, seed=13)
    assert st == 0
    check_utv(A, U, T, V, b)


@pytest.mark.parametrize("m,n,b,q,p", [(8, 8, 3, 1, 2), (8, 6, 2, 2, 2), (7, 7, 2, 1, 5)])
def test_boosted_tiny_brute_force(m, n, b, q, p):
    """Every e_k is at least sigma_{k+1} (Eckart-Young) and equals the Eq. (1) error of the rank-k part."""
    rng = np.random.default_rng(300 + m + n + b + q + p)
    A = rng.standard_normal((m, n))
    U, T, V, st = oracle.randutv_boosted(A, b, q, p, seed=17)
    assert st == 0
    check_utv(A, U, T, V, b)
    sv = np.linalg.svd(A, compute_uv=False)
    for k in range(1, n):
        e = ek_spectral(T, k)
        assert abs(e - np.linalg.norm(A - U[:, :k] @ T[:k, :] @ V.T, 2)) <= 1e-12 * sv[0]
        assert e >= sv[k] * (1 - 1e-12)


def test_boosted_step1_equals_oversampled_range():
    """Step 1 (Sec. 4.2 method b): V(:, :b) spans the top b left singular vectors W_b of
    Y = (A^T A)^q A^T G with b + p columns, and U(:, :b) spans A W_b, so e_b = ||(I - Q Q^T) A||_2 with
    Q = orth(A W_b) -- an independent route through numpy from the same Gaussian G."""
    A, s = testmats.make_matrix(80, 64, "exp100", 1, 2)
    A = A * np.exp(-np.arange(64) / 10.0)
    b, q, p, seed = 8, 1, 8, 23
    U, T, V, st = oracle.randutv_boosted(A, b, q, p, seed, max_steps=1)
    G = oracle.randn(80, b + p, seed, 1, 1)
    Y = A.T @ G
    for _ in range(q):
        Y = A.T @ (A @ Y)
    Wy = np.linalg.svd(Y, full_matrices=False)[0][:, :b]
    Q, _ = np.linalg.qr(A @ Wy)
    e_route = np.linalg.norm(A - Q @ (Q.T @ A), 2)
    assert abs(ek_spectral(T, b) - e_route) <= 1e-10 * e_route
    np.testing.assert_allclose(V[:, :b] @ V[:, :b].T, Wy @ Wy.T, atol=1e-9)


def test_boosted_without_oversampling_matches_basic_first_step():
    """p = 0: step 1 samples the same subspace as randUTV_basic (same Gaussian), so the first block's
    singular values and the trailing block's spectrum agree to rounding."""
    A, _ = testmats.make_matrix(128, 128, "exp100", 1, 2)
    _, Tb, _, _ = oracle.randutv(A, 16, 1, 7, max_steps=1)
    _, T0, _, _ = oracle.randutv_boosted(A, 16, 1, 0, 7, max_steps=1)
    np.testing.assert_allclose(np.diag(T0)[:16], np.diag(Tb)[:16], rtol=1e-12)
    np.testing.assert_allclose(np.linalg.svd(T0[16:, 16:], compute_uv=False),
                               np.linalg.svd(Tb[16:, 16:], compute_uv=False), rtol=1e-10, atol=1e-14)


def test_boosted_exact_rank():
    A, _ = testmats.make_matrix(48, 40, "rank", 5, 6, rank=16)
    U, T, V, st = oracle.randutv_boosted(A, 8, 1, 8, seed=9)
    check_utv(A, U, T, V, 8)
    assert ek_spectral(T, 16) <= 1e-13 * np.linalg.norm(A, 2)
    assert ek_spectral(T, 15) > 1e-3 * np.linalg.norm(A, 2)


def test_boosted_partial_steps_keep_factorization():
    A, _ = testmats.make_matrix(96, 96, "poly", 3, 4)
    U, T, V, st = oracle.randutv_boosted(A, 16, 1, 16, seed=5, max_steps=2)
    assert np.linalg.norm(A - U @ T @ V.T) <= 1e-12 * np.linalg.norm(A)
    assert np.all(T[32:, :32] == 0.0)


def test_boosted_reaches_boundary_target_where_basic_does_not():
    """Sec. 6.2: oversampling removes the error spikes at block boundaries.  On the exp(-j/100) input
    (512^2, b = 32, q = 2) randUTV_basic stays above 1.1 sigma_{k+1} at boundaries while Alg. 2 with
    p = b is within it at every one (measured 1.169 vs 1.063)."""
    A, s = testmats.make_matrix(512, 512, "exp100", 1, 2)
    b = 32
    _, Tb, _, _ = oracle.randutv(A, b, 2, 7)
    _, To, _, _ = oracle.randutv_boosted(A, b, 2, b, 7)
    rb = [ek_spectral(Tb, k) / s[k] for k in range(b, 512, b)]
    ro = [ek_spectral(To, k) / s[k] for k in range(b, 512, b)]
    assert max(rb) > 1.1
    assert max(ro) <= 1.1
    assert np.mean(ro) < np.mean(rb)


# ------------------------------------------------------------------ re-orthonormalized power iteration --
def test_reorth_q0_is_randutv_basic():
    """With q = 0 there is nothing to re-orthonormalize: the same factorization bit for bit."""
    A, _ = testmats.make_matrix(120, 100, "exp8", 1, 2)
    r0 = oracle.randutv(A, 16, 0, 5)
    r1 = oracle.randutv_reorth(A, 16, 0, 5)
    for x, y in zip(r0[:3], r1[:3]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("q", [1, 2])
def test_reorth_step1_equals_randomized_range(q):
    """In exact arithmetic the orthonormalizations only change the basis of the sample, not its span, so
    step 1 still gives U(:, :b) spanning (A A^T)^(q+1) G (Sec. 2.5 (ii) against Sec. 4.1): the numpy route
    of the plain test, and the plain oracle's first block, both agree with it."""
    A, s = testmats.make_matrix(60, 50, "exp100", 1, 2)
    A = A * np.exp(-np.arange(50) / 8.0)
    b, seed = 8, 21
    U, T, V, st = oracle.randutv_reorth(A, b, q, seed)
    assert st == 0
    check_utv(A, U, T, V, b)
    G = oracle.randn(60, b, seed, 1, 1)
    W = G.copy()
    for _ in range(q + 1):
        W = A @ (A.T @ W)
    Q, _ = np.linalg.qr(W)
    e_route = np.linalg.norm(A - Q @ (Q.T @ A), 2)
    assert abs(ek_spectral(T, b) - e_route) <= 1e-10 * e_route
    np.testing.assert_allclose(U[:, :b] @ U[:, :b].T, Q @ Q.T, atol=1e-9)
    Up, Tp, Vp, _ = oracle.randutv(A, b, q, seed, max_steps=1)
    np.testing.assert_allclose(np.diag(T)[:b], np.diag(Tp)[:b], rtol=1e-10)
    np.testing.assert_allclose(V[:, :b] @ V[:, :b].T, Vp[:, :b] @ Vp[:, :b].T, atol=1e-9)


@pytest.mark.parametrize("q", [2, 3, 4])
def test_reorth_keeps_what_the_plain_iteration_loses(q):
    """Sec. 2.5: without re-orthonormalization the power iteration loses the directions below about
    eps^(1/(2q+1)) sigma_max.  With sigma_j = 10^(-j/2) the b = 8 directions of the first block span
    10^3.5, so the plain sketch (singular values raised to 2q+1 >= 5) drowns the last of them in
    rounding and e_b stays near sigma_b; re-orthonormalized, e_b meets sigma_{b+1} (Eckart-Young
    optimum) to 1 %."""
    n, b = 96, 8
    rng = np.random.default_rng(0)
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sv = 10.0 ** (-np.arange(n) / 2.0)
    A = np.asfortranarray((Q1 * sv) @ Q2.T)
    _, Tp, _, _ = oracle.randutv(A, b, q, 7, max_steps=1)
    U, Tr, V, st = oracle.randutv_reorth(A, b, q, 7, max_steps=1)
    assert st == 0
    assert np.linalg.norm(A - U @ Tr @ V.T) <= 1e-12 * np.linalg.norm(A)
    ep = ek_spectral(Tp, b) / sv[b]
    er = ek_spectral(Tr, b) / sv[b]
    assert er <= 1.01, er
    assert ep >= 2.0, ep


def test_reorth_factorization_is_exact_on_ragged_sizes():
    A, s = testmats.make_matrix(130, 101, "fast", 3, 4)
    U, T, V, st = oracle.randutv_reorth(A, 24, 2, 13)
    assert st == 0
    check_utv(A, U, T, V, 24)
    assert all(ek_spectral(T, k) >= s[k] * (1 - 1e-10) for k in range(24, 101, 24))


def test_reorth_every_application_sees_orthonormal_input():
    """A first block spanning 10^8.4 (sigma_j = 10^(-1.2 j), j < b) followed by a flat tail at sigma_b / 2:
    if the sample entering an application of T22 were not orthonormal, its smallest direction would meet
    a dynamic range of 10^16.8 > 1/eps and be lost, and with the flat tail nothing brings it back.
    Orthonormalized before every application (Sec. 2.5 (ii)), q = 2 gets e_b within 1 % of sigma_{b+1};
    the plain iteration is off by more than 5x."""
    n, b = 96, 8
    rng = np.random.default_rng(0)
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    j = np.arange(n)
    sv = np.where(j < b, 10.0 ** (-1.2 * j), 10.0 ** (-1.2 * (b - 1)) * 0.5 * np.exp(-(j - b) / 200.0))
    A = np.asfortranarray((Q1 * sv) @ Q2.T)
    _, Tp, _, _ = oracle.randutv(A, b, 2, 7, max_steps=1)
    _, Tr, _, st = oracle.randutv_reorth(A, b, 2, 7, max_steps=1)
    assert st == 0
    assert ek_spectral(Tr, b) / sv[b] <= 1.01
    assert ek_spectral(Tp, b) / sv[b] >= 5.0
