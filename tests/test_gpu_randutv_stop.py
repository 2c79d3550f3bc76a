"""GPU randUTV with early termination by the Frobenius recurrence (Sec. 4.1: e_0 = ||A||_F,
e_i^2 = e_{i-1}^2 - ||T(I2, J2 u J3)||_F^2), through the C ABI, against the FP64 oracle.

e_i is the Frobenius norm of the trailing block after step i; later steps only rotate that block, so the
oracle's complete factorization gives every e_i as ||To(ib:, ib:)||_F.  Tolerances: the recurrence's e_i^2
within 1e-12 ||A||_F^2 of the oracle's (its cancellation error is of order eps ||A||_F^2 per step); a
stopped factorization keeps A = U T V^T and orthogonality to 1e-12, its first ib columns upper trapezoidal
with diagonal b x b blocks (exact zeros), and ||T(ib:, ib:)||_F within 1e-10 relative of the oracle's e_i.
A stopped factorization resumed from its step count equals the uninterrupted call bit for bit.
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


def run(A, b, q, seed, **kw):
    n = A.shape[1]
    o = rrf.make_opts(track_frob=True, steps=-(-n // b), **kw)
    U, T, V = (host(x) for x in rrf.randutv(dev(A), b, q, seed=seed, opts=o))
    return U, T, V, rrf.opts_steps_done(o), rrf.opts_frob(o)


def oracle_e(A, b, q, seed, p=0):
    n = A.shape[1]
    Uo, To, Vo, st = oracle.randutv_boosted(A, b, q, p, seed) if p else oracle.randutv(A, b, q, seed)
    assert st == 0
    return [np.linalg.norm(To[k * b:, k * b:]) for k in range(-(-n // b) + 1)]


CASES = [(300, 250, 32, 1, 0, "exp8"), (257, 129, 16, 2, 0, "fast"), (300, 250, 32, 1, 32, "exp8")]


@pytest.mark.parametrize("m,n,b,q,p,prof", CASES)
def test_frobenius_recurrence_matches_oracle(m, n, b, q, p, prof):
    A, s = testmats.make_matrix(m, n, prof, 3, 4)
    U, T, V, done, fr = run(A, b, q, 11, oversample=p)
    eo = oracle_e(A, b, q, 11, p)
    assert done == len(eo) - 1
    assert fr[-1] == 0.0
    nA2 = np.linalg.norm(A) ** 2
    for k in range(len(eo)):
        assert abs(fr[k] ** 2 - eo[k] ** 2) <= 1e-12 * nA2, (k, fr[k], eo[k])


@pytest.mark.parametrize("m,n,b,q,p,prof", CASES)
@pytest.mark.parametrize("kstop", [0, 1, 3])
def test_tolerance_stops_at_first_step_below(m, n, b, q, p, prof, kstop):
    A, s = testmats.make_matrix(m, n, prof, 3, 4)
    eo = oracle_e(A, b, q, 11, p)
    tol = np.sqrt(eo[kstop] * eo[kstop + 1])
    U, T, V, done, fr = run(A, b, q, 11, oversample=p, frob_tol=tol)
    assert done == kstop + 1
    res = np.linalg.norm(A - U @ T @ V.T) / np.linalg.norm(A)
    assert res <= 1e-12
    assert np.abs(U.T @ U - np.eye(m)).max() <= 1e-12
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
    k = done * b
    assert np.all(np.tril(T[:, :k], -1) == 0.0)
    for o in range(0, k, b):
        blk = T[o:o + b, o:o + b]
        assert np.all(blk * (1.0 - np.eye(*blk.shape)) == 0.0)
    tail = np.linalg.norm(T[k:, k:])
    assert abs(tail - eo[done]) <= 1e-10 * eo[done]
    assert abs(fr[-1] ** 2 - eo[done] ** 2) <= 1e-12 * np.linalg.norm(A) ** 2
    assert fr[-1] <= tol < fr[-2]


def test_tolerance_above_norm_does_no_step():
    A, s = testmats.make_matrix(100, 80, "exp8", 3, 4)
    U, T, V, done, fr = run(A, 32, 1, 11, frob_tol=2 * np.linalg.norm(A))
    assert done == 0
    assert np.array_equal(T, A)
    assert np.array_equal(U, np.eye(100)) and np.array_equal(V, np.eye(80))
    assert abs(fr[0] - np.linalg.norm(A)) <= 1e-13 * np.linalg.norm(A)


def test_low_rank_approximation_error_is_the_trailing_norm():
    """A_k = U1 (T11 V1^T + T12 V2^T) from the stopped factorization (Sec. 4.1): ||A - A_k||_F = e_done and
    ||A - A_k||_2 = ||T(k:, k:)||_2."""
    A, s = testmats.make_matrix(300, 250, "exp8", 3, 4)
    eo = oracle_e(A, 32, 1, 11)
    tol = np.sqrt(eo[2] * eo[3])
    o = rrf.make_opts(frob_tol=tol, track_frob=True, steps=8)
    U, T, V = rrf.randutv(dev(A), 32, 1, seed=11, opts=o)
    k = rrf.opts_steps_done(o) * 32
    assert k == 96
    Ak = host(rrf.low_rank(U, T, V, k))
    Th = host(T)
    err = A - Ak
    assert abs(np.linalg.norm(err) - eo[3]) <= 1e-10 * eo[3] + 1e-12 * np.linalg.norm(A)
    t2 = np.linalg.norm(Th[k:, k:], 2)
    assert abs(np.linalg.norm(err, 2) - t2) <= 1e-10 * t2 + 1e-12 * np.linalg.norm(A)


@pytest.mark.parametrize("m,n,b,q,prof", [(300, 250, 32, 1, "exp8"), (257, 129, 16, 2, "fast")])
def test_stop_then_resume_equals_one_call(m, n, b, q, prof):
    """A factorization stopped by the tolerance and resumed (opts.resume_steps) gives the uninterrupted
    call's U, T, V bit for bit; A is not read when resuming."""
    A, s = testmats.make_matrix(m, n, prof, 3, 4)
    steps = -(-n // b)
    Uf, Tf, Vf = (host(x) for x in rrf.randutv(dev(A), b, q, seed=5))
    eo = oracle_e(A, b, q, 5)
    o1 = rrf.make_opts(frob_tol=np.sqrt(eo[2] * eo[3]), track_frob=True, steps=steps)
    U, T, V = rrf.randutv(dev(A), b, q, seed=5, opts=o1)
    s0 = rrf.opts_steps_done(o1)
    assert s0 == 3
    o2 = rrf.make_opts(resume_steps=s0, track_frob=True, steps=steps)
    A_nan = dev(np.full((m, n), np.nan))
    U2, T2, V2 = rrf.randutv(A_nan, b, q, seed=5, opts=o2, out=(U, T, V))
    assert rrf.opts_steps_done(o2) == steps
    assert np.array_equal(host(U2), Uf) and np.array_equal(host(T2), Tf) and np.array_equal(host(V2), Vf)
    fr = rrf.opts_frob(o2)
    assert all(np.isnan(fr[:s0]))
    assert abs(fr[s0] - eo[s0]) <= 1e-10 * eo[s0]


def cliff_matrix(m, n, b, tail, seed):
    rng = np.random.default_rng(seed)
    Q1, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.where(np.arange(n) < b, 1.0, tail)
    return np.asfortranarray((Q1 * s) @ Q2.T)


def test_recurrence_floor_gives_true_trailing_norm():
    """Below 2^-30 e_0^2 the recurrence is dominated by rounding (its absolute error is some units of
    2^-53 ||A||_F^2 per step), so there the trailing block's norm is summed directly.  A cliff after the
    first block (s_j = 1, then 1e-6) puts e_1^2 near 1e-11 e_0^2, where the recurrence would be off by
    ~1e-5 relative; the reported e_1 .. e_{s-1} must match the oracle's trailing norms to 1e-7."""
    m, n, b = 300, 250, 32
    A = cliff_matrix(m, n, b, 1e-6, 77)
    U, T, V, done, fr = run(A, b, 1, 3)
    assert done == -(-n // b)
    eo = oracle_e(A, b, 1, 3)
    for k in range(1, len(eo) - 1):
        assert abs(fr[k] - eo[k]) <= 1e-7 * eo[k], (k, fr[k], eo[k])


def test_tolerance_near_rounding_level_stops_correctly():
    """With s_j = 1e-9 after the first block, e_1 ~ 1.5e-8 is below the recurrence's own rounding error
    (~1e-7 here).  A tolerance of 2 e_1 must stop after step 1, one of e_1 / 2 must not."""
    m, n, b = 300, 250, 32
    A = cliff_matrix(m, n, b, 1e-9, 78)
    eo = oracle_e(A, b, 1, 3)
    e1 = eo[1]
    U, T, V, done, fr = run(A, b, 1, 3, frob_tol=2.0 * e1)
    assert done == 1
    assert abs(np.linalg.norm(T[b:, b:]) - fr[1]) <= 1e-4 * fr[1]
    U, T, V, done, fr = run(A, b, 1, 3, frob_tol=0.5 * e1)
    assert done >= 2
