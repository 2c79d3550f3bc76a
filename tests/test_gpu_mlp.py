"""The learned power-iteration policy on the GPU: FP16 MLP kernels against the FP64 oracle, training,
and the policy inside randUTV.

Tolerances: parameters and activations are FP16 (unit roundoff 2^-11) with FP32 accumulation, so logits
agree with the FP64 oracle (same FP16-rounded parameters and inputs) within 5e-3 (1 + |z|) and the
gradient within 2 % in norm; the oracle's own gradient is pinned by finite differences.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2106_13402_gb300 import qpolicy, rrf, testmats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")


def _params(seed=0, scale=0.25):
    p = np.random.default_rng(seed).standard_normal(rrf.mlp_param_count()) * scale
    return p.astype(np.float16)


def test_mlp_forward_matches_oracle():
    p16 = _params(3)
    X = np.random.default_rng(4).standard_normal((1000, 16)).astype(np.float32)
    z = rrf.mlp_forward(torch.from_numpy(p16).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    zo, _ = oracle.mlp_forward(p16.astype(np.float64), X.astype(np.float64))
    assert np.all(np.abs(z - zo) <= 5e-3 * (1 + np.abs(zo)))
    margin = np.sort(zo, axis=1)[:, -1] - np.sort(zo, axis=1)[:, -2]
    sure = margin > 0.05
    assert np.array_equal(z.argmax(1)[sure], zo.argmax(1)[sure])


def test_mlp_gradient_matches_oracle():
    p16 = _params(5)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((777, 16)).astype(np.float32)
    y = rng.integers(0, 4, 777).astype(np.int32)
    g, loss = rrf.mlp_grad(torch.from_numpy(p16).cuda(), torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    lo, go = oracle.mlp_loss_grad(p16.astype(np.float64), X.astype(np.float64), y)
    g = g.cpu().numpy()
    assert abs(float(loss) - lo) <= 1e-2 * lo
    assert np.linalg.norm(g - go) <= 2e-2 * np.linalg.norm(go)


def test_mlp_training_learns_a_rule():
    """Labels from a fixed nonlinear rule of the features; Adam with the library kernels fits them."""
    rng = np.random.default_rng(7)
    X = rng.standard_normal((4096, 16)).astype(np.float32)
    y = (np.digitize(X[:, 0] + 0.5 * X[:, 1] ** 2, [-0.5, 0.5, 1.5])).astype(np.int32)
    params = qpolicy.train(X, y, epochs=40, batch=512, lr=3e-3, seed=1)
    acc = float((rrf.mlp_forward(params, torch.from_numpy(X).cuda()).argmax(1).cpu().numpy() == y).mean())
    assert acc > 0.9, acc


def test_policy_inside_randutv_keeps_an_exact_factorization():
    A, s = testmats.make_matrix(512, 512, "sshape", 1, 2)
    n, b = 512, 64
    steps = math.ceil(n / b)
    p16 = torch.from_numpy(_params(9, 0.1)).cuda()
    opts = rrf.make_opts(q_policy=rrf.Q_LEARNED, mlp_params=p16, steps=steps)
    Ad = rrf.as_fortran(torch.from_numpy(A).cuda())
    U, T, V = (x.cpu().numpy() for x in rrf.randutv(Ad, b, 2, seed=3, opts=opts))
    assert np.linalg.norm(A - U @ T @ V.T) / np.linalg.norm(A) <= 1e-12
    assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-12
    assert np.all(np.tril(T, -1) == 0.0)
    qs = rrf.opts_q_used(opts)[: steps - 1]
    assert all(0 <= q <= 3 for q in qs)
    F = rrf.opts_features(opts)[: steps - 1]
    assert np.all(np.isfinite(F)) and np.all(np.abs(F) <= 30)
    # f13..f15 use the previous step's singular values, which end up on the diagonal of T
    assert np.all(F[0, 13:16] == 0.0)
    d = np.abs(np.diag(T))
    for i in range(2, steps):
        D = d[(i - 2) * b:(i - 1) * b]
        assert abs(F[i - 1, 14] - np.log10(D[-1] / D[0])) <= 1e-5 * (1 + abs(F[i - 1, 14]))
    # the features reproduce the policy's choices through the standalone forward kernel and the
    # cumulative-probability rule
    z = rrf.mlp_forward(p16, torch.from_numpy(F).cuda()).cpu().numpy().astype(np.float64)
    assert list(qpolicy.decide(z)) == qs


def test_features_without_parameters_fall_back_to_q():
    A, s = testmats.make_matrix(256, 256, "exp8", 1, 2)
    opts = rrf.make_opts(q_policy=rrf.Q_LEARNED, steps=4)
    Ad = rrf.as_fortran(torch.from_numpy(A).cuda())
    U, T, V = rrf.randutv(Ad, 64, 2, seed=3, opts=opts)
    assert rrf.opts_q_used(opts)[:3] == [2, 2, 2]
    # same factorization as the fixed-q path (the feature QR works on a copy of the sketch)
    U2, T2, V2 = rrf.randutv(Ad, 64, 2, seed=3)
    assert torch.equal(T, T2)


def _policy_vs_fixed(params, count=8, n=1024, b=128, with_q3=False):
    """Learned policy against fixed q = 2 (and q = 3) on held-out matrices (seeds the training set never
    used): per boundary (matrix, i, q chosen, e_k learned, e_k q=2, sigma_{k+1}, e_k q=3)."""
    steps = n // b
    rows = []
    for t in range(count):
        A, s = qpolicy.make_matrix(n, 900000 + t)
        opts = rrf.make_opts(q_policy=rrf.Q_LEARNED, mlp_params=params, steps=steps)
        _, TL, _ = rrf.randutv(A, b, 2, seed=5, opts=opts)
        _, TF, _ = rrf.randutv(A, b, 2, seed=5)
        T3 = rrf.randutv(A, b, 3, seed=5)[1] if with_q3 else None
        qs = rrf.opts_q_used(opts)[: steps - 1]
        for i in range(1, steps):
            el = qpolicy.spectral_norm(torch, TL[i * b:, i * b:])
            ef = qpolicy.spectral_norm(torch, TF[i * b:, i * b:])
            e3 = qpolicy.spectral_norm(torch, T3[i * b:, i * b:]) if with_q3 else float("nan")
            rows.append((t, i, qs[i - 1], el, ef, float(s[i * b]), e3))
    return rows


def test_trained_policy_gains_over_fixed_q2():
    """The packaged network (trained on matrices the method factored itself) against the fallback q = 2 on
    held-out matrices of mixed decay: fewer power iterations in total, at least as many block boundaries
    meeting the quality target e_k <= 1.1 sigma_{k+1}, and no boundary more than 25 % above the fallback's
    e_k."""
    params = qpolicy.load()
    if params is None:
        pytest.skip("no trained policy packaged")
    rows = _policy_vs_fixed(params)
    q_learned = sum(r[2] for r in rows)
    q_fixed = 2 * len(rows)
    hit_l = sum(r[3] <= 1.1 * r[5] for r in rows)
    hit_f = sum(r[4] <= 1.1 * r[5] for r in rows)
    worst = max(r[3] / r[4] for r in rows)
    print(f"power iterations learned {q_learned} / fixed {q_fixed}; on target learned {hit_l} / fixed {hit_f} "
          f"of {len(rows)}; worst e_k learned / fixed {worst:.3f}")
    assert q_learned < q_fixed
    assert hit_l >= hit_f
    assert worst <= 1.25
