"""Batched FP32 powerURV (one CUDA graph of batched kernels) against the FP64 oracle.

Each matrix of the batch is compared with the oracle's powerURV of the same matrix (cast to FP64, key
seed + i).  FP32 Householder QR is backward stable with unit roundoff u = 2^-24, so residual and
orthogonality are held to 64 sqrt(n) u, |diag R| to that bound times ||A||_2, and the entries below
the diagonal of R must be exactly zero.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2106_13402_gb300 import rrf, testmats

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")


def _make_batch(shapes, seed0):
    profiles = ("exp8", "poly", "step")
    mats = []
    for i, (m, n) in enumerate(shapes):
        A, _ = testmats.make_matrix(m, n, profiles[i % 3], seed0 + 2 * i, seed0 + 2 * i + 1)
        mats.append(A)
    return mats


def _dev32(A):
    return rrf.as_fortran(torch.from_numpy(np.asfortranarray(A.astype(np.float32))).cuda())


@pytest.mark.parametrize("q", [0, 1, 2])
def test_batched_powerurv_matches_oracle(q):
    shapes = [(64, 64), (200, 130), (257, 129), (300, 300), (130, 64), (513, 200), (96, 33), (128, 128)]
    mats = _make_batch(shapes, 50)
    plan = rrf.BatchPlan(shapes, b=64, q=q)
    ws = rrf.workspace(plan.workspace_bytes())
    As = [_dev32(A) for A in mats]
    out = plan.allocate()
    U, T, V = plan.run(As, out, seed=1000, ws=ws)
    torch.cuda.synchronize()
    big, skinny = plan.tiles()
    assert big >= 0 and skinny >= 0
    for i, (A, (m, n)) in enumerate(zip(mats, shapes)):
        A32 = A.astype(np.float32).astype(np.float64)
        Ui, Ti, Vi = (x.cpu().numpy().astype(np.float64) for x in (U[i], T[i], V[i]))
        tol = 64 * np.sqrt(n) * U32
        assert np.linalg.norm(A32 - Ui @ Ti @ Vi.T) / np.linalg.norm(A32) <= tol
        assert np.abs(Ui.T @ Ui - np.eye(m)).max() <= tol
        assert np.abs(Vi.T @ Vi - np.eye(n)).max() <= tol
        assert np.all(np.tril(Ti, -1) == 0.0)
        Uo, Ro, Vo, st = oracle.powerurv(A32, q, 1000 + i)
        nrm = np.linalg.norm(A32, 2)
        np.testing.assert_allclose(np.abs(np.diag(Ti)), np.abs(np.diag(Ro)), rtol=0, atol=tol * nrm)


def test_batched_graph_replay_is_bitwise_repeatable():
    shapes = [(300, 200), (150, 150), (400, 128)]
    mats = _make_batch(shapes, 7)
    plan = rrf.BatchPlan(shapes, b=64, q=1)
    ws = rrf.workspace(plan.workspace_bytes())
    As = [_dev32(A) for A in mats]
    out = plan.allocate()
    plan.run(As, out, seed=3, ws=ws)
    first = [x.clone() for x in out[1]]
    plan.run(As, out, seed=3, ws=ws)     # replay of the captured graph
    torch.cuda.synchronize()
    for a, b in zip(first, out[1]):
        assert torch.equal(a, b)


@pytest.mark.slow
def test_batch_512_uneven_shapes():
    """512 matrices, m ~ U[256, 2048], n ~ U[128, m], decays exp / poly / step by index (the batch
    configuration); residual and orthogonality checked on every 16th matrix."""
    shapes = testmats.batch_shapes(512, 31)
    plan = rrf.BatchPlan(shapes, b=64, q=1)
    ws = rrf.workspace(plan.workspace_bytes())
    As = []
    for i, (m, n) in enumerate(shapes):
        A, _ = testmats.make_matrix(m, n, ("exp8", "poly", "step")[i % 3], 10000 + i, 20000 + i, device="cuda")
        As.append(rrf.as_fortran(A.float()))
    out = plan.allocate()
    U, T, V = plan.run(As, out, seed=31, ws=ws)
    torch.cuda.synchronize()
    for i in range(0, 512, 16):
        m, n = shapes[i]
        A = As[i].double()
        Ui, Ti, Vi = U[i].double(), T[i].double(), V[i].double()
        tol = 64 * np.sqrt(n) * U32
        assert float(torch.linalg.norm(A - Ui @ Ti @ Vi.t()) / torch.linalg.norm(A)) <= tol
        assert float((Ui.t() @ Ui - torch.eye(m, device="cuda", dtype=torch.float64)).abs().max()) <= tol
        assert bool((torch.tril(Ti, -1) == 0).all())
