"""Failure paths of the device-side waits and of the Jacobi sweep cap, driven on purpose through
rrf_test_inject, without faulting or hanging the GPU.

- A grid barrier of the Householder panel kernel that can never complete (it waits for one CTA more than
  was launched) gives up after a short limit: the call returns, the workspace status is RRF_TIMEOUT.
- The emulated GEMM's MMA warp waits on a barrier nothing arrives on and aborts: RRF_TIMEOUT after the other
  warps' own limit (~2 s), with the tile copies in flight drained and TMEM released.
- The FP64 Jacobi sweeps capped at 1 report RRF_NOT_CONVERGED for a matrix that needs more.
After each, normal operation resumes in the same process and context and gives the right answer.
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
    yield
    rrf.test_inject(rrf.INJECT_NONE, 0)


def dev(x):
    return rrf.as_fortran(torch.from_numpy(np.asfortranarray(x)).cuda())


def host(x):
    torch.cuda.synchronize()
    return x.cpu().numpy()


def test_panel_barrier_timeout_then_recovery():
    rng = np.random.default_rng(1)
    P = rng.standard_normal((4096, 64))
    with rrf.injected(rrf.INJECT_PANEL_STALL, 2_000_000):   # ~1 ms per wait
        with pytest.raises(rrf.RrfError) as err:
            rrf.panel_qr(dev(P))
    assert err.value.status == rrf.RRF_TIMEOUT
    Pd, tau, Y, Tf = rrf.panel_qr(dev(P))
    Ro, tau_o = oracle.hqr(P)
    np.testing.assert_allclose(np.diag(host(Pd)[:64]), np.diag(Ro[:64]), rtol=1e-12)
    np.testing.assert_allclose(host(tau), tau_o, rtol=1e-12, atol=1e-15)


def test_randutv_reports_barrier_timeout():
    A, _ = testmats.make_matrix(512, 512, "exp8", 1, 2)
    Ad = dev(A)
    ws = rrf.workspace(rrf.randutv_workspace_bytes(512, 512, 64), Ad.device)
    with rrf.injected(rrf.INJECT_PANEL_STALL, 2_000_000):
        rrf.randutv(Ad, 64, 1, seed=3, ws=ws, check_status=False)
        st = rrf.lib().rrf_workspace_status(rrf._vp(ws.data_ptr()), rrf._stream(None))
    assert st == rrf.RRF_TIMEOUT
    U, T, V = (host(x) for x in rrf.randutv(Ad, 64, 1, seed=3, ws=ws))
    assert np.linalg.norm(A - U @ T @ V.T) <= 1e-12 * np.linalg.norm(A)


def test_emulated_gemm_stall_times_out_then_recovers():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((1024, 512))
    B = rng.standard_normal((512, 768))
    with rrf.injected(rrf.INJECT_GEMM_STALL, 100_000):
        with pytest.raises(rrf.RrfError) as err:
            rrf.gemm("N", "N", dev(A), dev(B), emulated=True)
    assert err.value.status == rrf.RRF_TIMEOUT
    C = host(rrf.gemm("N", "N", dev(A), dev(B), emulated=True))
    ref = A @ B
    assert np.abs(C - ref).max() <= 1e-12 * np.abs(ref).max()


def test_jacobi_sweep_cap_reports_not_converged():
    rng = np.random.default_rng(3)
    for c in (16, 64, 200):        # FP64 sweeps from I (c < 32) and after the FP32 pre-pass
        M = rng.standard_normal((c, c))
        with rrf.injected(rrf.INJECT_JACOBI_CAP, 1):
            _, _, _, st = rrf.jacobi_svd(dev(M), check_status=False)
        assert st == rrf.RRF_NOT_CONVERGED, c
        Us, s, Vs, st = rrf.jacobi_svd(dev(M))
        assert st == rrf.RRF_OK
        sv = np.linalg.svd(M, compute_uv=False)
        np.testing.assert_allclose(host(s), sv, rtol=1e-12, atol=1e-14 * sv[0])
