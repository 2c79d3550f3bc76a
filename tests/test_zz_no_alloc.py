"""rrf_panel_qr_noalloc: the panel Householder QR for callers that cannot supply scratch memory.

Such callers (code under a memory manager that owns the whole device, loops that must not allocate
once running) get the kernel's scratch from a fixed array in device memory.  This test calls the
entry point through the C ABI twice in a row -- the array keeps the previous call's contents, so
the second call checks that what must start at zero is cleared -- and compares each result with the
workspace-based rrf_panel_qr under the same tolerances as the other panel tests.  The file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2106_13402_gb300 import rrf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    L = rrf.lib()
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    L.rrf_panel_qr_noalloc.argtypes = [i64, i64, vp, i64, vp, vp, i64, vp, vp]
    L.rrf_panel_qr_noalloc.restype = ctypes.c_int
    return L


def _noalloc(L, P):
    r, w = P.shape
    tau = torch.empty(w, dtype=torch.float64, device="cuda")
    Y = rrf.fortran_empty(r, w)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = L.rrf_panel_qr_noalloc(r, w, ctypes.c_void_p(P.data_ptr()), P.stride(1), ctypes.c_void_p(tau.data_ptr()),
                                ctypes.c_void_p(Y.data_ptr()), Y.stride(1), ctypes.c_void_p(status.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == rrf.RRF_OK, L.rrf_status_string(st)
    torch.cuda.synchronize()
    return P, tau, Y, int(status.item())


@pytest.mark.parametrize("shapes", [((3000, 128), (777, 64)), ((4100, 256), (4100, 256)),
                                    ((152 * 64 + 37, 256), (20000, 256))])
def test_noalloc_panel_matches_workspace_panel_twice(L, shapes):
    for call, (r, w) in enumerate(shapes):
        rng = np.random.default_rng(100 * call + r + w)
        P0 = np.asfortranarray(rng.standard_normal((r, w)))
        P1 = rrf.as_fortran(torch.from_numpy(P0).cuda())
        P2 = rrf.as_fortran(torch.from_numpy(P0).cuda())
        Pw, tau_w, Y_w, _ = rrf.panel_qr(P1)
        Pn, tau_n, Y_n, status = _noalloc(L, P2)
        assert status == 0
        Pw, tau_w, Y_w = Pw.cpu().numpy(), tau_w.cpu().numpy(), Y_w.cpu().numpy()
        Pn, tau_n, Y_n = Pn.cpu().numpy(), tau_n.cpu().numpy(), Y_n.cpu().numpy()
        np.testing.assert_allclose(np.triu(Pn[:w]), np.triu(Pw[:w]), rtol=0, atol=1e-12 * np.abs(Pw).max())
        np.testing.assert_allclose(tau_n, tau_w, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(Y_n, Y_w, rtol=0, atol=1e-11)
        np.testing.assert_allclose(np.tril(Pn, -1), np.tril(Pw, -1), rtol=0, atol=1e-11)


def test_noalloc_rejects_out_of_range_sizes(L):
    """Arguments are checked on the host.  The size check against the 2 MiB array (RRF_UNSUPPORTED) is not
    reachable on this GPU: with one CTA per SM (152) and w <= 256 the panel needs at most 1,151,232 bytes,
    which the largest case above (r >= 152 x 64, w = 256, all 152 CTAs) exercises."""
    fake = ctypes.c_void_p(0x10000)
    assert L.rrf_panel_qr_noalloc(1000, 257, fake, 1000, fake, fake, 1000, None, None) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 2
    assert L.rrf_panel_qr_noalloc(10, 20, fake, 10, fake, fake, 10, None, None) == rrf.RRF_INVALID_ARG
