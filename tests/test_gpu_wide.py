"""GPU factorizations of wide matrices (m < n) through the transpose (Sec. 1.3 footnote): the call factors
A^T = U' T' V'^T and returns U = V', T = T'^T (lower trapezoidal), V = U'.  The result must equal, bit for
bit, the tall call on A^T rearranged that way (same kernels on the same data), factor A exactly, and match
the FP64 oracle run on A^T (|diag T| within 1e-10 relative, as for tall inputs).  Also the in-place form
(T == A): bit for bit the out-of-place result.
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


def check_wide(A, U, T, V, b=None):
    m, n = A.shape
    assert np.linalg.norm(A - U @ T @ V.T) / np.linalg.norm(A) <= 1e-12
    assert np.abs(U.T @ U - np.eye(m)).max() <= 1e-12
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
    assert np.all(np.triu(T, 1) == 0.0)
    if b is not None:
        for o in range(0, m, b):
            blk = T[o:o + b, o:o + b]
            assert np.all(blk * (1.0 - np.eye(*blk.shape)) == 0.0)


@pytest.mark.parametrize("m,n,b,q,p", [(60, 100, 16, 1, 0), (129, 257, 32, 2, 0), (90, 300, 32, 1, 32),
                                       (5, 40, 8, 1, 0)])
def test_wide_randutv_is_transposed_tall(m, n, b, q, p):
    At, s = testmats.make_matrix(n, m, "exp8", 3, 4)
    A = np.asfortranarray(At.T)
    opts = rrf.make_opts(oversample=p)
    U, T, V = (host(x) for x in rrf.randutv(dev(A), b, q, seed=5, opts=opts))
    check_wide(A, U, T, V, b)
    U2, T2, V2 = (host(x) for x in rrf.randutv(dev(At), b, q, seed=5, opts=opts))
    assert np.array_equal(U, V2) and np.array_equal(T, T2.T) and np.array_equal(V, U2)
    Uo, To, Vo, st = oracle.randutv_boosted(At, b, q, p, 5) if p else oracle.randutv(At, b, q, 5)
    do = np.abs(np.diag(To))
    np.testing.assert_allclose(np.abs(np.diag(T)), do, rtol=1e-10, atol=1e-11 * do[0])


def test_wide_powerurv_is_transposed_tall():
    At, s = testmats.make_matrix(200, 120, "gaussian", 8, 9)
    A = np.asfortranarray(At.T)
    U, T, V = (host(x) for x in rrf.powerurv(dev(A), 32, 1, seed=3))
    check_wide(A, U, T, V)
    U2, T2, V2 = (host(x) for x in rrf.powerurv(dev(At), 32, 1, seed=3))
    assert np.array_equal(U, V2) and np.array_equal(T, T2.T) and np.array_equal(V, U2)
    Uo, Ro, Vo, st = oracle.powerurv(At, 1, seed=3)
    np.testing.assert_allclose(np.abs(np.diag(T)), np.abs(np.diag(Ro)), rtol=1e-8)


def test_wide_host_entry_point_matches_device():
    At, s = testmats.make_matrix(150, 70, "exp8", 1, 2)
    A = np.asfortranarray(At.T)
    Ud, Td, Vd = (host(x) for x in rrf.randutv(dev(A), 32, 1, seed=4))
    Uh, Th, Vh = rrf.randutv_host(A, 32, 1, seed=4)
    assert np.array_equal(Ud, Uh) and np.array_equal(Td, Th) and np.array_equal(Vd, Vh)


@pytest.mark.parametrize("m,n,p", [(200, 160, 0), (90, 300, 32)])
def test_randutv_in_place_equals_out_of_place(m, n, p):
    rng = np.random.default_rng(m)
    A = np.asfortranarray(rng.standard_normal((m, n)))
    opts = rrf.make_opts(oversample=p)
    U1, T1, V1 = (host(x) for x in rrf.randutv(dev(A), 32, 1, seed=5, opts=opts))
    Ad = dev(A)
    out = (rrf.fortran_empty(m, m, Ad.device), Ad, rrf.fortran_empty(n, n, Ad.device))
    U2, T2, V2 = rrf.randutv(Ad, 32, 1, seed=5, opts=opts, out=out)
    assert T2.data_ptr() == Ad.data_ptr()
    assert np.array_equal(host(U2), U1) and np.array_equal(host(T2), T1) and np.array_equal(host(V2), V1)
