"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every entry point that
include/rrf.h declares, and rejects bad arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

import __graft_entry__
from paper_2106_13402_gb300 import rrf, testmats

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    __graft_entry__.build()
    return rrf.lib()


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rrf_\w+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s
    assert set(rrf.EXPORTED) <= set(syms)


def test_status_strings_and_version(L):
    assert rrf.version().startswith("rrf-gb300")
    for code, name in enumerate(["RRF_OK", "RRF_INVALID_ARG", "RRF_CUDA_ERROR", "RRF_NOT_CONVERGED", "RRF_TIMEOUT",
                                 "RRF_NUMERICAL", "RRF_UNSUPPORTED", "RRF_WORKSPACE_TOO_SMALL"]):
        assert L.rrf_status_string(code).decode() == name


def _fakes():
    # distinct addresses that are never dereferenced: validation fails first
    return [ctypes.c_void_p(0x10000 * k) for k in (1, 2, 3, 4)]


def _call(L, name, m, n, lda, b, q, ldu, ldt, ldv, ws=1 << 20, nullA=False):
    fa, fu, ft, fv = _fakes()
    return getattr(L, name)(m, n, None if nullA else fa, lda, b, q, fu, ldu, ft, ldt, fv, ldv, 1,
                            ctypes.c_void_p(0x100000), ws, None, None)


@pytest.mark.parametrize("name", ["rrf_randutv", "rrf_powerurv"])
def test_argument_validation_is_host_side(L, name):
    # m < n goes through A^T (Sec. 1.3 footnote); its arguments keep their own meaning
    assert _call(L, name, 10, 20, 9, 4, 1, 10, 10, 20) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 4
    assert _call(L, name, 10, 20, 10, 4, 1, 9, 10, 20) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 8
    assert _call(L, name, 10, 20, 10, 4, 1, 10, 10, 19) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 12
    assert _call(L, name, 10, 20, 10, 4, -1, 10, 10, 20) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 6
    assert _call(L, name, 10, 20, 10, 300, 1, 10, 10, 20) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 5
    assert _call(L, name, 10, 20, 10, 4, 1, 10, 10, 20, ws=64) == rrf.RRF_WORKSPACE_TOO_SMALL
    assert L.rrf_last_arg_error() == 15
    assert _call(L, name, 0, 0, 1, 4, 1, 1, 1, 1) == rrf.RRF_INVALID_ARG
    assert _call(L, name, 20, 10, 20, 4, 1, 20, 20, 10, nullA=True) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 3
    assert _call(L, name, 20, 10, 19, 4, 1, 20, 20, 10) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 4
    assert _call(L, name, 20, 10, 20, 0, 1, 20, 20, 10) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 5
    assert _call(L, name, 20, 10, 20, 257, 1, 20, 20, 10) == rrf.RRF_INVALID_ARG
    assert _call(L, name, 20, 10, 20, 4, -1, 20, 20, 10) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 6
    assert _call(L, name, 20, 10, 20, 4, 1, 19, 20, 10) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 8
    assert _call(L, name, 20, 10, 20, 4, 1, 20, 19, 10) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 10
    assert _call(L, name, 20, 10, 20, 4, 1, 20, 20, 9) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 12


def test_oversample_option_validation(L):
    """randUTV_boosted (Algorithm 2) is selected by opts.oversample = p > 0: 1 <= b + p <= 256, FP64 sketch,
    no re-orthonormalization, fixed q; powerURV has no oversampling."""
    fake = ctypes.c_void_p(0x10000)
    fa, fu, ft, fv = _fakes()

    def call(name, b, **kw):
        o = rrf.make_opts(**kw)
        return getattr(L, name)(40, 30, fa, 40, b, 1, fu, 40, ft, 40, fv, 30, 1, ctypes.c_void_p(0x100000),
                                1 << 20, ctypes.byref(o), None)

    for kw in (dict(oversample=-1), dict(oversample=129), dict(oversample=8, sketch_prec=rrf.SKETCH_BF16),
               dict(oversample=8, reorth=True), dict(oversample=8, q_policy=rrf.Q_LEARNED)):
        assert call("rrf_randutv", 128, **kw) == rrf.RRF_INVALID_ARG, kw
        assert L.rrf_last_arg_error() == 16
    assert call("rrf_powerurv", 16, oversample=8) == rrf.RRF_UNSUPPORTED
    o = rrf.make_opts(oversample=64)
    o.reserved[0] = 1
    assert L.rrf_randutv(40, 30, fake, 40, 16, 1, fake, 40, fake, 40, fake, 30, 1, ctypes.c_void_p(0x100000), 1 << 20,
                         ctypes.byref(o), None) == rrf.RRF_INVALID_ARG
    # the boosted workspace holds the b + p column sample and its SVD
    assert rrf.randutv_workspace_bytes(1024, 1024, 64, rrf.make_opts(oversample=64)) > \
        rrf.randutv_workspace_bytes(1024, 1024, 64)
    assert rrf.randutv_workspace_bytes(1024, 1024, 64, rrf.make_opts(oversample=0)) == \
        rrf.randutv_workspace_bytes(1024, 1024, 64)


def test_opts_struct_layout_matches_header(tmp_path):
    """The ctypes mirror of rrf_opts has the C struct's size and field offsets (compiled from include/rrf.h)."""
    fields = [f[0] for f in rrf.Opts._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rrf.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(rrf_opts));\n' +
                   "".join(f'  printf("%zu\\n", offsetof(rrf_opts, {f}));\n' for f in fields) + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(rrf.Opts)
    assert out[1:] == [getattr(rrf.Opts, f).offset for f in fields]


def test_frobenius_option_validation(L):
    fake = ctypes.c_void_p(0x10000)
    for tol in (-1.0, float("nan"), float("inf")):
        o = rrf.make_opts(frob_tol=tol if tol == tol and tol > 0 else 0.0)
        o.frob_tol = tol
        assert L.rrf_randutv(40, 30, fake, 40, 16, 1, fake, 40, fake, 40, fake, 30, 1, ctypes.c_void_p(0x100000),
                             1 << 20, ctypes.byref(o), None) == rrf.RRF_INVALID_ARG
        assert L.rrf_last_arg_error() == 16
    o = rrf.make_opts(frob_tol=1e-3)
    fa, fu, ft, fv = _fakes()
    assert L.rrf_powerurv(40, 30, fa, 40, 16, 1, fu, 40, ft, 40, fv, 30, 1, ctypes.c_void_p(0x100000),
                          1 << 20, ctypes.byref(o), None) == rrf.RRF_UNSUPPORTED
    with pytest.raises(ValueError):
        rrf.make_opts(track_frob=True)


def test_in_place_rules(L):
    """T == A: randUTV factors in place when ldt == lda; powerURV (m >= n) reads A after writing T."""
    fa, fu, ft, fv = _fakes()
    ws = ctypes.c_void_p(0x100000)
    assert L.rrf_randutv(40, 30, fa, 40, 16, 1, fu, 40, fa, 41, fv, 30, 1, ws, 1 << 20, None, None) == \
        rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 10
    assert L.rrf_randutv(40, 30, fa, 40, 16, 1, fu, 40, fa, 40, fv, 30, 1, ws, 16, None, None) == \
        rrf.RRF_WORKSPACE_TOO_SMALL
    assert L.rrf_powerurv(40, 30, fa, 40, 16, 1, fu, 40, fa, 40, fv, 30, 1, ws, 1 << 20, None, None) == \
        rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 9
    # wide powerURV consumes A into A^T first: in place is accepted (stops here at the workspace size)
    assert L.rrf_powerurv(30, 40, fa, 30, 16, 1, fu, 30, fa, 30, fv, 40, 1, ws, 16, None, None) == \
        rrf.RRF_WORKSPACE_TOO_SMALL


def test_resume_option_validation(L):
    """resume_steps: 0 <= s0 <= ceil(n / b), tall randUTV_basic with fixed q only."""
    fa, fu, ft, fv = _fakes()
    ws = ctypes.c_void_p(0x100000)

    def call(name, m, n, **kw):
        o = rrf.make_opts(**kw)
        return getattr(L, name)(m, n, fa, m, 16, 1, fu, m, ft, m, fv, n, 1, ws, 1 << 20, ctypes.byref(o), None)

    for kw in (dict(resume_steps=-1), dict(resume_steps=3), dict(resume_steps=1, oversample=8),
               dict(resume_steps=1, q_policy=rrf.Q_LEARNED)):
        assert call("rrf_randutv", 40, 30, **kw) == rrf.RRF_INVALID_ARG, kw
        assert L.rrf_last_arg_error() == 16
    assert call("rrf_randutv", 30, 40, resume_steps=1) == rrf.RRF_UNSUPPORTED
    assert call("rrf_powerurv", 40, 30, resume_steps=1) == rrf.RRF_UNSUPPORTED
    o = rrf.make_opts(resume_steps=2)
    assert L.rrf_randutv(40, 30, fa, 40, 16, 1, fu, 40, ft, 40, fv, 30, 1, ws, 16, ctypes.byref(o), None) == \
        rrf.RRF_WORKSPACE_TOO_SMALL


def test_low_rank_validation(L):
    fa, fu, ft, fv = _fakes()
    ws = ctypes.c_void_p(0x100000)
    assert L.rrf_low_rank(40, 30, 31, fu, 40, ft, 40, fv, 30, fa, 40, ws, 1 << 20, None) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 3
    assert L.rrf_low_rank(40, 30, 8, fu, 39, ft, 40, fv, 30, fa, 40, ws, 1 << 20, None) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 5
    assert L.rrf_low_rank(40, 30, 8, fu, 40, ft, 40, fv, 30, fa, 39, ws, 1 << 20, None) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 11
    assert L.rrf_low_rank(40, 30, 8, fu, 40, ft, 40, fv, 30, fa, 40, ws, 16, None) == rrf.RRF_WORKSPACE_TOO_SMALL
    assert L.rrf_last_arg_error() == 13
    assert L.rrf_low_rank_workspace(40, 30, 8) >= 8 * 30 * 8


def test_small_entry_point_validation(L):
    fake = ctypes.c_void_p(0x10000)
    assert L.rrf_gemm(b"X", b"N", 2, 2, 2, 1.0, fake, 2, fake, 2, 0.0, fake, 2, None, 0, None) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 1
    assert L.rrf_gemm(b"N", b"N", 4, 2, 3, 1.0, fake, 3, fake, 3, 0.0, fake, 4, None, 0, None) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 8
    assert L.rrf_panel_qr(10, 11, fake, 10, fake, fake, 10, None, 0, fake, 1 << 20, None) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 2
    assert L.rrf_jacobi_svd(300, fake, 300, fake, 300, fake, fake, 300, fake, 1 << 20, None) == rrf.RRF_INVALID_ARG
    assert L.rrf_randn(-1, 2, fake, 1, 0, 0, 0, None) == rrf.RRF_INVALID_ARG


def test_workspace_queries_grow_with_size(L):
    a = rrf.randutv_workspace_bytes(1024, 1024, 64)
    b = rrf.randutv_workspace_bytes(2048, 2048, 64)
    assert 0 < a < b
    assert rrf.powerurv_workspace_bytes(1024, 512, 64) > 0
    assert L.rrf_randutv_workspace(0, 4, 4, None) == 0


def test_flop_model_matches_reference_counts():
    """The algorithmic flop model of Algorithm 3 / Algorithm 1 (per-step terms documented in testmats)."""
    n = 8192
    assert abs(testmats.flops_randutv(n, n, 128, 1) / 1e12 - 5.28) < 0.01
    assert abs(testmats.flops_powerurv(n, n, 1) / 1e12 - 7.70) < 0.01
    # single-block case: SVD-only cost terms
    assert testmats.flops_randutv(10, 8, 16, 0) == 2 * 10 * 64 + 4 * 10 * 10 * 8 + 2 * 8 * 64


def test_batch_shapes_are_seeded_and_in_range():
    s1 = testmats.batch_shapes(512, 31)
    assert s1 == testmats.batch_shapes(512, 31)
    assert all(256 <= m <= 2048 and 128 <= n <= m for m, n in s1)
    assert len(set(s1)) > 400


def test_failure_injection_arguments(L):
    """rrf_test_inject validates its arguments on the host and can always be switched off."""
    assert L.rrf_test_inject(9, 1) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 1
    assert L.rrf_test_inject(rrf.INJECT_PANEL_STALL, 0) == rrf.RRF_INVALID_ARG
    assert L.rrf_last_arg_error() == 2
    assert L.rrf_test_inject(rrf.INJECT_JACOBI_CAP, -3) == rrf.RRF_INVALID_ARG
    assert L.rrf_test_inject(rrf.INJECT_NONE, 0) == rrf.RRF_OK
