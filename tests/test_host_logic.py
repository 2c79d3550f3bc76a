"""Host-side logic on the CPU: the learned policy's label and decision rules, and the bench's clock record."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2106_13402_gb300 import qpolicy  # noqa: E402


def test_acceptable_meets_target_or_stays_near_the_better_fallback():
    sig = np.array([1.0, 1.0, 1.0])
    # columns: boundaries; rows: q = 0..3
    errs = np.array([[1.05, 1.50, 2.00],
                     [1.04, 1.30, 1.60],
                     [1.03, 1.20, 1.40],
                     [1.02, 1.12, 1.20]])
    ok = qpolicy.acceptable(errs, sig)
    assert ok[:, 0].all()                                  # every q within 1.1 sigma
    assert list(ok[:, 1]) == [False, False, False, True]   # none within 1.1; 1.05 x 1.12 = 1.176 admits q = 3 only
    assert list(ok[:, 2]) == [False, False, False, True]
    labels = np.argmax(ok, axis=0)
    assert list(labels) == [0, 3, 3]


def test_acceptable_requires_the_target_wherever_the_fallback_meets_it():
    """q = 1 within 5 % of q = 2 is not enough when q = 2 meets 1.1 sigma_{k+1} and q = 1 does not."""
    sig = np.array([1.0])
    errs = np.array([[1.30], [1.12], [1.08], [1.07]])
    ok = qpolicy.acceptable(errs, sig)[:, 0]
    assert list(ok) == [False, False, True, True]
    assert np.argmax(ok) == 2


def test_acceptable_uses_the_better_of_q2_and_q3_as_reference():
    sig = np.array([0.5])
    errs = np.array([[1.0], [0.80], [0.70], [0.69]])
    ok = qpolicy.acceptable(errs, sig)[:, 0]
    # reference min(0.70, 0.69) = 0.69 -> slack 0.7245: q = 2 and q = 3 qualify, q = 1 does not
    assert list(ok) == [False, False, True, True]


def test_decide_takes_smallest_q_reaching_the_confidence():
    # softmax probabilities 0.4, 0.35, 0.2, 0.05: argmax would say 0, the 0.8 rule says 2
    p = np.array([[0.4, 0.35, 0.2, 0.05], [0.9, 0.05, 0.03, 0.02], [0.1, 0.1, 0.1, 0.7]])
    z = np.log(p)
    assert list(qpolicy.decide(z)) == [2, 0, 3]
    assert list(qpolicy.decide(z, confidence=0.5)) == [1, 0, 3]


def test_clock_summary_reports_throttle_reasons():
    lines = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1995, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n",
        "0, 1500, 2070, 1390.0, 0x8, Active, Not Active, Not Active, Active\n",
        "garbage line\n",
    ]
    c = bench.ClockSampler.summarize(lines)
    assert c["samples"] == 3 and c["sm_mhz"] == 1995 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler.summarize(["x"]) is None


def test_measured_peaks_fall_back_when_absent(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench.measured_peaks()
    assert src == "fallback" and peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0


def test_boundary_ratios_use_the_spectral_norm():
    """bench's e_k / sigma_{k+1} helper (power iteration) against numpy's 2-norm of the trailing blocks."""
    torch = __import__("pytest").importorskip("torch")
    rng = np.random.default_rng(3)
    T = np.triu(rng.standard_normal((96, 96))) * np.logspace(0, -3, 96)
    s = np.logspace(0, -3, 96)
    r = bench._boundary_ratios(torch, torch.from_numpy(T), s, 32, [32, 64])
    for k in (32, 64):
        assert abs(r[str(k)] - np.linalg.norm(T[k:, k:], 2) / s[k]) <= 1e-4 * r[str(k)]


def test_input_recipes_have_the_prescribed_spectra():
    """The seeded inputs are Q1 diag(s) Q2^T with the recipe's singular values (numpy's SVD recovers them),
    and the 8192^2 spectrum is continuous at its plateau (s_{n/2 - 1} * 10^(-8/n) = 1e-4)."""
    from paper_2106_13402_gb300 import testmats
    for prof in ("exp100", "c2", "poly", "fast", "sshape", "step", "exp8"):
        A, s = testmats.make_matrix(120, 96, prof, 5, 6)
        assert abs(s[0] - 1.0) <= 1e-5 and np.all(np.diff(s) <= 0)   # the S-shape starts at 1 - 4e-6
        sv = np.linalg.svd(A, compute_uv=False)
        assert np.max(np.abs(sv - s)) <= 1e-13, prof
    n = 8192
    s = testmats.singular_values(n, "c2")
    assert s[n // 2] == 1e-4 and abs(s[n // 2 - 1] * 10 ** (-8 / n) - 1e-4) <= 1e-18
    A, s = testmats.make_matrix(60, 40, "rank", 1, 2, rank=8)
    assert np.linalg.matrix_rank(A) == 8
    G, none = testmats.make_matrix(30, 20, "gaussian", 3, 4)
    assert none is None and G.flags["F_CONTIGUOUS"]


class _FakeProfiler:
    """Stands in for the library's event-profiler getters (no GPU): fixed per-kind sums."""

    def __init__(self, emu_ms, pan_ms, dfma_ms):
        self.emu_ms, self.pan_ms, self.dfma_ms = emu_ms, pan_ms, dfma_ms

    def gemm_profile_end(self):
        return self.dfma_ms, 1e9, 10

    def gemm_profile_emulated(self):
        return self.emu_ms, 2e12, 56e12, 100

    def gemm_profile_emulated_bytes(self):
        return 2.0e10

    def gemm_profile_panel(self):
        return self.pan_ms, 2.6e8 * 30, 1.2e7 * 30, 30


PEAKS = {"hbm_gbs": 6674.5, "bf16_tflops": 1903.3, "bf16_tflops_sustained": 1712.4}


def test_roofline_reports_the_kernel_with_the_most_time():
    r = bench.dominant_kernel_roofline(_FakeProfiler(40.0, 50.0, 2.0), 100.0, 1, PEAKS, "measured")
    assert r["kernel"].startswith("panel_qr_kernel") and r["bound"] == "alu"
    assert [o["kernel"].split()[0] for o in r["others"]] == ["ozaki_gemm_kernel", "gemm_f64_kernel"]
    # achieved = flops / time; frac against the FP64 pipe's peak
    assert abs(r["achieved"] - 2.6e8 * 30 / 0.05 / 1e12) < 1e-3
    assert abs(r["frac"] - r["achieved"] / bench.FP64_PEAK_TFLOPS) < 1e-3
    r = bench.dominant_kernel_roofline(_FakeProfiler(60.0, 50.0, 2.0), 100.0, 1, PEAKS, "measured")
    assert r["kernel"].startswith("ozaki_gemm_kernel") and r["bound"] == "tensor"
    assert abs(r["achieved"] - 56e12 / 0.06 / 1e12) < 1e-2
    assert r["peak"] == PEAKS["bf16_tflops_sustained"]
    assert abs(r["share_of_step"] - 0.6) < 1e-9
    r = bench.dominant_kernel_roofline(_FakeProfiler(0.0, 0.0, 0.0), 100.0, 1, PEAKS, "measured")
    assert r["kernel"] is None and r["others"] == []


def test_kernel_traffic_is_withdrawn_when_the_source_changes(monkeypatch):
    entry = dict(bench.KERNEL_TRAFFIC["ozaki_step_8192"])
    monkeypatch.setitem(bench.KERNEL_TRAFFIC, "probe", dict(entry, kernel_sha1=bench.source_sha1(entry["source"])))
    assert bench.kernel_traffic("probe")[0] == entry["bytes_per_launch"]
    monkeypatch.setitem(bench.KERNEL_TRAFFIC, "probe", dict(entry, kernel_sha1="0" * 40))
    value, why = bench.kernel_traffic("probe")
    assert value is None and "changed" in why
    monkeypatch.setitem(bench.KERNEL_TRAFFIC, "probe", dict(entry, bytes_per_launch=None))
    assert bench.kernel_traffic("probe") == (None, "no capture recorded")


def test_kernel_code_hash_ignores_comments_only():
    code = "// header\n__global__ void k(int* p) {  /* body */\n  p[0] = 1;  // store\n}\n"
    same = "// another header\n\n__global__ void k(int* p) {\n  p[0] = 1;\n}\n"
    other = "__global__ void k(int* p) {\n  p[0] = 2;\n}\n"
    assert bench.source_sha1("x", code) == bench.source_sha1("x", same)
    assert bench.source_sha1("x", code) != bench.source_sha1("x", other)
