"""Host-side logic of bench.py that needs no GPU: per-step statistics, the
source hashes that gate the ncu-derived traffic and flop figures, and the
roofline entries built from them."""
import os
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    # compiled from the source text (not through a cached .pyc, which can lag
    # behind an edit that keeps the file's size within the same second)
    path = os.path.join(ROOT, "bench.py")
    mod = types.ModuleType("bench_under_test")
    mod.__file__ = path
    exec(compile(open(path).read(), path, "exec"), mod.__dict__)
    return mod


def test_step_stats(bench):
    st = bench.step_stats([1.0, 2.0, 3.0, 10.0])
    assert st["n"] == 4 and st["mean"] == 4.0 and st["median"] == 2.5
    assert st["min"] == 1.0 and st["max"] == 10.0
    assert st["rms"] == pytest.approx(float(np.std([1.0, 2.0, 3.0, 10.0])))


def test_source_hashes_gate_the_measured_constants(bench, monkeypatch):
    for f in (bench.mixed_kernel_sources_sha256, bench.ext_kernel_sources_sha256):
        h = f()
        assert len(h) == 64 and int(h, 16) >= 0
    # with the sources the constants were captured on, the entry is reported
    monkeypatch.setattr(bench, "EXT_SOURCES_SHA256", bench.ext_kernel_sources_sha256())
    r = bench.ext_roofline("adjoint_chi2", 100000, 50.0)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(bench.EXT_FLOPS_PER_TRACK["adjoint_chi2"] * 1e5 / 0.05 / 1e12)
    assert bench.ext_roofline("no such kernel", 100000, 50.0) is None
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS)
    # a kernel changed since the capture reports no figure
    monkeypatch.setattr(bench, "EXT_SOURCES_SHA256", "0" * 64)
    assert bench.ext_roofline("variants", 100000, 40.0) is None


def test_peaks(bench):
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2 * 2070e6 / 1e12)
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert isinstance(bench.cpu_model(), str)


def test_accuracy_metric(bench):
    """The error report of the timed fits against the oracle: zero for equal
    outputs, the planted parameter error recovered exactly, failed tracks
    left out and a status mismatch flagged."""
    rng = np.random.default_rng(0)
    T = 500
    A = rng.normal(size=(6, 6, T))
    C = np.einsum("ijt,kjt->ikt", A, A) + 6 * np.eye(6)[:, :, None]
    packed = np.stack([C[i, j] for i in range(6) for j in range(i + 1)])
    ref = {"params": rng.normal(size=(6, T)), "cov": packed, "chi2": rng.uniform(0, 60, T),
           "status": np.zeros(T, np.uint8)}
    gpu = {k: v.copy() for k, v in ref.items()}
    a = bench.accuracy(gpu, ref)
    assert a["tracks"] == T and a["status_agree"] and a["params"]["max"] == 0 and a["cov"]["max"] == 0
    scale = max(abs(ref["params"][2, 7]), np.sqrt(C[2, 2, 7]))
    gpu["params"][2, 7] += 3e-5 * scale
    assert bench.accuracy(gpu, ref)["params"]["max"] == pytest.approx(3e-5, rel=1e-6)
    gpu["status"][9] = 2
    gpu["params"][:, 9] = np.nan
    a = bench.accuracy(gpu, ref)
    assert a["tracks"] == T - 1 and not a["status_agree"]


def test_roofline_counts():
    """The roofline numerator: per-transition, per-measurement and
    per-smoother-step counts add up as documented (one track of 3 states,
    the middle one a hole; the mixed path's FP64 part is the Joseph update
    (less its K W term) and chi2 per measurement plus the two inverse columns and the noise-rank
    terms per smoother step)."""
    from paper_2105_01796_gb300 import roofline as rf
    offsets = np.array([0, 3])
    is_hole = np.array([1, 1, 0], dtype=np.uint8)   # state 0 is the reference plane
    f64, f32 = rf.batch_flops(offsets, is_hole, 0)
    prop = 2 * (4 * rf.RKN_STEP + rf.FRAME + rf.TRANSPORT + rf.NOISE)
    assert f32 == 0 and f64 == prop + 1 * (rf.GAIN + rf.JOSEPH) + 2 * (rf.CHOL + rf.SOLVE6 + rf.RTS_UPD)
    m64, m32 = rf.batch_flops(offsets, is_hole, 1)
    # the mixed Joseph update sums its K W term (21 elements x 2 FMA) in FP32
    assert m64 == (rf.JOSEPH - 84 + rf.CHI2) + 2 * (rf.INV_COLS + rf.NRANK)
    assert m32 == prop + (rf.GAIN - rf.CHI2 + 84) + 2 * rf.MIXED_SMOOTH_FP32
    assert rf.JOSEPH == 219 and rf.JOSEPH_64 == 135 and rf.INV_COLS == 141
    # inputs plus outputs once, per track and per state
    assert rf.algorithmic_bytes(offsets, is_hole) == (4 + 6 * 8 + 21 * 8 + 6 * 8 + 21 * 8 + 8 + 4 + 1) + 3 * (4 + 16 + 24 + 1)
