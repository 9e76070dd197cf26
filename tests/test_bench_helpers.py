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
    # the committed constants belong to the committed sources
    assert bench.mixed_kernel_sources_sha256() == bench.MIXED_TRAFFIC_SOURCES_SHA256
    assert bench.ext_kernel_sources_sha256() == bench.EXT_SOURCES_SHA256
    r = bench.ext_roofline("adjoint", 100000, 50.0)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(bench.EXT_FLOPS_PER_TRACK["adjoint"] * 1e5 / 0.05 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS)
    # a kernel changed since the capture reports no figure
    monkeypatch.setattr(bench, "EXT_SOURCES_SHA256", "0" * 64)
    assert bench.ext_roofline("variants", 100000, 40.0) is None


def test_peaks(bench):
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2 * 2070e6 / 1e12)
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert isinstance(bench.cpu_model(), str)
