"""Benchmark: tracks fitted per second on one GB300, mixed vs FP64 fit.

Workload: 100,000 synthetic muon tracks through a telescope of 30 planes
(25 mm spacing, 1 % X0 each), Bz = 2 T, p log-uniform 0.5-100 GeV, 30 um hits
(one state on the reference plane plus 30 measured states per track).
A step is one complete fit of the batch: forward filter + RTS smoother of
every track.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain FP64 C fitter) on the host
cores on a bounded sample of the same workload.  Under torchrun every rank
fits its own 100k-track batch (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "tel30_100k"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Roofline denominators for plain ALU work, from the unit counts and clocks of
# the part: 152 SMs at 2070 MHz; FP64 1.25 TFLOP/s nominal = 2 DFMA lanes per
# SM per clock; FP32 128 lanes per SM per clock.
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
FP64_PEAK_TFLOPS = SM_COUNT * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12      # 1.259
FP32_PEAK_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12    # 80.5

# DRAM traffic of the mixed kernel (dram__bytes_read.sum + dram__bytes_write.sum)
# from one ncu capture of both wave-split launches of a 100k-track, 3.1M-state
# step of the same workload: launch A 442.7 + 356.2 MB, launch B 372.7 +
# 309.2 MB.  Traffic grows in proportion to the states, so a launch's traffic
# is this per-state figure times its states.  It holds only for the kernel
# sources and build flags that were captured: any change to them makes the
# figure null.
MIXED_TRAFFIC_BYTES_PER_STATE = (442.68288e6 + 356.226304e6 + 372.705536e6 + 309.217792e6) / 3.1e6
MIXED_TRAFFIC_SOURCES_SHA256 = "97aced5b5c14c3999e2f1739b2b6d73320a1d0671d27f427ceaa7a9bae368779"
# the same for the FP64 path's kernel (one launch of the 100k-track step:
# 2301.875 + 2223.671 MB)
FP64_TRAFFIC_BYTES_PER_STATE = (2301.875e6 + 2223.671e6) / 3.1e6
FP64_TRAFFIC_SOURCES_SHA256 = "021253bb834cb2d2d256b0a9917e45781ba32226a69ae9577eb6016de1512920"


# FP64 flops the hardware counted (ncu: 2 x DFMA + DADD + DMUL thread
# instructions) per track in one 100k-track launch of the variant kernel
# (fringe30, 31 states, all three variants) and of the adjoint kernel
# (align20, 21 states; the chi2 objective and the whole-fit objective);
# reported while those kernels' sources match
EXT_FLOPS_PER_TRACK = {"variants": (2 * 12582105289 + 2760501554 + 5733751583) / 1e5,
                       "adjoint_chi2": (2 * 14277599975 + 1627200021 + 7860000013) / 1e5,
                       "adjoint_whole": (2 * 27684800044 + 2716200085 + 11449099947) / 1e5}
EXT_SOURCES_SHA256 = "3a16bfd21128941923a73fcc50dc8a0a20e200ebe1a9e8fd66701d3eb829c210"


def ext_kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in ("csrc/kf_variants.cu", "csrc/kf_adjoint.cu", "csrc/kf_fp64.cuh", "csrc/kf_device.cuh",
              "csrc/kf_internal.h", "_build.py"):
        with open(os.path.join(ROOT, "paper_2105_01796_gb300", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ext_roofline(kind, tracks, ms):
    """Roofline entry of the variant or adjoint kernel from its hardware-
    counted FP64 flops per track (None once the kernel has changed)."""
    if ext_kernel_sources_sha256() != EXT_SOURCES_SHA256 or kind not in EXT_FLOPS_PER_TRACK:
        return None
    flops = EXT_FLOPS_PER_TRACK[kind] * tracks
    achieved = flops / (ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "flops_per_launch": flops,
            "flops_source": "hardware-counted FP64 flops (ncu) of a 100k-track launch, per track"}


def kernel_sources_sha256(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2105_01796_gb300", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def mixed_kernel_sources_sha256():
    return kernel_sources_sha256(("csrc/kf_mixed.cu", "csrc/kf_device.cuh", "csrc/kf_internal.h", "_build.py"))


def fp64_kernel_sources_sha256():
    return kernel_sources_sha256(("csrc/kf_kernels.cu", "csrc/kf_transport.cuh", "csrc/kf_fp64.cuh",
                                  "csrc/kf_device.cuh", "csrc/kf_internal.h", "_build.py"))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tracks", type=int, default=None, help="override the track count")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="plain launches instead of graph replay")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the method-variant kernel (backward filter + energy loss + field map)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (chi2 gradient) kernel")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the further configurations (1k FP64 10-plane tracks, 1M uneven tracks)")
    ap.add_argument("--configs", default="all",
                    help="comma-separated names of the further configurations to run (default: all)")
    ap.add_argument("--no-scale", action="store_true",
                    help="skip the 4M-track throughput-scale workload (mixed and FP64)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm
    implementer / part codes), plus the machine type."""
    import platform
    name = None
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        kv = [ln.split(":", 1) for ln in info if ":" in ln]
        d = {}
        for k, v in kv:
            d.setdefault(k.strip(), v.strip())
        if "model name" in d:
            name = d["model name"]
        elif "CPU part" in d:
            name = "implementer %s part %s" % (d.get("CPU implementer", "?"), d["CPU part"])
    except OSError:
        pass
    return "%s (%s)" % (name or "unknown", platform.machine())


def oracle_tracks_per_s(ev, n_sample, cores, method=None, keep=None):
    """Oracle (plain FP64 C, POSIX threads) over the first n_sample tracks;
    keep (a dict) receives the oracle's outputs."""
    import oracle
    from paper_2105_01796_gb300 import synth
    sub = synth.subset(ev, np.arange(min(n_sample, ev["n_tracks"])))
    t0 = time.perf_counter()
    r = oracle.fit_batch(sub, n_threads=cores, method=method)
    dt = time.perf_counter() - t0
    if keep is not None:
        keep.update(r)
    return sub["n_tracks"] / dt, dt, sub["n_tracks"]


def accuracy(gpu, ref):
    """Error of a GPU fit against the FP64 oracle on the tracks both fitted:
    parameters |dx_i| / max(|x_i|, sqrt(C_ii)), covariance |dC_ij| /
    sqrt(C_ii C_jj) (oracle values), chi2 |d chi2| / max(chi2, 1); per track
    the largest element, then the maximum and the 99.9th percentile over
    tracks."""
    ok = (ref["status"] == 0) & (gpu["status"] == 0)
    diag = [i * (i + 1) // 2 + i for i in range(6)]
    c, g = ref["cov"][:, ok], gpu["cov"][:, ok]
    d = np.abs(c[diag])
    sd = np.sqrt(d)
    pe = np.max(np.abs(gpu["params"][:, ok] - ref["params"][:, ok]) / np.maximum(np.abs(ref["params"][:, ok]), sd), axis=0)
    scale = np.stack([np.sqrt(d[i] * d[j]) for i in range(6) for j in range(i + 1)])
    ce = np.max(np.abs(g - c) / scale, axis=0)
    xe = np.abs(gpu["chi2"][ok] - ref["chi2"][ok]) / np.maximum(np.abs(ref["chi2"][ok]), 1.0)
    q = lambda a: {"max": float(a.max()), "p99.9": float(np.percentile(a, 99.9))}
    return {"tracks": int(ok.sum()), "status_agree": bool(np.array_equal(ref["status"], gpu["status"])),
            "params": q(pe), "cov": q(ce), "chi2": q(xe)}


ADJOINT_WORKLOAD = "align20_100k"


def smoother_weights(ev, seed=5):
    """Weights v [6][T], W [21][T] of the smoothed state-0 terms of the
    whole-fit objective, of order one per term: v_i ~ N(0,1) / max(|x_i|,
    sigma_i), W_ij ~ N(0,1) / (sigma_i sigma_j) with the seed's values and
    prior widths (synthetic inputs, no fit output)."""
    T = int(ev["n_tracks"])
    rng = np.random.default_rng(seed)
    diag = [i * (i + 1) // 2 + i for i in range(6)]
    sd = np.sqrt(np.asarray(ev["seed_cov"])[diag])
    v = rng.normal(size=(6, T)) / np.maximum(np.abs(ev["seed_params"]), sd)
    W = rng.normal(size=(21, T)) / np.stack([sd[i] * sd[j] for i in range(6) for j in range(i + 1)])
    return v, W


def time_adjoint(h, kf, synth, torch, stream, l2_flush, steps, warmup, n_tracks, reduce=None):
    """The adjoint kernel on the misaligned 20-plane telescope at zero
    alignment, for two objectives: the summed chi2 (the filter's adjoint,
    kf_chi2_grad) and the whole fit's sum [chi2 + v . x_s0 + W . C_s0]
    (filter and smoother, kf_grad); each returns the values and the gradient
    with respect to the seeds and the 6 x 21 alignment parameters.  With
    several ranks, each fits its own batch and the alignment gradient is
    summed over ranks (one all-reduce of 126 doubles) inside the timed
    region."""
    ev = synth.make_event(synth.scaled(synth.WORKLOADS[ADJOINT_WORKLOAD], n_tracks))
    dev = kf.event_to_device(ev)
    T, S = int(ev["n_tracks"]), int(ev["center"].shape[1])
    d = lambda *shape: torch.empty(shape, dtype=torch.float64, device="cuda")
    chi2, par, cov, gs, ga = d(T), d(6, T), d(21, T), d(6, T), d(6, S)
    v, W = smoother_weights(ev)
    tv, tW = torch.from_numpy(v).cuda(), torch.from_numpy(W).cuda()
    calls = {"chi2": lambda: kf.kf_chi2_grad(h, dev, out_chi2=chi2, grad_seed=gs, grad_align=ga, stream=stream),
             "whole": lambda: kf.kf_grad(h, dev, dl_dparams=tv, dl_dcov=tW, out_chi2=chi2, out_params=par,
                                         out_cov=cov, grad_seed=gs, grad_align=ga, stream=stream)}
    res = {"workload": ADJOINT_WORKLOAD, "tracks": T, "states_per_track": 21}
    for name, call in calls.items():
        for _ in range(warmup):
            call()
        torch.cuda.synchronize()
        ms = []
        torch.cuda.nvtx.range_push("timed_adjoint_" + name)
        for _ in range(steps):
            l2_flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            call()
            if reduce is not None:
                reduce(ga)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        torch.cuda.nvtx.range_pop()
        step = float(np.mean(ms))
        res[name] = {"value": T / (step / 1e3), "unit": "tracks/s", "ms_per_step": step,
                     "step_ms": step_stats(ms)}
    res["chi2"]["gradient"] = "d(sum chi2)/d(seeds [6][T], alignment [6][21]) at zero alignment (FP64; filter)"
    res["whole"]["gradient"] = ("d(sum [chi2 + v . x_s0 + W . C_s0])/d(seeds, alignment) at zero alignment "
                                "(FP64; filter and RTS smoother), with chi2, x_s0, C_s0")
    # the headline entry of the adjoint: the whole fit
    res.update(value=res["whole"]["value"], unit="tracks/s", ms_per_step=res["whole"]["ms_per_step"])
    return ev, res, (v, W)


def adjoint_accuracy(h, kf, torch, ev, v, W, n_sample, cores):
    """The adjoint's gradients of the first n_sample tracks (a separate call
    on those tracks, so that the alignment gradient is theirs alone) against
    the oracle's central differences, element by element: |g - fd| /
    max(|fd|, floor), the floor being the larger of the rounding-noise model
    (1e-13 |L| / h / 1e-5) and twice the element's step-h / step-2h spread
    over 1e-5.  Both objectives; returns the accuracy entry and the oracle's
    rate."""
    import oracle
    from paper_2105_01796_gb300 import synth
    sub = synth.subset(ev, np.arange(min(n_sample, ev["n_tracks"])))
    n = int(sub["n_tracks"])
    dev = kf.event_to_device(sub)
    S = sub["center"].shape[1]
    vs, Ws = v[:, :n], W[:, :n]
    out = {}
    t_or = 0.0
    for name, wkw in (("chi2", {}), ("whole", {"dl_dparams": vs, "dl_dcov": Ws})):
        d = lambda *shape: torch.empty(shape, dtype=torch.float64, device="cuda")
        gs, ga = d(6, n), d(6, S)
        cu = {k: torch.from_numpy(np.ascontiguousarray(a)).cuda() for k, a in wkw.items()}
        kf.kf_grad(h, dev, grad_seed=gs, grad_align=ga, **cu)
        torch.cuda.synchronize()
        gs, ga = gs.cpu().numpy(), ga.cpu().numpy()
        t0 = time.perf_counter()
        fs, fa = oracle.objective_gradient_fd(sub, n_threads=cores, **wkw)
        t_or += time.perf_counter() - t0
        fs2, fa2 = oracle.objective_gradient_fd(sub, n_threads=cores, h_seed=2e-6, h_shift=2e-6, h_rot=2e-6, **wkw)
        _, l_abs = oracle.objective_per_track(sub, n_threads=cores, **wkw)
        hs = np.full((6, n), 1e-6)
        hs[4] = 1e-6 * np.abs(sub["seed_params"][4])
        fl_s = np.maximum(1e-13 * l_abs[None, :] / hs / 1e-5, 2 * np.abs(fs - fs2) / 1e-5)
        fl_a = np.maximum(1e-13 * np.sum(l_abs) / 1e-6 / 1e-5, 2 * np.abs(fa - fa2) / 1e-5)
        es = np.abs(gs - fs) / np.maximum(np.abs(fs), fl_s)
        ea = np.abs(ga - fa) / np.maximum(np.abs(fa), fl_a)
        out[name] = {"grad_seed_err_max": float(es.max()), "grad_align_err_max": float(ea.max()),
                     "grad_seed_resolved": float(np.mean(np.abs(fs) > fl_s)),
                     "grad_align_resolved": float(np.mean(np.abs(fa) > fl_a))}
    out.update(tracks=n, reference="oracle central finite differences (step 1e-6), element by element; "
               "floor = max(1e-13 |L| / h, 2 |fd(h) - fd(2h)|) / 1e-5; resolved = fraction of elements above it")
    rate = {"value": 2 * n / t_or, "unit": "tracks/s", "cores": cores,
            "kind": "oracle central finite differences",
            "sample": "%d tracks, both objectives, %d + 12 x %d batch fits each (%.1f s)" % (n, 12, S, t_or)}
    return out, rate


VARIANT_WORKLOAD = "fringe30_100k"
VARIANT_ORACLE_SAMPLE = 10_000


def time_variants(h, kf, synth, torch, stream, l2_flush, steps, warmup, n_tracks):
    """The method-variant kernel (FP64) with all three variants at once:
    backward-filter smoother, energy loss and the fringe field map, on the
    fringe-field workload (every track simulated; the oracle's rate beside
    it is taken on the first 10k)."""
    w = synth.WORKLOADS[VARIANT_WORKLOAD]
    ev = synth.make_event(synth.scaled(w, n_tracks), with_truth_states=False)
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(n_tracks)
    kw = dict(smoother=kf.KF_SMOOTHER_BACKWARD_FILTER, energy_loss=1)
    best, _ = kf.kf_autotune(h, dev, out, kf.kf_default_options(kf.KF_PRECISION_FP64, **kw), stream)
    opt = kf.kf_default_options(kf.KF_PRECISION_FP64, schedule=best.schedule, block=best.block,
                                resident_warps=best.resident_warps, use_graph=1, **kw)
    for _ in range(warmup):
        kf.kf_fit_ex(h, dev, out, opt, stream)
    torch.cuda.synchronize()
    ms = []
    torch.cuda.nvtx.range_push("timed_variants")
    for _ in range(steps):
        l2_flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        kf.kf_fit_ex(h, dev, out, opt, stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    torch.cuda.nvtx.range_pop()
    st = out["status"].cpu().numpy()
    step = float(np.mean(ms))
    host = {k: out[k].cpu().numpy() for k in ("params", "cov", "chi2", "status")}
    return ev, host, {"workload": VARIANT_WORKLOAD, "tracks": n_tracks,
                  "method": "backward-filter smoother + energy loss + field map (FP64)",
                  "value": n_tracks / (step / 1e3), "unit": "tracks/s", "ms_per_step": step,
                  "ok_tracks": int((st == 0).sum()),
                  "launch_shape": {"schedule": SCHEDULE_NAMES[best.schedule],
                                   "block": best.block, "resident_warps": best.resident_warps,
                                   "cuda_graph": True}}


SCALE_WORKLOAD = "tel30_4m"
SCHEDULE_NAMES = ["grid", "persistent", "sorted", "waves"]


def step_stats(ms):
    """Per-step device times: mean and RMS spread over the timed steps
    (the paper's protocol), plus the median, minimum and maximum."""
    a = np.asarray(ms, dtype=np.float64)
    return {"mean": float(a.mean()), "rms": float(a.std()), "median": float(np.median(a)),
            "min": float(a.min()), "max": float(a.max()), "n": int(a.size)}


def time_scale(kf, synth, torch, stream, l2_flush, steps, warmup, rank, no_cpu):
    """The throughput-scale workload: 4,000,000 tracks x 30 planes in one
    batch, mixed and FP64, each in its autotuned launch shape replayed from a
    CUDA graph.  Its own handle, freed afterwards (the FP64 record alone
    takes 89 GB)."""
    w = synth.WORKLOADS[SCALE_WORKLOAD]
    w = synth.scaled(w, w.n_tracks, seed=w.seed + 1000 * rank)
    t0 = time.perf_counter()
    ev = synth.make_event(w, with_truth_states=False)
    gen_s = time.perf_counter() - t0
    T = int(ev["n_tracks"])
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(T)
    h = kf.Handle()
    res = {"workload": SCALE_WORKLOAD, "tracks": T, "planes": 30, "x_over_x0": 0.01, "sigma_um": 50,
           "p_GeV": [1, 100], "generation_s": gen_s}
    for name, prec in (("mixed", kf.KF_PRECISION_MIXED), ("fp64", kf.KF_PRECISION_FP64)):
        best, _ = kf.kf_autotune(h, dev, out, kf.kf_default_options(prec), stream)
        opt = kf.kf_default_options(prec, schedule=best.schedule, block=best.block, min_blocks=best.min_blocks,
                                    resident_warps=best.resident_warps, team_warps=best.team_warps, use_graph=1)
        for _ in range(warmup):
            kf.kf_fit_ex(h, dev, out, opt, stream)
        torch.cuda.synchronize()
        ms = []
        torch.cuda.nvtx.range_push("timed_scale_" + name)
        for _ in range(steps):
            l2_flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            kf.kf_fit_ex(h, dev, out, opt, stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        torch.cuda.nvtx.range_pop()
        st = step_stats(ms)
        res[name] = {"value": T / (st["mean"] / 1e3), "unit": "tracks/s", "ms_per_step": st["mean"],
                     "step_ms": st, "ok_tracks": int((out["status"] == 0).sum().item()),
                     "launch_shape": {"schedule": SCHEDULE_NAMES[best.schedule],
                                      "block": best.block, "min_blocks": best.min_blocks,
                                      "resident_warps": best.resident_warps, "cuda_graph": True}}
    res["mixed_over_fp64"] = res["mixed"]["value"] / res["fp64"]["value"]
    del h, out, dev
    torch.cuda.empty_cache()
    if not no_cpu and rank == 0:
        cores = os.cpu_count() or 1
        v, dt, n = oracle_tracks_per_s(ev, 20_000, cores)
        res["cpu_oracle"] = {"value": v, "unit": "tracks/s", "cores": cores, "kind": "oracle",
                             "sample": "first %d tracks, one pass (%.1f s)" % (n, dt)}
    return res


# Further configurations of the fit, each timed as the headline is (autotuned
# launch shape, graph replay, L2 flushed between steps) and checked against
# the oracle: the small plain FP64 batch of 10-plane tracks, and the
# 1M-track batch of uneven tracks with holes (mixed precision, one persistent
# launch over the tracks sorted longest first, as the autotuner picks).
CONFIGS = (("tel10_1k", "fp64", "all"), ("uneven30_1m", "mixed", "all"))


def fit_roofline(roofline, offsets, is_hole, prec_id, ms, hbm):
    """Roofline entry of a fit from the required flops of its own states."""
    f64, f32 = roofline.batch_flops(offsets, is_hole, prec_id)
    nbytes = roofline.algorithmic_bytes(offsets, is_hole)
    achieved = f64 / (ms / 1e3) / 1e12
    t_roof = max(f64 / (FP64_PEAK_TFLOPS * 1e12), f32 / (FP32_PEAK_TFLOPS * 1e12), nbytes / (hbm * 1e9))
    return {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "peak_source": "derived: 152 SM x 2 DFMA/clk x 2070 MHz",
            "fp64_flops_per_launch": f64, "fp32_flops_per_launch": f32, "algorithmic_bytes_per_launch": nbytes,
            "t_roof_ms": 1e3 * t_roof, "roof_frac": 1e3 * t_roof / ms, "traffic": None}


def time_config(h, kf, synth, roofline, torch, stream, l2_flush, steps, warmup, name, prec, hbm, rank):
    """One further configuration (see CONFIGS): tracks/s, its roofline and
    the event (for the oracle check)."""
    w = synth.WORKLOADS[name]
    w = synth.scaled(w, w.n_tracks, seed=w.seed + 1000 * rank)
    t0 = time.perf_counter()
    ev = synth.make_event(w, with_truth_states=False)
    gen_s = time.perf_counter() - t0
    T = int(ev["n_tracks"])
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(T)
    pid = kf.KF_PRECISION_MIXED if prec == "mixed" else kf.KF_PRECISION_FP64
    best, _ = kf.kf_autotune(h, dev, out, kf.kf_default_options(pid), stream)
    opt = kf.kf_default_options(pid, schedule=best.schedule, block=best.block, min_blocks=best.min_blocks,
                                resident_warps=best.resident_warps, team_warps=best.team_warps, use_graph=1)
    for _ in range(warmup):
        kf.kf_fit_ex(h, dev, out, opt, stream)
    torch.cuda.synchronize()
    ms = []
    torch.cuda.nvtx.range_push("timed_" + name)
    for _ in range(steps):
        l2_flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        kf.kf_fit_ex(h, dev, out, opt, stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    torch.cuda.nvtx.range_pop()
    st = step_stats(ms)
    one = None
    if best.team_warps > 1:
        # the same batch with one thread per track (grid of 64-thread CTAs),
        # for comparison with the track-team mapping the autotuner picked
        opt1 = kf.kf_default_options(pid, schedule=kf.KF_SCHEDULE_GRID, block=64, use_graph=1)
        for _ in range(warmup):
            kf.kf_fit_ex(h, dev, out, opt1, stream)
        torch.cuda.synchronize()
        ms1 = []
        for _ in range(steps):
            l2_flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            kf.kf_fit_ex(h, dev, out, opt1, stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms1.append(a.elapsed_time(b))
        s1 = step_stats(ms1)
        one = {"value": T / (s1["mean"] / 1e3), "unit": "tracks/s", "ms_per_step": s1["mean"], "step_ms": s1,
               "launch_shape": {"schedule": "grid", "block": 64, "team_warps": 1, "cuda_graph": True}}
        # the timed fit's outputs are the tuned launch's
        kf.kf_fit_ex(h, dev, out, opt, stream)
        torch.cuda.synchronize()
    holes = np.asarray(ev["is_hole"], dtype=bool)
    res = {"workload": name, "tracks": T, "states": int(ev["surface_id"].shape[0]),
           "precision": prec, "holes": int(holes.sum()) - T, "generation_s": gen_s,
           "value": T / (st["mean"] / 1e3), "unit": "tracks/s", "ms_per_step": st["mean"], "step_ms": st,
           "ok_tracks": int((out["status"] == 0).sum().item()),
           "launch_shape": {"schedule": SCHEDULE_NAMES[best.schedule], "block": best.block,
                            "min_blocks": best.min_blocks, "resident_warps": best.resident_warps,
                            "team_warps": max(1, best.team_warps), "cuda_graph": True},
           "roofline": fit_roofline(roofline, ev["offsets"], ev["is_hole"], pid, st["mean"], hbm)}
    if one is not None:
        one["roofline"] = fit_roofline(roofline, ev["offsets"], ev["is_hole"], pid, one["ms_per_step"], hbm)
        res["one_thread_per_track"] = one
    host = {k: out[k].cpu().numpy() for k in ("params", "cov", "chi2", "status")}
    return ev, host, res


def run_reference(args, rank, world):
    """CPU oracle arm: each step fits a bounded sample on the host cores."""
    if rank != 0:
        return
    from paper_2105_01796_gb300 import synth
    w = synth.WORKLOADS[WORKLOAD]
    if args.tracks:
        w = synth.scaled(w, args.tracks)
    ev = synth.make_event(w)
    cores = os.cpu_count() or 1
    sample = min(20000, ev["n_tracks"])
    for _ in range(args.warmup):
        oracle_tracks_per_s(ev, min(sample, 2000), cores)
    times = []
    for _ in range(args.steps):
        _, dt, n = oracle_tracks_per_s(ev, sample, cores)
        times.append(dt)
    ms = 1e3 * float(np.mean(times))
    value = sample / (ms / 1e3)
    line = {
        "impl": "reference", "metric": "tracks_fitted_per_s", "value": value,
        "unit": "tracks/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "tracks": int(ev["n_tracks"]), "planes": 30,
                   "sample_tracks_per_step": sample, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "tracks/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                         "sample": "first %d of %d tracks per step" % (sample, ev["n_tracks"])},
        "e2e": {"value": value, "unit": "tracks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch
    import paper_2105_01796_gb300 as kf
    from paper_2105_01796_gb300 import _build, roofline, synth
    from paper_2105_01796_gb300 import dist as kdist

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    w = synth.WORKLOADS[WORKLOAD]
    if args.tracks:
        w = synth.scaled(w, args.tracks)
    w = synth.scaled(w, w.n_tracks, seed=w.seed + 1000 * rank)
    ev = synth.make_event(w)
    T = int(ev["n_tracks"])
    M = int(ev["surface_id"].shape[0])
    dev = kf.event_to_device(ev)
    h = kf.Handle()
    stream = torch.cuda.Stream()          # graphs need a non-default stream
    torch.cuda.set_stream(stream)
    prec_id = {"mixed": kf.KF_PRECISION_MIXED, "fp64": kf.KF_PRECISION_FP64}
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    tuned = {}

    def timed(prec, steps, warmup):
        out = kf.alloc_outputs(T)
        # launch shape from the autotuner (untimed), then CUDA-graph replay
        best, _ = kf.kf_autotune(h, dev, out, kf.kf_default_options(prec_id[prec]), stream)
        opt = kf.kf_default_options(prec_id[prec], schedule=best.schedule, block=best.block,
                                    min_blocks=best.min_blocks, resident_warps=best.resident_warps,
                                    team_warps=best.team_warps, use_graph=0 if args.no_graph else 1)
        tuned[prec] = {"schedule": SCHEDULE_NAMES[best.schedule], "block": best.block,
                       "min_blocks": best.min_blocks, "resident_warps": best.resident_warps,
                       "team_warps": max(1, best.team_warps), "cuda_graph": not args.no_graph}
        for _ in range(warmup):
            kf.kf_fit_ex(h, dev, out, opt, stream)
        torch.cuda.synchronize()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        launches = 0
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed")        # profilers select the timed launches by this range
        for i in range(steps):
            l2_flush.zero_()                       # flush L2 between timed steps
            ev0[i].record(stream)
            kf.kf_fit_ex(h, dev, out, opt, stream)
            ev1[i].record(stream)
            launches += h.last_launch_count()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        wall = time.perf_counter() - wall0
        if dist is not None:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
        st = out["status"].cpu().numpy()
        results[prec] = {k: out[k].cpu().numpy() for k in ("params", "cov", "chi2", "status")}
        return ms, launches, wall, st

    results = {}
    # the precision not being headlined is timed first, untimed for clocks
    other = "fp64" if args.precision == "mixed" else "mixed"
    ms_other, _, _, st_other = timed(other, max(3, args.steps // 2), args.warmup)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    ms, launches, wall, st = timed(args.precision, args.steps, args.warmup)
    clocks = sampler.stop() if sampler else None
    step_ms = kdist.max_over_ranks(float(np.mean(ms)), device="cuda")
    value = world * T / (step_ms / 1e3)

    adjoint = None
    adjoint_event = None
    if not args.no_adjoint:
        adjoint_event, adjoint, adjoint_w = time_adjoint(h, kf, synth, torch, stream, l2_flush,
                                                         max(3, args.steps // 2), args.warmup, T,
                                                         reduce=kdist.sum_over_ranks if world > 1 else None)
        for name in ("chi2", "whole"):
            a_ms = kdist.max_over_ranks(adjoint[name]["ms_per_step"], device="cuda")
            adjoint[name].update(ms_per_step=a_ms, value=world * adjoint["tracks"] / (a_ms / 1e3))
            adjoint[name]["roofline"] = ext_roofline("adjoint_" + name, adjoint["tracks"], a_ms)
        adjoint.update(ms_per_step=adjoint["whole"]["ms_per_step"], value=adjoint["whole"]["value"])
    scale = None
    if not args.no_scale:
        scale = time_scale(kf, synth, torch, stream, l2_flush, max(3, args.steps // 2), args.warmup,
                           rank, args.no_cpu)
        for name in ("mixed", "fp64"):
            s_ms = kdist.max_over_ranks(scale[name]["ms_per_step"], device="cuda")
            scale[name].update(ms_per_step=s_ms, value=world * scale["tracks"] / (s_ms / 1e3))
    hbm = json.load(open(MEASURED_PEAKS)).get("hbm_gbs", 6780.0) if os.path.exists(MEASURED_PEAKS) else 6780.0
    configs = {}
    config_data = {}
    if not args.no_configs:
        for cname, cprec, _ in CONFIGS:
            if args.configs != "all" and cname not in args.configs.split(","):
                continue
            c_ev, c_out, c_res = time_config(h, kf, synth, roofline, torch, stream, l2_flush,
                                             max(3, args.steps // 2), args.warmup, cname, cprec, hbm, rank)
            c_ms = kdist.max_over_ranks(c_res["ms_per_step"], device="cuda")
            c_res.update(ms_per_step=c_ms, value=world * c_res["tracks"] / (c_ms / 1e3))
            configs[cname] = c_res
            config_data[cname] = (c_ev, c_out)
    variants = None
    variant_event = None
    if not args.no_variants:
        variant_event, variant_out, variants = time_variants(h, kf, synth, torch, stream, l2_flush,
                                                max(3, args.steps // 2), args.warmup, T)
        variants["roofline"] = ext_roofline("variants", variants["tracks"], variants["ms_per_step"])

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        host = kf.host_event(ev)
        pinned = {}
        for k in kf._HOST_DTYPES:
            t_ = torch.from_numpy(host[k]).pin_memory()
            pinned[k] = t_.numpy()
        hev = dict(host)
        hev.update(pinned)
        hev["max_states"] = kf.max_states_of(ev["offsets"])
        outs = {"params": torch.empty((6, T), dtype=torch.float64).pin_memory().numpy(),
                "cov": torch.empty((21, T), dtype=torch.float64).pin_memory().numpy(),
                "chi2": torch.empty((T,), dtype=torch.float64).pin_memory().numpy(),
                "ndf": torch.empty((T,), dtype=torch.int32).pin_memory().numpy(),
                "status": torch.empty((T,), dtype=torch.uint8).pin_memory().numpy(),
                "states": None}
        sh = tuned[args.precision]
        opt = kf.kf_default_options(prec_id[args.precision], block=sh["block"], min_blocks=sh["min_blocks"],
                                    resident_warps=sh["resident_warps"],
                                    schedule=SCHEDULE_NAMES.index(sh["schedule"]))
        for _ in range(args.warmup):
            kf.kf_fit_host(h, hev, opt, out=outs, stream=stream)
        torch.cuda.synchronize()
        e_ms = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            kf.kf_fit_host(h, hev, opt, out=outs, stream=stream)   # synchronous
            e_ms.append(1e3 * (time.perf_counter() - t0))
        h2d = sum(hev[k].nbytes for k in kf._HOST_DTYPES)
        d2h = sum(v.nbytes for v in outs.values() if v is not None)
        e2e_ms = kdist.max_over_ranks(float(np.mean(e_ms)), device="cuda")
        e2e = {"value": world * T / (e2e_ms / 1e3), "unit": "tracks/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": e2e_ms}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    f64, f32 = roofline.batch_flops(ev["offsets"], ev["is_hole"], prec_id[args.precision])
    nbytes = roofline.algorithmic_bytes(ev["offsets"], ev["is_hole"])
    kern_s = step_ms / 1e3
    achieved = f64 / kern_s / 1e12
    t_roof = max(f64 / (FP64_PEAK_TFLOPS * 1e12), f32 / (FP32_PEAK_TFLOPS * 1e12), nbytes / (hbm * 1e9))
    traffic = None
    if args.precision == "mixed" and mixed_kernel_sources_sha256() == MIXED_TRAFFIC_SOURCES_SHA256:
        traffic = MIXED_TRAFFIC_BYTES_PER_STATE * M
    cpu = None
    acc = None
    if not args.no_cpu:
        cores = os.cpu_count() or 1
        # warm the oracle build, then time a bounded sample
        oracle_tracks_per_s(ev, 500, cores)
        ref = {}
        v, dt, n = oracle_tracks_per_s(ev, T, cores, keep=ref)
        v1, dt1, n1 = oracle_tracks_per_s(ev, 5000, 1)
        # the timed fits' outputs against the oracle's on the same tracks
        acc = {prec: accuracy(res, ref) for prec, res in results.items()}
        acc["reference"] = "FP64 oracle on all %d tracks" % n
        cpu = {"value": v, "unit": "tracks/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
               "sample": "all %d tracks of the workload, one pass (%.1f s)" % (n, dt),
               "single_core": {"value": v1, "unit": "tracks/s",
                               "sample": "first %d tracks, one thread (%.1f s)" % (n1, dt1)}}
        for cname, (c_ev, c_out) in config_data.items():
            cref = {}
            cv, cdt, cn = oracle_tracks_per_s(c_ev, c_ev["n_tracks"], cores, keep=cref)
            configs[cname]["accuracy"] = dict(accuracy(c_out, cref),
                                              reference="FP64 oracle on all %d tracks" % cn)
            configs[cname]["cpu_oracle"] = {"value": cv, "unit": "tracks/s", "cores": cores, "kind": "oracle",
                                            "sample": "all %d tracks, one pass (%.1f s)" % (cn, cdt)}
        if adjoint is not None:
            acc_a, rate = adjoint_accuracy(h, kf, torch, adjoint_event, adjoint_w[0], adjoint_w[1], 200, cores)
            adjoint["accuracy"] = acc_a
            adjoint["cpu_oracle"] = rate
        if variants is not None:
            vref = {}
            vv, vdt, vn = oracle_tracks_per_s(variant_event, VARIANT_ORACLE_SAMPLE, cores,
                                              method={"smoother": "backward", "energy_loss": True}, keep=vref)
            variants["cpu_oracle"] = {"value": vv, "unit": "tracks/s", "cores": cores,
                                      "sample": "first %d tracks, one pass (%.1f s)" % (vn, vdt)}
            first = {k: (v[..., :vn]) for k, v in variant_out.items()}
            variants["accuracy"] = dict(accuracy(first, vref),
                                        reference="FP64 oracle with the same variants, first %d tracks" % vn)
    other_ms = float(np.mean(ms_other))
    line = {
        "metric": "tracks_fitted_per_s", "value": value, "unit": "tracks/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "step_ms": step_stats(ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "tracks_per_gpu": T, "planes": 30, "states": M,
                   "precision": args.precision, "field_T": 2.0, "x_over_x0": 0.01,
                   "sigma_um": 30, "p_GeV": [0.5, 100],
                   "l2": "flushed between timed steps (256 MiB write); inputs 165 MB > L2",
                   "parallelism": "one independent batch per GPU" if world > 1 else "single GPU"},
        "fp64_path" if args.precision == "mixed" else "mixed_path": {
            "value": world * T / (other_ms / 1e3), "ms_per_step": other_ms, "step_ms": step_stats(ms_other),
            "ok_tracks": int((st_other == 0).sum()),
            "roofline": dict(fit_roofline(roofline, ev["offsets"], ev["is_hole"], prec_id[other], other_ms, hbm),
                             traffic=(FP64_TRAFFIC_BYTES_PER_STATE * M
                                      if other == "fp64" and fp64_kernel_sources_sha256() == FP64_TRAFFIC_SOURCES_SHA256
                                      else None))},
        "ok_tracks": int((st == 0).sum()),
        "launch_shape": tuned,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "kernel": "fit_kernel<MixedBody>" if args.precision == "mixed" else "fit_kernel<Fp64Body>",
                     "pipe": "fp64",
                     "peak_source": "derived: 152 SM x 2 DFMA/clk x 2070 MHz",
                     "t_roof_ms": 1e3 * t_roof, "roof_frac": 1e3 * t_roof / step_ms,
                     "fp64_flops_per_launch": f64, "fp32_flops_per_launch": f32,
                     "algorithmic_bytes_per_launch": nbytes,
                     "traffic_note": ("ncu capture of both launches of a 100k-track step of this kernel (wave split, 168 registers); "
                                      "mostly the smoother's per-state record round trip (216 B each way)")
                     if traffic else "kernel changed since the last ncu capture"},
        "cpu_baseline": cpu,
        "accuracy": acc,
        "scale": scale,
        "configs": configs or None,
        "variants": variants,
        "adjoint": adjoint,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if clocks and clocks.get("sm_mhz"):
        # the same derived peak at the median SM clock sampled under load
        pk = FP64_PEAK_TFLOPS * clocks["sm_mhz"] / 2070.0
        line["roofline"].update(peak_at_sampled_clock=pk, frac_at_sampled_clock=achieved / pk)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
