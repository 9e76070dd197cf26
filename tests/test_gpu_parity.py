"""GPU parity: the CUDA fit (through the C ABI) against the CPU oracle.

Tolerances are those the fit is specified to: FP64 path within 1e-9
relative; mixed path within 1e-4 on parameters and 1e-3 on covariances
(metrics in tests/metrics.py).  Inputs are seeded synthetic telescope events.
"""
import numpy as np
import pytest

import oracle
import paper_2105_01796_gb300 as kf
from paper_2105_01796_gb300 import synth
from tests.metrics import chi2_err, cov_err, param_err, state_sigmas, states_err

pytestmark = pytest.mark.gpu

FP64, MIXED = kf.KF_PRECISION_FP64, kf.KF_PRECISION_MIXED
TOL = {FP64: (1e-9, 1e-9, 1e-9), MIXED: (1e-4, 1e-3, 1e-4)}


@pytest.fixture(scope="module")
def handle():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    h = kf.Handle()
    yield h
    h.close()


def gpu_fit(handle, ev, prec, with_states=False, **opt):
    import torch
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(int(ev["n_tracks"]), int(ev["surface_id"].shape[0]),
                           with_states=with_states)
    kf.kf_fit_ex(handle, dev, out, kf.kf_default_options(prec, **opt))
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def compare(g, r, prec, tracks=None):
    tp, tc, tx = TOL[prec]
    if tracks is None:
        tracks = np.arange(g["params"].shape[1])
    st_g, st_r = g["status"][tracks], r["status"][tracks]
    assert np.array_equal(st_g, st_r), (np.bincount(st_g), np.bincount(st_r))
    ok = tracks[st_r == 0]
    assert np.array_equal(g["ndf"][ok], r["ndf"][ok])
    pe = param_err(g["params"][:, ok], r["params"][:, ok], r["cov"][:, ok])
    ce = cov_err(g["cov"][:, ok], r["cov"][:, ok])
    xe = chi2_err(g["chi2"][ok], r["chi2"][ok])
    assert pe.max() < tp, ("params", pe.max(), np.unravel_index(pe.argmax(), pe.shape))
    assert ce.max() < tc, ("cov", ce.max(), np.unravel_index(ce.argmax(), ce.shape))
    assert xe.max() < tx, ("chi2", xe.max())
    bad = tracks[st_r != 0]
    assert np.all(np.isnan(g["params"][:, bad])) and np.all(np.isnan(g["chi2"][bad]))
    return pe.max(), ce.max()


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_tel10_1k_full(handle, prec):
    ev = synth.make_event(synth.WORKLOADS["tel10_1k"])
    compare(gpu_fit(handle, ev, prec), oracle.fit_batch(ev), prec)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_tel30_several_tiles_ragged_tail(handle, prec):
    # 3001 tracks = 23 full CTAs of 128 plus a ragged tail
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["tel30_100k"], 3001))
    compare(gpu_fit(handle, ev, prec), oracle.fit_batch(ev), prec)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_uneven_tracks_with_holes_and_all_states(handle, prec):
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 2000))
    g = gpu_fit(handle, ev, prec, with_states=True)
    r = oracle.fit_batch(ev, with_states=True)
    compare(g, r, prec)
    # smoothed parameters on every state, in the parameter contract with each
    # state's own smoothed sigma as the floor
    ok = np.repeat(r["status"] == 0, np.diff(ev["offsets"].astype(np.int64)))
    err = states_err(g["states"][:, ok], r["states"][:, ok], state_sigmas(ev)[:, ok])
    assert err.max() < TOL[prec][0], err.max()


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_general_constant_field(handle, prec):
    w = synth.scaled(synth.WORKLOADS["tel10_1k"], 700)
    ev = dict(synth.make_event(w))
    ev["bfield"] = np.array([0.3, -0.2, 2.0])  # the fit's field differs from the simulation's
    compare(gpu_fit(handle, ev, prec), oracle.fit_batch(ev), prec)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_tilted_planes(handle, prec):
    ev = dict(synth.make_event(synth.scaled(synth.WORKLOADS["tel10_1k"], 500)))
    rng = np.random.default_rng(11)
    S = ev["center"].shape[1]
    rot = ev["rot"].copy()
    center = ev["center"].copy()
    for s in range(1, S):
        a, b, c = rng.normal(size=3) * 0.02
        Rx = np.array([[1, 0, 0], [0, np.cos(a), -np.sin(a)], [0, np.sin(a), np.cos(a)]])
        Ry = np.array([[np.cos(b), 0, np.sin(b)], [0, 1, 0], [-np.sin(b), 0, np.cos(b)]])
        Rz = np.array([[np.cos(c), -np.sin(c), 0], [np.sin(c), np.cos(c), 0], [0, 0, 1]])
        rot[:, s] = (Rz @ Ry @ Rx @ rot[:, s].reshape(3, 3)).ravel()
        center[:, s] += rng.normal(size=3) * 0.1
    ev["rot"], ev["center"] = rot, center
    compare(gpu_fit(handle, ev, prec), oracle.fit_batch(ev), prec)


def _edge_event():
    """Tracks of 1..11 states, holes first/last/everywhere-but-3, a bad
    surface id, a non-positive measurement variance."""
    base = synth.make_event(synth.scaled(synth.WORKLOADS["tel10_1k"], 12))
    lengths = [1, 2, 11, 11, 11, 5, 11, 3, 11, 11, 7, 11]
    keep = []
    o = base["offsets"]
    for t, L in enumerate(lengths):
        keep.append(np.arange(o[t], o[t] + L))
    idx = np.concatenate(keep)
    ev = dict(base)
    ev["offsets"] = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
    for k in ("loc", "cov", "truth_states"):
        ev[k] = np.ascontiguousarray(base[k][:, idx])
    for k in ("surface_id", "is_hole"):
        ev[k] = np.ascontiguousarray(base[k][idx]).copy()
    off = ev["offsets"]
    ev["is_hole"][off[3] + 1] = 1            # first measurement plane is a hole
    ev["is_hole"][off[4] + 10] = 1           # last state is a hole
    ev["is_hole"][off[6] + 1:off[6] + 9] = 1  # only 2 measured planes left
    ev["surface_id"][off[8] + 4] = 77        # surface that does not exist
    ev["cov"][0, off[9] + 5] = -1e-4         # non-positive variance -> S not SPD
    ev["is_hole"][off[1] + 1] = 0
    return ev


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_step_length_and_correction_options(handle, prec):
    """Several RKN sub-steps per gap (h_max below the plane spacing, and not
    dividing it) and 1, 2 or 5 plane corrections (and none, FP64 only): the
    stepping rule is deterministic, so the GPU follows the oracle's discrete
    map in each case (smoothed states of every surface compared too).
    Without corrections the path length is the straight-line estimate
    itself, which the mixed path takes in FP32: about 1e-4 of a sigma per
    fit, at the tolerance, so that case is not part of the mixed contract."""
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["tel30_100k"], 400))
    cases = [(7.0, 3), (3.0, 2), (7.0, 1), (50.0, 1), (50.0, 5)] + ([(50.0, 0), (7.0, 0)] if prec == FP64 else [])
    for h_max, n_iter in cases:
        g = gpu_fit(handle, ev, prec, with_states=True, h_max=h_max, n_iter=n_iter)
        r = oracle.fit_batch(ev, h_max=h_max, n_iter=n_iter, with_states=True)
        compare(g, r, prec)
        ok = r["status"] == 0
        assert ok.all(), (h_max, n_iter)
        # smoothed parameters on every state (each state's own sigma as the
        # floor, as in the uneven-track test)
        err = states_err(g["states"], r["states"], state_sigmas(ev, h_max=h_max, n_iter=n_iter))
        assert err.max() < TOL[prec][0], (h_max, n_iter, err.max())


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_edge_cases(handle, prec):
    ev = _edge_event()
    g = gpu_fit(handle, ev, prec, with_states=True)
    r = oracle.fit_batch(ev, with_states=True)
    assert r["status"][8] == oracle.BAD_INPUT and r["status"][9] == oracle.NON_SPD
    compare(g, r, prec)
    assert g["ndf"][0] == 0 and g["chi2"][0] == 0.0  # seed only: x_s = seed
    assert np.array_equal(g["params"][:, 0], ev["seed_params"][:, 0])


def test_empty_batch(handle):
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["tel10_1k"], 3))
    ev = synth.subset(ev, [])
    ev["offsets"] = np.zeros(1, dtype=np.int32)
    dev = kf.event_to_device(ev)
    dev["max_states"] = 1
    out = kf.alloc_outputs(0)
    kf.kf_fit_ex(handle, dev, out)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_chunked_equals_single_launch(handle, prec):
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["tel30_100k"], 1500))
    a = gpu_fit(handle, ev, prec)
    per_track = 31 * (720 if prec == FP64 else 6 * 8 + 54 * 4)
    b = gpu_fit(handle, ev, prec, workspace_bytes=per_track * 400)  # 4 chunks
    assert handle.last_launch_count() == 1 + 4
    for k in ("params", "cov", "chi2", "ndf", "status"):
        assert np.array_equal(a[k], b[k])


def test_fit_host_and_default_entry(handle):
    import torch
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["tel10_1k"], 300))
    a = gpu_fit(handle, ev, FP64)
    hb = kf.kf_fit_host(handle, ev, kf.kf_default_options(FP64))
    for k in ("params", "cov", "chi2", "ndf", "status"):
        assert np.array_equal(a[k], hb[k])
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(300)
    kf.kf_fit(dev, out)
    torch.cuda.synchronize()
    assert np.array_equal(out["params"].cpu().numpy(), a["params"])
    assert np.array_equal(out["cov"].cpu().numpy(), a["cov"])


def test_invalid_arguments(handle):
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["tel10_1k"], 4))
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(4)
    with pytest.raises(kf.KfError, match="unsupported"):
        kf.kf_fit_ex(handle, dev, out, kf.kf_default_options(7))
    with pytest.raises(kf.KfError, match="invalid"):
        kf.kf_fit_ex(handle, dev, out, kf.kf_default_options(FP64, h_max=-1.0))
    # CTA sizes: multiples of 32 up to what the register variant allows
    for prec, block, mb in ((FP64, 48, 0), (FP64, 384, 0), (MIXED, 384, 0), (MIXED, 512, 3), (MIXED, 544, 4)):
        with pytest.raises(kf.KfError, match="unsupported"):
            kf.kf_fit_ex(handle, dev, out, kf.kf_default_options(prec, block=block, min_blocks=mb))
    bad = dict(out)
    bad["params"] = None
    with pytest.raises(kf.KfError, match="invalid"):
        kf.kf_fit_ex(handle, dev, bad)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_full_size_tel30_100k_sampled(handle, prec):
    """The benchmark workload at full size, in the benchmark's launch
    configuration (the autotuner's shape, replayed from a CUDA graph into
    NaN-filled outputs); the oracle checks a random sample of 1500 tracks,
    and the whole batch equals the default launch bit for bit."""
    import torch
    ev = synth.make_event(synth.WORKLOADS["tel30_100k"])
    ref = gpu_fit(handle, ev, prec)
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(ev["n_tracks"])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        best, _ = kf.kf_autotune(handle, dev, out, kf.kf_default_options(prec), stream)
        opt = kf.kf_default_options(prec, schedule=best.schedule, block=best.block, min_blocks=best.min_blocks,
                                    resident_warps=best.resident_warps, use_graph=1)
        kf.kf_fit_ex(handle, dev, out, opt, stream)        # captures the graph
        for k in ("params", "cov", "chi2"):
            out[k].fill_(float("nan"))
        kf.kf_fit_ex(handle, dev, out, opt, stream)        # replays it
    torch.cuda.synchronize()
    g = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    for k in ("params", "cov", "chi2", "ndf", "status"):
        assert np.array_equal(g[k], ref[k]), k
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(ev["n_tracks"], 1500, replace=False))
    r = oracle.fit_batch(synth.subset(ev, sample))
    gs = {k: (v[..., sample] if v is not None else None) for k, v in g.items()}
    compare(gs, r, prec)
    assert np.all(g["status"] == 0)


def test_numeric_helpers_selftest(handle):
    """Integer-pipe float<->double conversions match the hardware ones bit for
    bit; the Newton-refined 1/sqrt and 1/x meet their stated error bounds."""
    assert kf.kf_selftest(1 << 22) == [0, 0, 0, 0, 0, 0]


def test_double_float_selftest(handle):
    """The mixed path's double-float sums, products and compensated dot
    products stay within 2^-44 of FP64 arithmetic on the same inputs
    (cancelling sums included), a bound that the float parts alone miss on
    most patterns."""
    n = 1 << 22
    c = kf.kf_selftest_df(n)
    assert c[:4] == [0, 0, 0, 0], c
    assert c[4] > n // 2, c


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_every_launch_variant_agrees(handle, prec):
    """All schedules, block sizes and register-cap variants a tuner may pick:
    FP64 results identical bit for bit, mixed results within tolerance of the
    oracle (uneven tracks with holes, so the sorted schedule reorders)."""
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 3001))
    r = oracle.fit_batch(ev)
    base = None
    shapes = [(64, 0), (128, 0), (256, 0)]
    if prec == MIXED:
        shapes += [(64, 3), (128, 3), (192, 3), (384, 3), (128, 4), (512, 4)]
    for sched in (kf.KF_SCHEDULE_GRID, kf.KF_SCHEDULE_PERSISTENT, kf.KF_SCHEDULE_SORTED, kf.KF_SCHEDULE_WAVES):
        for block, mb in shapes:
            g = gpu_fit(handle, ev, prec, schedule=sched, block=block, min_blocks=mb)
            compare(g, r, prec)
            if prec == FP64:
                if base is None:
                    base = g
                for k in ("params", "cov", "chi2", "ndf", "status"):
                    assert np.array_equal(g[k], base[k]), (sched, block, k)
    # the track teams the tuner may pick for FP64: the same status and ndf,
    # and values within 1e-11 of the one-thread kernel (a team sums some
    # matrix products in a different order, so not bit for bit; measured
    # 1.0e-12 on these 30-state tracks)
    if prec == FP64:
        ok = base["status"] == 0
        for tw in (2, 4):
            g = gpu_fit(handle, ev, prec, team_warps=tw)
            compare(g, r, prec)
            for k in ("ndf", "status"):
                assert np.array_equal(g[k], base[k]), ("team", tw, k)
            assert param_err(g["params"][:, ok], base["params"][:, ok], base["cov"][:, ok]).max() < 1e-11
            assert cov_err(g["cov"][:, ok], base["cov"][:, ok]).max() < 1e-11
            assert chi2_err(g["chi2"][ok], base["chi2"][ok]).max() < 1e-11
    # persistent launches of one-warp CTAs with a few resident warps per SM
    # (fewer warps than units: every warp takes several units)
    for sched in (kf.KF_SCHEDULE_PERSISTENT, kf.KF_SCHEDULE_SORTED):
        for w in (1, 5, 7):
            g = gpu_fit(handle, ev, prec, schedule=sched, block=32, resident_warps=w)
            compare(g, r, prec)
            if prec == FP64:
                for k in ("params", "cov", "chi2", "ndf", "status"):
                    assert np.array_equal(g[k], base[k]), (sched, w, k)


def test_graph_capture_and_replay(handle):
    """use_graph: the first call captures the launches into a CUDA graph, the
    next identical call replays it; results equal the plain launches bit for
    bit; changing an argument re-captures."""
    import torch
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 2500))
    dev = kf.event_to_device(ev)
    s = torch.cuda.Stream()
    ref = gpu_fit(handle, ev, MIXED, schedule=kf.KF_SCHEDULE_SORTED)
    opt = kf.kf_default_options(MIXED, schedule=kf.KF_SCHEDULE_SORTED, use_graph=1)
    outs = [kf.alloc_outputs(ev["n_tracks"]) for _ in range(2)]
    for out in (outs[0], outs[0], outs[1], outs[0]):   # capture, replay, re-capture, re-capture
        for v in out.values():
            if v is not None:
                v.zero_()
        with torch.cuda.stream(s):
            kf.kf_fit_ex(handle, dev, out, opt, s)
        s.synchronize()
        assert handle.last_launch_count() == 5   # pack + 3 sort kernels + fit
        for k in ("params", "cov", "chi2", "ndf", "status"):
            assert np.array_equal(out[k].cpu().numpy(), ref[k])


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_autotuner_choice_is_valid_and_cached(handle, prec):
    import time
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 20000))
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(ev["n_tracks"])
    best, ms = kf.kf_autotune(handle, dev, out, kf.kf_default_options(prec))
    assert ms > 0 and best.precision == prec
    assert best.schedule in (0, 1, 2, 3) and best.block % 32 == 0 and 32 <= best.block <= 512
    t0 = time.perf_counter()
    best2, ms2 = kf.kf_autotune(handle, dev, out, kf.kf_default_options(prec))
    assert time.perf_counter() - t0 < 0.05 and ms2 == ms       # cached
    assert (best2.schedule, best2.block, best2.min_blocks) == (best.schedule, best.block, best.min_blocks)
    # the fit with the tuned shape, and the AUTO schedule, agree with the oracle
    rng = np.random.default_rng(3)
    sample = np.sort(rng.choice(ev["n_tracks"], 1500, replace=False))
    r = oracle.fit_batch(synth.subset(ev, sample))
    for o in (best, kf.kf_default_options(prec, schedule=kf.KF_SCHEDULE_AUTO)):
        g = gpu_fit(handle, ev, prec, schedule=o.schedule, block=o.block, min_blocks=o.min_blocks)
        compare({k: (v[..., sample] if v is not None else None) for k, v in g.items()}, r, prec)


def test_full_size_uneven_1m_sampled(handle):
    """1,000,000 uneven tracks with holes in one persistent launch with the
    autotuner's launch shape (mixed precision); oracle on a 1500-track sample."""
    ev = synth.make_event(synth.WORKLOADS["uneven30_1m"])
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(ev["n_tracks"])
    best, _ = kf.kf_autotune(handle, dev, out, kf.kf_default_options(MIXED))
    g = gpu_fit(handle, ev, MIXED, schedule=best.schedule, block=best.block, min_blocks=best.min_blocks)
    assert handle.last_launch_count() <= 5       # pack (+ sort) + one fit launch
    rng = np.random.default_rng(9)
    sample = np.sort(rng.choice(ev["n_tracks"], 1500, replace=False))
    r = oracle.fit_batch(synth.subset(ev, sample))
    compare({k: (v[..., sample] if v is not None else None) for k, v in g.items()}, r, MIXED)
    assert np.all(g["status"] == 0)


@pytest.fixture(scope="module")
def tel30_4m():
    ev = synth.make_event(synth.WORKLOADS["tel30_4m"], with_truth_states=False)
    rng = np.random.default_rng(13)
    sample = np.sort(rng.choice(ev["n_tracks"], 1500, replace=False))
    return ev, sample, oracle.fit_batch(synth.subset(ev, sample))


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_full_size_tel30_4m_sampled(handle, tel30_4m, prec):
    """4,000,000 tracks x 30 planes (the throughput-scale workload) in the
    autotuner's launch shape, replayed from a CUDA graph as the benchmark
    times it; the oracle checks a random sample of 1500 tracks."""
    import torch
    ev, sample, r = tel30_4m
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(ev["n_tracks"])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        best, _ = kf.kf_autotune(handle, dev, out, kf.kf_default_options(prec), stream)
        opt = kf.kf_default_options(prec, schedule=best.schedule, block=best.block, min_blocks=best.min_blocks,
                                    resident_warps=best.resident_warps, use_graph=1)
        kf.kf_fit_ex(handle, dev, out, opt, stream)        # captures the graph
        for k in ("params", "cov", "chi2"):
            out[k].fill_(float("nan"))
        kf.kf_fit_ex(handle, dev, out, opt, stream)        # replays it
    torch.cuda.synchronize()
    g = {k: (v[..., sample].cpu().numpy() if v is not None else None) for k, v in out.items()}
    compare(g, r, prec)
    assert np.all(out["status"].cpu().numpy() == 0)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_wave_split_launch_equals_grid(handle, prec):
    """The wave-split schedule: 50k uneven tracks in 64-thread CTAs are one
    full wave (every SM's resident CTAs) plus a second launch that spreads
    the rest over all SMs in smaller CTAs. Per-track results do not depend
    on the launch shape, so they equal the plain grid launch bit for bit."""
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 50000))
    a = gpu_fit(handle, ev, prec, schedule=kf.KF_SCHEDULE_GRID, block=64)
    b = gpu_fit(handle, ev, prec, schedule=kf.KF_SCHEDULE_WAVES, block=64)
    assert handle.last_launch_count() == 1 + 2          # pack + two fit launches
    for k in ("params", "cov", "chi2", "ndf", "status"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    rng = np.random.default_rng(17)
    sample = np.sort(rng.choice(ev["n_tracks"], 1000, replace=False))
    r = oracle.fit_batch(synth.subset(ev, sample))
    compare({k: (v[..., sample] if v is not None else None) for k, v in b.items()}, r, prec)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_fault_inputs_and_extreme_tracks(handle, prec):
    """Host-made faults give a per-track status and NaN outputs for that
    track only, never a trap: NaN and Inf inputs, a non-SPD seed covariance,
    a track nearly parallel to the planes; and a straight track (q/p ~ 0)
    fits normally.  Statuses and the other tracks agree with the oracle."""
    ev = dict(synth.make_event(synth.scaled(synth.WORKLOADS["tel10_1k"], 16)))
    sp = ev["seed_params"].copy()
    sc = ev["seed_cov"].copy()
    loc = ev["loc"].copy()
    o = ev["offsets"]
    sp[2, 1] = np.nan                        # NaN seed angle
    loc[0, o[2] + 3] = np.inf                # Inf measurement
    sc[0, 3] = -sc[0, 3]                     # negative seed variance of loc0
    sp[2, 4] = 0.5 * np.pi - 1e-12           # direction parallel to the planes
    sp[4, 5] = 1e-9                          # (nearly) infinite momentum
    ev["seed_params"], ev["seed_cov"], ev["loc"] = sp, sc, loc
    g = gpu_fit(handle, ev, prec)
    r = oracle.fit_batch(ev)
    bad = [1, 2, 3, 4]
    for t in bad:
        assert g["status"][t] != 0 and r["status"][t] != 0, (t, g["status"][t], r["status"][t])
        assert np.all(np.isnan(g["params"][:, t])) and np.isnan(g["chi2"][t])
    assert g["status"][5] == 0 and r["status"][5] == 0
    good = np.setdiff1d(np.arange(16), bad)
    compare(g, r, prec, tracks=good)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_pipelined_host_entry_equals_device_entry(handle, prec):
    """A large host batch runs in 2 to 8 chunks whose copies overlap other
    chunks' fits, each fit on its own stream; the results equal the device
    entry's bit for bit (uneven tracks,
    smoothed states requested, every schedule, and a workspace cap that
    splits the batch, which serialises the fits)."""
    for n in (30001, 90001):
        ev = synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], n))
        ref = gpu_fit(handle, ev, prec, with_states=True, schedule=kf.KF_SCHEDULE_PERSISTENT)
        per_track = 31 * (720 if prec == FP64 else 6 * 8 + 54 * 4)
        for sched, cap in ((kf.KF_SCHEDULE_PERSISTENT, 0), (kf.KF_SCHEDULE_SORTED, 0), (kf.KF_SCHEDULE_GRID, 0),
                           (kf.KF_SCHEDULE_WAVES, 0), (kf.KF_SCHEDULE_PERSISTENT, 7000 * per_track),
                           (kf.KF_SCHEDULE_GRID, 7000 * per_track), (kf.KF_SCHEDULE_WAVES, 7000 * per_track)):
            opt = kf.kf_default_options(prec, schedule=sched, workspace_bytes=cap)
            host = kf.kf_fit_host(handle, ev, opt, with_states=True)
            for k in ("params", "cov", "chi2", "ndf", "status", "states"):
                assert np.array_equal(host[k], ref[k], equal_nan=True), (n, sched, cap, k)
            assert handle.last_launch_count() >= 3


# ---------------------------------------------------------------- far from the origin

def test_translated_geometry_far_from_origin(handle):
    """Moving every surface by the same vector leaves every local quantity
    (seeds, measurements, the constant field's effect) unchanged, so the fit
    must not change.  At 10 m from the origin a float position would be off
    by about 1e-3 mm (tens of sigma of a 30 um hit); the mixed path carries
    the point, direction and angles as double-float pairs and must stay
    within its contract of the oracle and of the untranslated fit."""
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["tel30_100k"], 2000))
    moved = dict(ev)
    moved["center"] = ev["center"] + np.array([[9000.0], [-7000.0], [11000.0]])
    r = oracle.fit_batch(moved)
    r0 = oracle.fit_batch(ev)
    ok = r0["status"] == 0
    # the oracle itself: translation moves its FP64 results by rounding only
    assert np.array_equal(r["status"], r0["status"])
    assert param_err(r["params"][:, ok], r0["params"][:, ok], r0["cov"][:, ok]).max() < 1e-9
    for prec in (FP64, MIXED):
        g = gpu_fit(handle, moved, prec)
        compare(g, r, prec)
        g0 = gpu_fit(handle, ev, prec)
        assert param_err(g["params"][:, ok], g0["params"][:, ok], g0["cov"][:, ok]).max() < TOL[prec][0]
        assert cov_err(g["cov"][:, ok], g0["cov"][:, ok]).max() < TOL[prec][1]


# ---------------------------------------------------------------- track teams (FP64)

@pytest.mark.parametrize("team", [2, 4])
def test_track_team_matches_oracle(handle, team):
    """Each track shared by a team of 2 or 4 warps: the 1k-track batch,
    uneven tracks with holes (the CTA's tracks step in lockstep over
    different lengths) with every smoothed state, a general field with tilted
    planes (the field-along-z shortcut off), and the edge cases -- all in
    the FP64 contract, and within 1e-12 of the one-thread-per-track kernel
    (the same arithmetic per element, summed in a few different orders)."""
    ev = synth.make_event(synth.WORKLOADS["tel10_1k"])
    g = gpu_fit(handle, ev, FP64, team_warps=team)
    compare(g, oracle.fit_batch(ev), FP64)
    one = gpu_fit(handle, ev, FP64)
    assert param_err(g["params"], one["params"], one["cov"]).max() < 1e-12
    assert cov_err(g["cov"], one["cov"]).max() < 1e-12

    ev = synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 1500))
    g = gpu_fit(handle, ev, FP64, with_states=True, team_warps=team)
    r = oracle.fit_batch(ev, with_states=True)
    compare(g, r, FP64)
    ok = np.repeat(r["status"] == 0, np.diff(ev["offsets"].astype(np.int64)))
    err = states_err(g["states"][:, ok], r["states"][:, ok], state_sigmas(ev)[:, ok])
    assert err.max() < TOL[FP64][0], err.max()

    ev = dict(synth.make_event(synth.scaled(synth.WORKLOADS["tel10_1k"], 333)))
    ev["bfield"] = np.array([0.3, -0.2, 2.0])
    rng = np.random.default_rng(12)
    rot, center = ev["rot"].copy(), ev["center"].copy()
    for s in range(1, center.shape[1]):
        a, b = rng.normal(size=2) * 0.02
        Rx = np.array([[1, 0, 0], [0, np.cos(a), -np.sin(a)], [0, np.sin(a), np.cos(a)]])
        Ry = np.array([[np.cos(b), 0, np.sin(b)], [0, 1, 0], [-np.sin(b), 0, np.cos(b)]])
        rot[:, s] = (Ry @ Rx @ rot[:, s].reshape(3, 3)).ravel()
    ev["rot"], ev["center"] = rot, center
    compare(gpu_fit(handle, ev, FP64, team_warps=team), oracle.fit_batch(ev), FP64)

    ev = _edge_event()
    g = gpu_fit(handle, ev, FP64, with_states=True, team_warps=team)
    compare(g, oracle.fit_batch(ev, with_states=True), FP64)
    assert g["ndf"][0] == 0 and np.array_equal(g["params"][:, 0], ev["seed_params"][:, 0])


def test_track_team_options(handle):
    """Team sizes other than 2 and 4 are refused; so is a team in mixed
    precision; the autotuner's choice (which includes the teams for FP64)
    fits within the contract."""
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["tel10_1k"], 64))
    with pytest.raises(kf.KfError, match="-1"):
        gpu_fit(handle, ev, FP64, team_warps=3)
    with pytest.raises(kf.KfError, match="-4"):
        gpu_fit(handle, ev, MIXED, team_warps=2)
    ev = synth.make_event(synth.WORKLOADS["tel10_1k"])
    compare(gpu_fit(handle, ev, FP64, schedule=kf.KF_SCHEDULE_AUTO), oracle.fit_batch(ev), FP64)
