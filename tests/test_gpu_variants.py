"""GPU parity of the method variants (FP64 variant kernel, through the C ABI)
against the CPU oracle with the same variants: the backward-filter smoother
(Sect. 2, Fig. 2), the mean energy loss with straggling (Sect. 1) and a
position-dependent field map (Sect. 4.3), alone and together, within the
FP64 path's 1e-9 relative tolerance."""
import numpy as np
import pytest

import oracle
import paper_2105_01796_gb300 as kf
from paper_2105_01796_gb300 import synth
from tests.test_gpu_parity import FP64, MIXED, compare, gpu_fit, handle  # noqa: F401

pytestmark = pytest.mark.gpu

BACKWARD = {"smoother": "backward"}
ELOSS = {"energy_loss": True}


def kopts(method):
    """kf_options fields for an oracle method dict."""
    method = method or {}
    kw = {}
    if method.get("smoother") == "backward":
        kw["smoother"] = kf.KF_SMOOTHER_BACKWARD_FILTER
        kw["bf_scale"] = float(method.get("bf_scale", 1e4))
    if method.get("energy_loss"):
        kw["energy_loss"] = 1
    return kw


def states_err(g, r, ev):
    """max |dx| / max(|x|, 1e-3) over the smoothed states of OK tracks."""
    ok_tracks = np.nonzero(r["status"] == 0)[0]
    o = ev["offsets"]
    idx = np.concatenate([np.arange(o[t], o[t + 1]) for t in ok_tracks])
    d = np.abs(g["states"][:, idx] - r["states"][:, idx]) / np.maximum(np.abs(r["states"][:, idx]), 1e-3)
    return d.max()


@pytest.mark.parametrize("method", [BACKWARD, ELOSS, dict(BACKWARD, **ELOSS)],
                         ids=["backward", "eloss", "backward+eloss"])
@pytest.mark.parametrize("wl,n", [("tel30_100k", 3001), ("uneven30_1m", 2500)])
def test_variants_match_oracle(handle, method, wl, n):
    ev = synth.make_event(synth.scaled(synth.WORKLOADS[wl], n))
    r = oracle.fit_batch(ev, with_states=True, method=method)
    g = gpu_fit(handle, ev, FP64, with_states=True, **kopts(method))
    compare(g, r, FP64)
    assert states_err(g, r, ev) < 1e-9


@pytest.mark.parametrize("method", [None, BACKWARD, dict(BACKWARD, **ELOSS)], ids=["rts", "backward", "all"])
def test_field_map_matches_oracle(handle, method):
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["fringe30_100k"], 2000))
    r = oracle.fit_batch(ev, with_states=True, method=method)
    g = gpu_fit(handle, ev, FP64, with_states=True, **kopts(method))
    compare(g, r, FP64)
    assert states_err(g, r, ev) < 1e-9


def test_uniform_map_equals_the_constant_field_kernel(handle):
    """The variant kernel with a uniform map reproduces the baseline FP64
    kernel (a different code path for the same method)."""
    ev = dict(synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 1500)))
    base = gpu_fit(handle, ev, FP64)
    B = np.asarray(ev["bfield"], dtype=float)
    b = np.broadcast_to(B, (4, 5, 5, 3)).copy()
    ev["field_map"] = {"origin": [-100.0, -800.0, -800.0], "spacing": [300.0, 400.0, 400.0], "b": b}
    g = gpu_fit(handle, ev, FP64)
    compare(g, base, FP64)


def test_variants_edge_cases(handle):
    """Single-state tracks, every plane a hole but three, a stopping
    particle (status NONFINITE from the energy loss), bad surface ids."""
    w = synth.scaled(synth.WORKLOADS["uneven30_1m"], 300, hole_prob=0.6)
    ev = dict(synth.make_event(w))
    sid = ev["surface_id"].copy()
    sid[ev["offsets"][5] + 1] = 999
    ev["surface_id"] = sid
    sp = ev["seed_params"].copy()
    sp[4, 7] = np.sign(sp[4, 7]) / 0.02  # 20 MeV/c: stops in the first planes
    ev["seed_params"] = sp
    one = synth.subset(ev, [0])
    one["offsets"] = np.array([0, 1], dtype=np.int32)
    for k in ("loc", "cov", "truth_states"):
        one[k] = one[k][:, :1]
    for k in ("surface_id", "is_hole"):
        one[k] = one[k][:1]
    for e in (ev, one):
        for method in (BACKWARD, dict(BACKWARD, **ELOSS)):
            r = oracle.fit_batch(e, method=method)
            g = gpu_fit(handle, e, FP64, **kopts(method))
            compare(g, r, FP64)
    r = oracle.fit_batch(ev, method=ELOSS)
    assert r["status"][7] == oracle.NONFINITE and r["status"][5] == oracle.BAD_INPUT


def test_variants_need_fp64_and_the_baseline_entry_points(handle):
    import torch
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["tel10_1k"], 64))
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(64)
    for kw in (dict(smoother=kf.KF_SMOOTHER_BACKWARD_FILTER), dict(energy_loss=1)):
        with pytest.raises(kf.KfError):
            kf.kf_fit_ex(handle, dev, out, kf.kf_default_options(MIXED, **kw))
        with pytest.raises(kf.KfError):
            kf.kf_fit_static(dev, out, kf.kf_default_options(FP64, **kw))
        with pytest.raises(kf.KfError):
            kf.kf_chi2_grad(handle, dev, opt=kf.kf_default_options(FP64, **kw),
                            out_chi2=torch.empty(64, dtype=torch.float64, device="cuda"))
    with pytest.raises(kf.KfError):  # a bad backward-filter scale
        kf.kf_fit_ex(handle, dev, out, kf.kf_default_options(FP64, smoother=1, bf_scale=-1.0))
    torch.cuda.synchronize()


def test_field_map_host_entry_and_graph_replay(handle):
    """kf_fit_host copies the map with the other inputs; a captured graph
    replays the variant kernel bit for bit."""
    import torch
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["fringe30_100k"], 700))
    method = dict(BACKWARD, **ELOSS)
    ref = gpu_fit(handle, ev, FP64, **kopts(method))
    host = kf.kf_fit_host(handle, ev, kf.kf_default_options(FP64, **kopts(method)))
    for k in ("params", "cov", "chi2", "ndf", "status"):
        assert np.array_equal(host[k], ref[k]), k
    dev = kf.event_to_device(ev)
    s = torch.cuda.Stream()
    out = kf.alloc_outputs(ev["n_tracks"])
    opt = kf.kf_default_options(FP64, use_graph=1, **kopts(method))
    for _ in range(2):
        kf.kf_fit_ex(handle, dev, out, opt, s)
        s.synchronize()
        assert np.array_equal(out["params"].cpu().numpy(), ref["params"])


def test_full_size_variants_sampled(handle):
    """The bench's variant configuration: the 100k-track fringe-field
    workload with all three variants, in the autotuned launch shape replayed
    from a CUDA graph; 300 sampled tracks against the oracle."""
    import torch
    ev = synth.make_event(synth.WORKLOADS["fringe30_100k"], with_truth_states=False)
    T = int(ev["n_tracks"])
    dev = kf.event_to_device(ev)
    out = kf.alloc_outputs(T)
    method = dict(BACKWARD, **ELOSS)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        best, _ = kf.kf_autotune(handle, dev, out, kf.kf_default_options(FP64, **kopts(method)), stream)
        opt = kf.kf_default_options(FP64, schedule=best.schedule, block=best.block,
                                    resident_warps=best.resident_warps, use_graph=1, **kopts(method))
        kf.kf_fit_ex(handle, dev, out, opt, stream)        # captures the graph
        out["params"].fill_(float("nan"))
        kf.kf_fit_ex(handle, dev, out, opt, stream)        # replays it
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    pick = np.random.default_rng(5).choice(T, 300, replace=False)
    r = oracle.fit_batch(synth.subset(ev, pick), method=method)
    gs = {k: (v[..., pick] if v.ndim == 2 else v[pick]) for k, v in g.items()}
    compare(gs, r, FP64)
