"""The adjoint kernel: gradients with respect to the seed parameters and the
per-surface alignment of the summed chi2 (kf_chi2_grad, the filter) and of
the whole fit's objective sum_t [w chi2 + v . x_s0 + W . C_s0] (kf_grad,
filter and smoother), against central finite differences of the CPU oracle
(step 1e-6) on 100 tracks of a misaligned telescope, element by element;
plus the values themselves against the fit and the torch.autograd
wrappers."""
import numpy as np
import pytest

import oracle
import paper_2105_01796_gb300 as kf
from paper_2105_01796_gb300 import synth
from tests.metrics import PAIRS, DIAG, cov_err, fd_floor, fd_floor_measured, grad_err, param_err, seed_steps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    h = kf.Handle()
    yield h
    h.close()


def _grad(handle, ev, align, weights=None):
    import torch
    dev = kf.event_to_device(ev)
    T, S = int(ev["n_tracks"]), ev["center"].shape[1]
    chi2 = torch.empty(T, dtype=torch.float64, device="cuda")
    gs = torch.empty((6, T), dtype=torch.float64, device="cuda")
    ga = torch.empty((6, S), dtype=torch.float64, device="cuda")
    a = torch.from_numpy(np.ascontiguousarray(align)).cuda()
    w = None if weights is None else torch.from_numpy(np.ascontiguousarray(weights)).cuda()
    kf.kf_chi2_grad(handle, dev, align=a, dl_dchi2=w, out_chi2=chi2, grad_seed=gs, grad_align=ga)
    torch.cuda.synchronize()
    return chi2.cpu().numpy(), gs.cpu().numpy(), ga.cpu().numpy()


def _floors(fd_h, fd_2h, seeds, l_track):
    """Element-wise floors of the seed and alignment gradients: the rounding
    noise model (tests/metrics.py; seeds from the track's |L|, alignment from
    the batch's) or each element's measured step-h / step-2h spread."""
    (fs, fa), (fs2, fa2) = fd_h, fd_2h
    fl_s = fd_floor_measured(fs, fs2, fd_floor(l_track[None, :], seed_steps(seeds)))
    fl_a = fd_floor_measured(fa, fa2, fd_floor(np.sum(np.abs(l_track)), 1e-6))
    return fl_s, fl_a


def _check_grads(gs, ga, fd_h, fd_2h, seeds, l_track, min_resolved=0.6):
    """Element-wise against the oracle's central differences (step 1e-6),
    each element to 1e-5 relative above its finite-difference floor; at
    least min_resolved of the elements lie above it (the test is not
    vacuous)."""
    (fs, fa) = fd_h
    fl_s, fl_a = _floors(fd_h, fd_2h, seeds, l_track)
    es = grad_err(gs, fs, fl_s)
    ea = grad_err(ga, fa, fl_a)
    assert es.max() < 1e-5, ("seed", es.max(), np.unravel_index(es.argmax(), es.shape))
    assert ea.max() < 1e-5, ("align", ea.max(), np.unravel_index(ea.argmax(), ea.shape))
    # elements above their floor are checked at 1e-5 relative
    assert np.mean(np.abs(fs) > fl_s) > min_resolved and np.mean(np.abs(fa) > fl_a) > min_resolved
    return fl_s, fl_a


def _fd2(fn, **kw):
    """Central differences at steps 1e-6 and 2e-6."""
    return (fn(**kw), fn(h_seed=2e-6, h_shift=2e-6, h_rot=2e-6, **kw))


@pytest.mark.parametrize("nonzero_align", [False, True])
def test_gradients_match_oracle_finite_differences(handle, nonzero_align):
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["align20_100k"], 100))
    S = ev["center"].shape[1]
    rng = np.random.default_rng(1)
    align = np.zeros((6, S))
    if nonzero_align:
        align[:3, 1:] = rng.normal(size=(3, S - 1)) * 0.05
        align[3:, 1:] = rng.normal(size=(3, S - 1)) * 5e-4
    w = rng.uniform(0.5, 1.5, size=100)
    chi2, gs, ga = _grad(handle, ev, align, w)
    ref_chi2 = oracle.chi2_per_track(ev, align)
    assert np.max(np.abs(chi2 - ref_chi2) / ref_chi2) < 1e-9
    fd = _fd2(oracle.chi2_gradient_fd, ev=ev, align=align, weights=w)
    # every element, the reference plane's alignment (which moves the seed's
    # frame) included
    _check_grads(gs, ga, fd[0], fd[1], ev["seed_params"], w * ref_chi2)


def test_chi2_equals_the_fit_and_autograd_wrapper(handle):
    import torch
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["align20_100k"], 300))
    dev = kf.event_to_device(ev)
    S = ev["center"].shape[1]
    out = kf.alloc_outputs(300)
    kf.kf_fit_ex(handle, dev, out, kf.kf_default_options(kf.KF_PRECISION_FP64))
    seeds = dev["seed_params"].clone().requires_grad_(True)
    align = torch.zeros((6, S), dtype=torch.float64, device="cuda", requires_grad=True)
    chi2 = kf.chi2_autograd(seeds, align, dev, handle)
    torch.cuda.synchronize()
    assert torch.allclose(chi2, out["chi2"], rtol=1e-12, atol=0)
    loss = (chi2 * torch.linspace(0.5, 2.0, 300, dtype=torch.float64, device="cuda")).sum()
    loss.backward()
    c2, gs, ga = _grad(handle, ev, np.zeros((6, S)), np.linspace(0.5, 2.0, 300))
    assert np.allclose(seeds.grad.cpu().numpy(), gs, rtol=1e-12, atol=0)
    assert np.allclose(align.grad.cpu().numpy(), ga, rtol=1e-9, atol=1e-9 * np.abs(ga).max())


def test_gradient_points_towards_the_true_misalignment(handle):
    """Fitting the misaligned detector with the nominal geometry: a few
    gradient-descent steps on the shifts along v (loc1) reduce the summed chi2."""
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["align20_100k"], 5000))
    S = ev["center"].shape[1]
    align = np.zeros((6, S))
    c0 = None
    for it in range(3):
        chi2, gs, ga = _grad(handle, ev, align)
        total = float(np.sum(chi2))
        if c0 is None:
            c0 = total
        # a Gauss-Newton-like diagonal step on the loc1 shifts only
        step = -ga[1] / np.maximum(np.abs(ga[1]).max(), 1e-30) * 0.02
        step[0] = 0.0
        align[1] += step
    assert total < c0


def test_full_size_gradients_sampled_and_additive(handle):
    """The bench's adjoint workload at full size (100k tracks x 21 states):
    seed gradients of 40 sampled tracks against the oracle's central
    differences on those tracks, chi2 against the oracle, and the alignment
    gradient of the batch equal to the sum of its two halves' (one sum over
    tracks, so it holds at any size)."""
    ev = synth.make_event(synth.WORKLOADS["align20_100k"], with_truth_states=False)
    T, S = int(ev["n_tracks"]), ev["center"].shape[1]
    align = np.zeros((6, S))
    chi2, gs, ga = _grad(handle, ev, align)
    pick = np.sort(np.random.default_rng(21).choice(T, 40, replace=False))
    sub = synth.subset(ev, pick)
    ref_chi2 = oracle.chi2_per_track(sub, align)
    assert np.max(np.abs(chi2[pick] - ref_chi2) / ref_chi2) < 1e-9
    fd = _fd2(oracle.chi2_gradient_fd, ev=sub, align=align)
    fl_s, _ = _floors(fd[0], fd[1], sub["seed_params"], ref_chi2)
    es = grad_err(gs[:, pick], fd[0][0], fl_s)
    assert es.max() < 1e-5, es.max()
    half = T // 2
    _, _, ga0 = _grad(handle, synth.subset(ev, np.arange(half)), align)
    _, _, ga1 = _grad(handle, synth.subset(ev, np.arange(half, T)), align)
    assert np.max(np.abs(ga - (ga0 + ga1))) <= 1e-10 * np.max(np.abs(ga))


# ---------------------------------------------------------------- the whole fit (filter + smoother)

def _smoother_weights(ev, seed=5):
    """Weights v [6][T] and W [21][T] that make every smoother term of L of
    order one: v_i ~ N(0, 1) / max(|x_i|, sigma_i), W_ij ~ N(0, 1) /
    (sigma_i sigma_j), from the oracle's smoothed state 0."""
    r = oracle.fit_batch(ev)
    T = int(ev["n_tracks"])
    rng = np.random.default_rng(seed)
    sd = np.sqrt(np.abs(r["cov"][DIAG]))
    v = rng.normal(size=(6, T)) / np.maximum(np.abs(r["params"]), sd)
    W = rng.normal(size=(21, T)) / np.stack([sd[i] * sd[j] for i, j in PAIRS])
    return v, W


def _whole(handle, ev, align, w=None, v=None, W=None, opt=None):
    import torch
    dev = kf.event_to_device(ev)
    T, S = int(ev["n_tracks"]), ev["center"].shape[1]
    d = lambda *shape: torch.empty(shape, dtype=torch.float64, device="cuda")
    cu = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    o = {"chi2": d(T), "params": d(6, T), "cov": d(21, T), "gs": d(6, T), "ga": d(6, S)}
    kf.kf_grad(handle, dev, align=cu(align), dl_dchi2=cu(w), dl_dparams=cu(v), dl_dcov=cu(W),
               out_chi2=o["chi2"], out_params=o["params"], out_cov=o["cov"], grad_seed=o["gs"],
               grad_align=o["ga"], opt=opt)
    torch.cuda.synchronize()
    return {k: t.cpu().numpy() for k, t in o.items()}


@pytest.mark.parametrize("terms,nonzero_align", [("all", False), ("all", True), ("params", False),
                                                 ("cov", False)])
def test_whole_fit_gradients_match_oracle_finite_differences(handle, terms, nonzero_align):
    """L = sum_t [w chi2 + v . x_s0 + W . C_s0]: all three terms, and the
    smoother terms alone (w = 0; then every derivative goes through the
    smoother's reverse)."""
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["align20_100k"], 100))
    S = ev["center"].shape[1]
    rng = np.random.default_rng(2)
    align = np.zeros((6, S))
    if nonzero_align:
        align[:3, 1:] = rng.normal(size=(3, S - 1)) * 0.05
        align[3:, 1:] = rng.normal(size=(3, S - 1)) * 5e-4
    v, W = _smoother_weights(ev)
    w = rng.uniform(0.5, 1.5, size=100)
    if terms == "params":
        w, W = np.zeros(100), None
    elif terms == "cov":
        w, v = np.zeros(100), None
    g = _whole(handle, ev, align, w, v, W)
    # the values: the smoothed state 0 and chi2 of the fit at this alignment
    ea = dict(ev)
    ea["center"], ea["rot"] = oracle.apply_alignment(ev["center"], ev["rot"], align)
    ref = oracle.fit_batch(ea)
    assert np.all(ref["status"] == 0)
    assert param_err(g["params"], ref["params"], ref["cov"]).max() < 1e-9
    assert cov_err(g["cov"], ref["cov"]).max() < 1e-9
    assert np.max(np.abs(g["chi2"] - ref["chi2"]) / ref["chi2"]) < 1e-9
    # the gradients, element by element
    fd = _fd2(oracle.objective_gradient_fd, ev=ev, align=align, weights=w, dl_dparams=v, dl_dcov=W)
    _, l_abs = oracle.objective_per_track(ev, align, weights=w, dl_dparams=v, dl_dcov=W)
    # the covariance depends on the seed and the alignment only through the
    # linearisation point (the Jacobians, the scattering at the predicted
    # momenta): a weak dependence that central differences resolve for a
    # minority of its elements
    fl_s, fl_a = _check_grads(g["gs"], g["ga"], fd[0], fd[1], ev["seed_params"], l_abs,
                              min_resolved=0.15 if terms == "cov" else 0.6)
    # the smoother terms carry real weight: they move some element of each
    # gradient by more than 100x that element's tolerance
    _, gs0, ga0 = _grad(handle, ev, align, w)
    fs, fa = fd[0]
    assert np.max(np.abs(g["gs"] - gs0) / (1e-5 * np.maximum(np.abs(fs), fl_s))) > 100
    assert np.max(np.abs(g["ga"] - ga0) / (1e-5 * np.maximum(np.abs(fa), fl_a))) > 100


def test_whole_fit_autograd_and_chunked_launches(handle):
    """fit_autograd's values equal the FP64 fit's outputs (within the FP64
    contract: the adjoint kernel's smoother inverts explicitly), its backward
    equals kf_grad with the same weights, and a workspace cap that splits the
    batch into several launches changes nothing."""
    import torch
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["align20_100k"], 300))
    dev = kf.event_to_device(ev)
    S = ev["center"].shape[1]
    out = kf.alloc_outputs(300)
    kf.kf_fit_ex(handle, dev, out, kf.kf_default_options(kf.KF_PRECISION_FP64))
    seeds = dev["seed_params"].clone().requires_grad_(True)
    align = torch.zeros((6, S), dtype=torch.float64, device="cuda", requires_grad=True)
    chi2, params, cov = kf.fit_autograd(seeds, align, dev, handle)
    torch.cuda.synchronize()
    f = {k: out[k].cpu().numpy() for k in ("params", "cov", "chi2")}
    assert param_err(params.detach().cpu().numpy(), f["params"], f["cov"]).max() < 1e-9
    assert cov_err(cov.detach().cpu().numpy(), f["cov"]).max() < 1e-9
    assert np.max(np.abs(chi2.detach().cpu().numpy() - f["chi2"]) / f["chi2"]) < 1e-9
    v, W = _smoother_weights(ev)
    w = np.linspace(0.5, 2.0, 300)
    tw = lambda a: torch.from_numpy(a).cuda()
    loss = (chi2 * tw(w)).sum() + (params * tw(v)).sum() + (cov * tw(W)).sum()
    loss.backward()
    g = _whole(handle, ev, np.zeros((6, S)), w, v, W)
    assert np.allclose(seeds.grad.cpu().numpy(), g["gs"], rtol=1e-12, atol=0)
    assert np.allclose(align.grad.cpu().numpy(), g["ga"], rtol=1e-9, atol=1e-9 * np.abs(g["ga"]).max())
    # 300 tracks through a workspace that holds 64 of them: five launches
    # (one thread per track; the pipelined form adds two hand-off slots of
    # kSlot doubles to each track's scratch)
    per_track = 8 * (27 * 5 + 27 * 6 + 79 * 21)
    opt = kf.kf_default_options(kf.KF_PRECISION_FP64, block=0, team_warps=1, workspace_bytes=64 * per_track)
    gc = _whole(handle, ev, np.zeros((6, S)), w, v, W, opt=opt)
    # the surface packing, the alignment angles' cosines and sines, 5 chunks
    assert handle.last_launch_count() == 1 + 1 + 5
    g1 = _whole(handle, ev, np.zeros((6, S)), w, v, W, opt=kf.kf_default_options(block=0, team_warps=1))
    for k in ("chi2", "params", "cov", "gs"):
        assert np.array_equal(gc[k], g1[k]), k
        assert np.array_equal(g1[k], g[k]), k   # the default here is the pipelined form
    assert np.allclose(gc["ga"], g["ga"], rtol=1e-11, atol=1e-11 * np.abs(g["ga"]).max())


def test_full_size_whole_fit_gradients_sampled(handle):
    """The bench's workload at full size (100k tracks x 21 states) through
    the whole-fit adjoint: values and seed gradients of 40 sampled tracks
    against the oracle (central differences of those tracks), and the
    alignment gradient of the batch equal to the sum of its two halves'."""
    ev = synth.make_event(synth.WORKLOADS["align20_100k"], with_truth_states=False)
    T, S = int(ev["n_tracks"]), ev["center"].shape[1]
    v, W = _smoother_weights(ev)
    g = _whole(handle, ev, np.zeros((6, S)), None, v, W)
    pick = np.sort(np.random.default_rng(22).choice(T, 40, replace=False))
    sub = synth.subset(ev, pick)
    ref = oracle.fit_batch(sub)
    assert param_err(g["params"][:, pick], ref["params"], ref["cov"]).max() < 1e-9
    assert cov_err(g["cov"][:, pick], ref["cov"]).max() < 1e-9
    fd = _fd2(oracle.objective_gradient_fd, ev=sub, dl_dparams=v[:, pick], dl_dcov=W[:, pick])
    _, l_abs = oracle.objective_per_track(sub, dl_dparams=v[:, pick], dl_dcov=W[:, pick])
    fl_s, _ = _floors(fd[0], fd[1], sub["seed_params"], l_abs)
    es = grad_err(g["gs"][:, pick], fd[0][0], fl_s)
    assert es.max() < 1e-5, es.max()
    half = T // 2
    g0 = _whole(handle, synth.subset(ev, np.arange(half)), np.zeros((6, S)), None, v[:, :half], W[:, :half])
    g1 = _whole(handle, synth.subset(ev, np.arange(half, T)), np.zeros((6, S)), None, v[:, half:], W[:, half:])
    assert np.max(np.abs(g["ga"] - (g0["ga"] + g1["ga"]))) <= 1e-10 * np.max(np.abs(g["ga"]))


def test_whole_fit_gradients_uneven_tracks_with_holes(handle):
    """Tracks of 1 to 30 states with holes (segment boundaries at every
    place, warps whose tracks have different segment counts, holes on the
    reference-plane side and at the last state): the whole-fit objective's
    values and gradients against the oracle, element by element."""
    ev = dict(synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 96)))
    # a few very short tracks: 1, 2 and 3 states (cut from the first three)
    o = ev["offsets"].astype(np.int64)
    keep = []
    lengths = []
    for t in range(96):
        n = int(o[t + 1] - o[t])
        L = {0: 1, 1: 2, 2: 3}.get(t, n)
        keep.append(np.arange(o[t], o[t] + L))
        lengths.append(L)
    idx = np.concatenate(keep)
    ev["offsets"] = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
    for k in ("loc", "cov", "truth_states"):
        if ev.get(k) is not None:
            ev[k] = np.ascontiguousarray(ev[k][:, idx])
    for k in ("surface_id", "is_hole"):
        ev[k] = np.ascontiguousarray(ev[k][idx]).copy()
    ev["is_hole"][ev["offsets"][5 + 1] - 1] = 1      # a track ending on a hole
    v, W = _smoother_weights(ev)
    w = np.random.default_rng(4).uniform(0.5, 1.5, size=96)
    S = ev["center"].shape[1]
    g = _whole(handle, ev, np.zeros((6, S)), w, v, W)
    ref = oracle.fit_batch(ev)
    assert np.all(ref["status"] == 0)
    assert param_err(g["params"], ref["params"], ref["cov"]).max() < 1e-9
    assert cov_err(g["cov"], ref["cov"]).max() < 1e-9
    fd = _fd2(oracle.objective_gradient_fd, ev=ev, weights=w, dl_dparams=v, dl_dcov=W)
    _, l_abs = oracle.objective_per_track(ev, weights=w, dl_dparams=v, dl_dcov=W)
    _check_grads(g["gs"], g["ga"], fd[0], fd[1], ev["seed_params"], l_abs)


@pytest.mark.parametrize("objective", ["chi2", "whole"])
def test_pipelined_adjoint_equals_sequential(handle, objective):
    """team_warps = 2 runs the filter's reverse on two warps per 32 tracks
    (the forward half one transition ahead on one, the reverse half on the
    other) and the smoother's passes likewise (each segment recomputed one
    segment ahead of its RTS steps; with the chi2 objective the smoothed
    outputs alone, with the whole one their reverse as well): the same
    arithmetic, so the same chi2, smoothed outputs and seed
    gradients bit for bit, and the alignment gradient up to the order of its
    atomic sums; on uneven tracks with holes, zero and non-zero alignment."""
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 333))
    S = ev["center"].shape[1]
    v, W = _smoother_weights(ev) if objective == "whole" else (None, None)
    rng = np.random.default_rng(6)
    for nonzero in (False, True):
        align = np.zeros((6, S))
        if nonzero:
            align[:3, 1:] = rng.normal(size=(3, S - 1)) * 0.05
            align[3:, 1:] = rng.normal(size=(3, S - 1)) * 5e-4
        seq = _whole(handle, ev, align, None, v, W, opt=kf.kf_default_options(block=0, team_warps=1))
        pip = _whole(handle, ev, align, None, v, W, opt=kf.kf_default_options(block=0, team_warps=2))
        assert handle.last_launch_count() == 3  # packing, alignment trig, the adjoint
        for k in ("chi2", "params", "cov", "gs"):
            assert np.array_equal(seq[k], pip[k]), k
        assert np.allclose(pip["ga"], seq["ga"], rtol=1e-12, atol=1e-12 * np.abs(seq["ga"]).max())
    with pytest.raises(kf.KfError, match="-4"):
        _whole(handle, ev, align, None, v, W, opt=kf.kf_default_options(block=0, team_warps=4))
