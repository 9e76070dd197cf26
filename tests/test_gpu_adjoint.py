"""The adjoint kernel (kf_chi2_grad): gradients of the summed chi2 with
respect to the seed parameters and the per-surface alignment, against
central finite differences of the CPU oracle (step 1e-6) on 100 tracks of a
misaligned telescope, plus the chi2 itself against the fit and the
torch.autograd wrapper."""
import numpy as np
import pytest

import oracle
import paper_2105_01796_gb300 as kf
from paper_2105_01796_gb300 import synth
from tests.metrics import fd_floor, grad_err, seed_steps

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


def _check_grads(gs, ga, fs, fa, seeds, l_track):
    """Element-wise against the oracle's central differences, each element
    to 1e-5 relative with the finite-difference floor (tests/metrics.py):
    seeds per track from that track's |L|, alignment from the batch's."""
    es = grad_err(gs, fs, fd_floor(l_track[None, :], seed_steps(seeds)))
    ea = grad_err(ga, fa, fd_floor(np.sum(np.abs(l_track)), 1e-6))
    assert es.max() < 1e-5, ("seed", es.max(), np.unravel_index(es.argmax(), es.shape))
    assert ea.max() < 1e-5, ("align", ea.max(), np.unravel_index(ea.argmax(), ea.shape))
    return es.max(), ea.max()


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
    fs, fa = oracle.chi2_gradient_fd(ev, align, weights=w)
    # every element, the reference plane's alignment (which moves the seed's
    # frame) included
    _check_grads(gs, ga, fs, fa, ev["seed_params"], w * ref_chi2)


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
    fs, _ = oracle.chi2_gradient_fd(sub, align)
    es = grad_err(gs[:, pick], fs, fd_floor(ref_chi2[None, :], seed_steps(sub["seed_params"])))
    assert es.max() < 1e-5, es.max()
    half = T // 2
    _, _, ga0 = _grad(handle, synth.subset(ev, np.arange(half)), align)
    _, _, ga1 = _grad(handle, synth.subset(ev, np.arange(half, T)), align)
    assert np.max(np.abs(ga - (ga0 + ga1))) <= 1e-10 * np.max(np.abs(ga))
