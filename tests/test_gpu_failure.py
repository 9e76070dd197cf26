"""Failure detection without a GPU fault: the kernels' bounded waits.

Every kernel stages the surface table into shared memory with one bulk copy
and waits on an mbarrier for at most a fixed number of polls.  The
diagnostic option test_wait_timeout announces the copy's bytes on the
barrier without issuing the copy, so the wait runs out with nothing left in
flight (a flag that nothing sets): no fault, no hang.  These tests check
that such a call reports the failure -- status KF_TRACK_TIMEOUT and NaN
results for every track, KF_EDEVICE from the synchronous host entry point,
NaN chi2 and seed gradients from the adjoint -- and that the next call on
the same handle, or through the static entry point, succeeds with results
equal to a fresh handle's."""
import numpy as np
import pytest

import paper_2105_01796_gb300 as kf
from paper_2105_01796_gb300 import synth

pytestmark = pytest.mark.gpu

TIMEOUT = 5


@pytest.fixture(scope="module")
def handle():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    h = kf.Handle()
    yield h
    h.close()


@pytest.fixture(scope="module")
def event():
    return synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 700))


def _host(out):
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def _assert_timed_out(o, n_states):
    assert np.all(o["status"] == TIMEOUT)
    assert np.all(np.isnan(o["params"])) and np.all(np.isnan(o["cov"])) and np.all(np.isnan(o["chi2"]))
    assert np.all(o["ndf"] == 0)
    if o.get("states") is not None:
        assert np.all(np.isnan(o["states"]))


@pytest.mark.parametrize("prec", [kf.KF_PRECISION_FP64, kf.KF_PRECISION_MIXED])
@pytest.mark.parametrize("schedule", [kf.KF_SCHEDULE_GRID, kf.KF_SCHEDULE_PERSISTENT, kf.KF_SCHEDULE_WAVES])
def test_timed_out_wait_marks_every_track_and_the_next_call_succeeds(handle, event, prec, schedule):
    import torch
    dev = kf.event_to_device(event)
    T, M = int(event["n_tracks"]), int(event["surface_id"].shape[0])
    bad = kf.alloc_outputs(T, M, with_states=True)
    kf.kf_fit_ex(handle, dev, bad, kf.kf_default_options(prec, schedule=schedule, block=64,
                                                         wait_limit=64, test_wait_timeout=1))
    torch.cuda.synchronize()
    _assert_timed_out(_host(bad), M)
    # the same handle, a normal call: the flag of the failed call is cleared
    out = kf.alloc_outputs(T, M, with_states=True)
    kf.kf_fit_ex(handle, dev, out, kf.kf_default_options(prec, schedule=schedule, block=64))
    h2 = kf.Handle()
    ref = kf.alloc_outputs(T, M, with_states=True)
    kf.kf_fit_ex(h2, dev, ref, kf.kf_default_options(prec, schedule=schedule, block=64))
    torch.cuda.synchronize()
    h2.close()
    a, r = _host(out), _host(ref)
    assert np.all(a["status"] == 0)
    for k in ("params", "cov", "chi2", "ndf", "status", "states"):
        assert np.array_equal(a[k], r[k]), k


@pytest.mark.parametrize("team", [2, 4])
def test_timed_out_wait_in_a_track_team(handle, event, team):
    import torch
    dev = kf.event_to_device(event)
    T, M = int(event["n_tracks"]), int(event["surface_id"].shape[0])
    bad = kf.alloc_outputs(T, M, with_states=True)
    kf.kf_fit_ex(handle, dev, bad, kf.kf_default_options(kf.KF_PRECISION_FP64, team_warps=team, wait_limit=64,
                                                         test_wait_timeout=1))
    torch.cuda.synchronize()
    _assert_timed_out(_host(bad), M)
    out = kf.alloc_outputs(T, M, with_states=True)
    kf.kf_fit_ex(handle, dev, out, kf.kf_default_options(kf.KF_PRECISION_FP64, team_warps=team))
    torch.cuda.synchronize()
    assert torch.all(out["status"] == 0)


def test_host_entry_reports_the_timeout_then_recovers(handle, event):
    T = int(event["n_tracks"])
    with pytest.raises(kf.KfError, match="kf error -5"):
        kf.kf_fit_host(handle, event, kf.kf_default_options(kf.KF_PRECISION_MIXED, wait_limit=64,
                                                            test_wait_timeout=1))
    out = kf.kf_fit_host(handle, event, kf.kf_default_options(kf.KF_PRECISION_MIXED))
    assert np.all(out["status"] == 0) and np.all(np.isfinite(out["params"]))
    assert out["params"].shape == (6, T)


def test_adjoint_reports_the_timeout_then_recovers(handle):
    import torch
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["align20_100k"], 100))
    dev = kf.event_to_device(ev)
    T, S = int(ev["n_tracks"]), ev["center"].shape[1]
    chi2 = torch.empty(T, dtype=torch.float64, device="cuda")
    gs = torch.empty((6, T), dtype=torch.float64, device="cuda")
    ga = torch.empty((6, S), dtype=torch.float64, device="cuda")
    kf.kf_chi2_grad(handle, dev, out_chi2=chi2, grad_seed=gs, grad_align=ga,
                    opt=kf.kf_default_options(block=0, wait_limit=64, test_wait_timeout=1))
    torch.cuda.synchronize()
    assert torch.all(torch.isnan(chi2)) and torch.all(torch.isnan(gs))
    assert torch.all(ga == 0)
    kf.kf_chi2_grad(handle, dev, out_chi2=chi2, grad_seed=gs, grad_align=ga)
    torch.cuda.synchronize()
    assert torch.all(torch.isfinite(chi2)) and torch.all(torch.isfinite(gs)) and torch.any(ga != 0)


def test_static_entry_reports_the_timeout_in_the_outputs(event):
    import torch
    dev = kf.event_to_device(event)
    T, M = int(event["n_tracks"]), int(event["surface_id"].shape[0])
    bad = kf.alloc_outputs(T, M, with_states=True)
    kf.kf_fit_static(dev, bad, kf.kf_default_options(kf.KF_PRECISION_FP64, wait_limit=64, test_wait_timeout=1))
    torch.cuda.synchronize()
    _assert_timed_out(_host(bad), M)
    out = kf.alloc_outputs(T, M)
    kf.kf_fit_static(dev, out, kf.kf_default_options(kf.KF_PRECISION_FP64))
    torch.cuda.synchronize()
    assert torch.all(out["status"] == 0)
