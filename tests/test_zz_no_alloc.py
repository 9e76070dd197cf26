"""kf_fit_static: the fit without any device allocation.

Callers that cannot allocate device memory -- real-time loops that must
never wait on the CUDA allocator, hosts that give the library a fixed memory
budget and own all other device memory -- call kf_fit_static.  Its scratch space is one
fixed block of device memory per GPU that the library reserves for the life
of the process.  These tests check, through the C ABI, that its results
equal kf_fit_ex's bit for bit on two different batches fitted one after the
other (the second call must not be affected by what the first left in the
block), with the grid and the persistent schedule, and
that a batch too large for the block is refused with a clear error.

This file is collected last so that a run stopping at the first failure has
run every other test already; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import paper_2105_01796_gb300 as kf
from paper_2105_01796_gb300 import synth

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


def _host(out):
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


@pytest.mark.parametrize("schedule", [kf.KF_SCHEDULE_GRID, kf.KF_SCHEDULE_PERSISTENT])
@pytest.mark.parametrize("prec", [kf.KF_PRECISION_FP64, kf.KF_PRECISION_MIXED])
def test_static_block_matches_fit_ex_on_two_calls_in_a_row(handle, prec, schedule):
    """Both entry points run the same kernel on every track (one thread per
    track; how the batch is cut into launches does not enter a track's
    arithmetic), so their outputs are equal bit for bit."""
    import torch
    opt = kf.kf_default_options(prec, schedule=schedule)
    # 7000 x 31 states needs several launches through the fixed block in FP64
    # (about 3000 tracks per launch) and in mixed precision (about 5800)
    events = [synth.make_event(synth.scaled(synth.WORKLOADS["tel30_100k"], 7000)),
              synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 5000))]
    devs = [kf.event_to_device(ev) for ev in events]
    outs = []
    for ev, dev in zip(events, devs):           # two kf_fit_static calls back to back
        out = kf.alloc_outputs(ev["n_tracks"])
        kf.kf_fit_static(dev, out, opt)
        outs.append(out)
    torch.cuda.synchronize()
    for ev, dev, out in zip(events, devs, outs):
        ref = kf.alloc_outputs(ev["n_tracks"])
        kf.kf_fit_ex(handle, dev, ref, opt)
        torch.cuda.synchronize()
        a, r = _host(out), _host(ref)
        assert np.all(r["status"] == 0)
        for k in ("params", "cov", "chi2", "ndf", "status"):
            assert np.array_equal(a[k], r[k]), k


def test_static_block_refuses_batches_that_do_not_fit(handle):
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["tel10_1k"], 8))
    dev = kf.event_to_device(ev)
    dev["max_states"] = 200_000   # one track's records alone would exceed the block
    out = kf.alloc_outputs(8)
    with pytest.raises(kf.KfError, match="fixed device block"):
        kf.kf_fit_static(dev, out)
