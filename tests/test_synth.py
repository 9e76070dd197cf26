"""The seeded input generator: every draw is keyed by (seed, track, attempt,
purpose), so a batch simulated in parallel ranges equals the same batch
simulated in one process, bit for bit, and any track is reproducible alone."""
import numpy as np
import pytest

from paper_2105_01796_gb300 import synth


@pytest.mark.parametrize("name", ["uneven30_1m", "fringe30_100k"])
def test_parallel_generation_equals_serial(name):
    w = synth.scaled(synth.WORKLOADS[name], 901)
    a = synth.make_event(w, workers=1)
    b = synth.make_event(w, workers=3)
    for k, v in a.items():
        if isinstance(v, np.ndarray):
            assert np.array_equal(v, b[k]), k
    assert a["rejected"] == b["rejected"]


def test_track_is_reproducible_alone_and_truth_states_optional():
    w = synth.scaled(synth.WORKLOADS["uneven30_1m"], 400)
    ev = synth.make_event(w)
    lean = synth.make_event(w, with_truth_states=False)
    assert lean["truth_states"] is None
    for k in ("loc", "cov", "surface_id", "is_hole", "seed_params", "offsets"):
        assert np.array_equal(ev[k], lean[k]), k
    # the first 100 tracks of a smaller batch are the same tracks
    small = synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 100))
    sub = synth.subset(ev, np.arange(100))
    for k in ("loc", "cov", "surface_id", "is_hole", "seed_params", "truth_states", "offsets"):
        assert np.array_equal(sub[k], small[k]), k
