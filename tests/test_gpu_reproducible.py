"""Bitwise reproducibility of whole simulations: the benchmark's 64-event
batch run twice on one handle and once on a second handle gives the same
pixel maps, step counts, retire steps, collection points and interaction
counts bit for bit.  Every field sum has a fixed order: the symmetric kernel
adds each tile's partial fields in list order, the per-pair kernel adds a
split tile's pieces in piece order, and the counters are integers.  (The
induced-charge records, not used here, add per-warp FP64 sums atomically in
arbitrary order and may differ in their last bits.)"""
import numpy as np
import pytest

import paper_2506_09712_gb300 as cts
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09712_gb300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(sim, evs):
    res = sim.run(evs, keep_xy_capacity=5525)
    return {r["event_id"]: r for r in res}


def _same(a, b):
    assert a.keys() == b.keys()
    for eid in a:
        x, y = a[eid], b[eid]
        assert x["status"] == y["status"] == 0
        assert x["n_steps"] == y["n_steps"]
        assert x["interactions"] == y["interactions"]
        assert np.array_equal(x["pixels"], y["pixels"])
        assert np.array_equal(x["retire_step"], y["retire_step"])
        # identical bits, NaN (never collected) in the same places
        assert np.array_equal(x["final_xy"].view(np.int64), y["final_xy"].view(np.int64))


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_batch_is_bitwise_reproducible(variant):
    # variant 0: the default (symmetric kernel while many events run, the
    # per-pair kernel for the last few); 1: symmetric only; 2: per-pair only
    name = "batch_20keV_320um"
    p = W.preset(name)
    evs = W.make_events(name)
    opts = dict(max_slots=64, keep_final_xy=1, variant=variant)
    with cts.Simulator(p["sensor"], p["mobility"], **opts) as sim:
        first = _run(sim, evs)
        again = _run(sim, evs)
    with cts.Simulator(p["sensor"], p["mobility"], **opts) as sim:
        other = _run(sim, evs)
    _same(first, again)
    _same(first, other)
