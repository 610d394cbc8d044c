"""Per-pixel transient signals (Shockley-Ramo with pixel weighting potentials,
the extension the paper names in Sec. 5.3) on the GPU, through the C ABI,
against the FP64 oracle.

Tolerances: the device evaluates the weighting potentials in FP32 (about
3e-7 absolute per evaluation) with a truncated image series (below 2e-7 over
the pixel grid), and its trajectories follow the oracle's to FP32 rounding of
the fields; the signals telescope, so their end values carry only the start
and end evaluations.  Waveforms: within 1e-3 of the carrier count per step;
end values: within 2e-3 once the pixel counts' own difference is allowed for.
"""
import numpy as np
import pytest

import oracle
import paper_2506_09712_gb300 as cts
import workloads as W

pytestmark = pytest.mark.gpu

BOTH_FLAGS = cts.SIM_INDUCED_TOTAL | cts.SIM_INDUCED_PIXELS


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09712_gb300 import build
    build.build()
    oracle.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _window(pixels, g):
    c = g // 2
    return pixels[c - 1:c + 2, c - 1:c + 2].astype(np.float64)


def _check_against_oracle(got, refs, g):
    for d, r in zip(got, refs):
        q, qr = d["induced_px"], r.induced_px
        assert q.shape == (d["n_steps"], 3, 3)
        m = min(len(q), len(qr))
        assert m >= len(q) - 1
        assert np.abs(q[:m] - qr[:m]).max() <= 1e-3 * d["n_carriers"]
        # end values: count - sum of start potentials on both sides
        dc = _window(d["pixels"], g) - _window(r.pixels, g)
        assert np.abs(q[-1] - (qr[-1] + dc)).max() <= 2e-3


@pytest.mark.parametrize("mode", [cts.CTS_MODE_BATCHED, cts.CTS_MODE_PLAIN])
def test_pixel_signals_match_the_oracle(mode):
    name = "plain_3keV_100um"
    p = W.preset(name)
    evs = W.make_events(name, n=4, first_id=120)
    refs = oracle.run_events(oracle.make_params(p["sensor"], W.field_switches(), p["mobility"]),
                             evs, induced_px=True)
    with cts.Simulator(p["sensor"], p["mobility"], mode=mode, keep_induced=BOTH_FLAGS) as sim:
        got = sim.run(evs, induced_capacity=4096)
    _check_against_oracle(got, refs, p["sensor"]["grid_n"])
    # the whole-surface signal of the same runs still ends at sum(z0) / H
    for d, r in zip(got, refs):
        assert d["induced"][-1] == pytest.approx(r.induced[-1], rel=1e-9)


def test_pixel_recording_leaves_the_transport_unchanged():
    name = "plain_3keV_100um"
    p = W.preset(name)
    evs = W.make_events(name, n=4, first_id=130)
    outs = []
    for flags in (0, cts.SIM_INDUCED_TOTAL, cts.SIM_INDUCED_PIXELS, BOTH_FLAGS):
        with cts.Simulator(p["sensor"], p["mobility"], keep_induced=flags) as sim:
            outs.append(sim.run(evs, induced_capacity=4096))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert a["n_steps"] == b["n_steps"]
            assert np.array_equal(a["pixels"], b["pixels"])
    for a, b in zip(outs[1], outs[3]):
        assert np.allclose(a["induced"], b["induced"], rtol=1e-12, atol=1e-12)
    for a, b in zip(outs[2], outs[3]):
        assert np.allclose(a["induced_px"], b["induced_px"], rtol=1e-12, atol=1e-12)
    assert outs[1][0]["induced_px"] is None and outs[2][0]["induced"] is not None


def test_spherical_model_pixel_signals_match_the_oracle():
    name = "plain_3keV_100um"
    p = W.preset(name)
    sph = W.field_switches(spherical=1)
    evs = W.make_events(name, n=3, first_id=140)
    refs = oracle.run_events(oracle.make_params(p["sensor"], sph, p["mobility"]), evs,
                             induced_px=True)
    with cts.Simulator(p["sensor"], p["mobility"], sph, keep_induced=BOTH_FLAGS) as sim:
        got = sim.run(evs, induced_capacity=4096)
    _check_against_oracle(got, refs, p["sensor"]["grid_n"])


def test_two_species_pixel_signals_end_at_the_pixel_counts():
    # holes and electrons from the same points: the start potentials cancel
    # bit for bit (the same FP32 evaluation), holes end with potential 1 on
    # their readout pixel and electrons 0 on the back surface, so every
    # pixel's signal ends at its count
    pr = W.preset("track_200keV_320um")
    sensor = dict(pr["sensor"], thickness_um=50.0, bias_V=50.0, depletion_V=20.0, dt_ps=5.0,
                  grid_n=9)
    rng = np.random.default_rng(21)
    evs = []
    for e in range(3):
        xyz = np.column_stack([rng.normal(4.0, 6.0, 200), rng.normal(-3.0, 6.0, 200),
                               rng.uniform(25.0, 48.0, 200)])
        sign = np.concatenate([np.ones(200), -np.ones(200)]).astype(np.int8)
        evs.append(W.explicit_event(np.concatenate([xyz, xyz]), sign, event_id=300 + e))
    with cts.Simulator(sensor, pr["mobility"], keep_induced=BOTH_FLAGS) as sim:
        got = sim.run(evs, induced_capacity=8192)
    for d in got:
        assert d["status"] == 0 and d["n_lost"] == 0
        win = _window(d["pixels"], 9)
        assert win.sum() > 150
        assert np.abs(d["induced_px"][-1] - win).max() < 1e-6
        assert d["induced"][-1] == pytest.approx(200.0, abs=1e-6)
