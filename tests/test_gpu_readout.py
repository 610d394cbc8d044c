"""GPU readout (Sec. 4.1 cluster selection, Sec. 4.2 noise) against the
oracle: the same count maps and random streams give the same clusters, veto
and window decisions and the same single-pixel spectrum."""
import numpy as np
import pytest

import oracle
import paper_2506_09712_gb300 as cts
import workloads as W

pytestmark = pytest.mark.gpu


def _compare(counts, seeds, ids, beam, n_bins=300, **kw):
    g = cts.sim_readout(counts, seeds, ids, beam, n_bins, want_pixels=True, **kw)
    o = oracle.readout(counts, seeds, ids, beam, n_bins, **kw)
    assert np.array_equal(g["cx"], o["cx"]) and np.array_equal(g["cy"], o["cy"])
    assert np.array_equal(g["vetoed"], o["vetoed"])
    assert np.array_equal(g["accepted"], o["accepted"])
    np.testing.assert_allclose(g["e"], o["e"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(g["e_cluster"], o["e_cluster"], rtol=0, atol=1e-11)
    assert np.array_equal(np.isnan(g["cluster"]), np.isnan(o["cluster"]))
    np.testing.assert_allclose(np.nan_to_num(g["cluster"]), np.nan_to_num(o["cluster"]),
                               rtol=0, atol=1e-12)
    assert np.array_equal(g["spectrum"], o["spectrum"])
    return g


def _cloud_maps(n_ev, g, rng, n_pairs=5525, spread=12.0):
    # charge clouds of random width and position binned into 25 um pixels
    maps = np.zeros((n_ev, g, g), np.int32)
    for k in range(n_ev):
        c = rng.uniform(-12.5, 12.5, 2)
        s = rng.uniform(0.5, spread)
        xy = c + s * rng.standard_normal((n_pairs, 2))
        ij = np.floor(xy / 25.0 + g / 2).astype(int)
        ok = (ij >= 0).all(1) & (ij < g).all(1)
        np.add.at(maps[k], (ij[ok, 1], ij[ok, 0]), 1)
    return maps


@pytest.mark.parametrize("noise", [0.13, 0.0])
def test_readout_matches_the_oracle_on_cloud_maps(noise):
    rng = np.random.default_rng(5)
    maps = _cloud_maps(300, 9, rng)
    seeds = np.full(300, 20250611, np.uint64)
    g = _compare(maps, seeds, np.arange(300), 20.0, noise_keV=noise)
    assert 0 < g["accepted"].sum() < 300        # the window and veto both act


def test_readout_edge_cases():
    rng = np.random.default_rng(9)
    # hand-built maps: ties, corner centre, annulus veto, far pixel
    m = np.zeros((5, 9, 9), np.int32)
    m[0, 2, 6] = m[0, 6, 2] = m[0, 2, 5] = 100
    m[1, 0, 0] = 3000
    m[1, 0, 1] = 10
    m[2, 4, 4] = 5000
    m[2, 4, 6] = 5
    m[3, 4, 4] = 5000
    m[3, 4, 8] = 5
    _compare(m, np.ones(5, np.uint64), np.arange(5), 18.1, noise_keV=0.0)
    # a 1 x 1 grid, and the largest grid (32 x 32) with noise
    _compare(np.full((3, 1, 1), 2000, np.int32), [1, 2, 3], [0, 0, 0], 7.24, noise_keV=0.13)
    _compare(_cloud_maps(20, 32, rng), np.arange(20), np.arange(20), 20.0, noise_keV=0.13)
    # no events
    r = cts.sim_readout(np.zeros((0, 9, 9), np.int32), [], [], 20.0, 10)
    assert r["spectrum"].sum() == 0


def test_readout_of_simulated_events_with_fano_counts():
    # the serving mix with Fano-distributed pair counts, simulated on the GPU;
    # its pixel maps read out on the GPU and by the oracle agree
    name = "serve_mix_320um"
    p = W.preset(name)
    evs = W.make_events(name, n=40, first_id=300)
    for e in evs:
        e["n_pairs"] = cts.cts_fano_pairs(e["seed"], e["event_id"], e["energy_keV"], 0.13)
    with cts.Simulator(p["sensor"], p["mobility"]) as sim:
        res = sim.run(evs)
    assert all(r["status"] == 0 for r in res)
    assert [r["n_carriers"] for r in res] == [e["n_pairs"] for e in evs]
    maps = np.stack([r["pixels"].reshape(9, 9) for r in res])
    for beam in (8.0, 17.5, 25.0):
        _compare(maps, [e["seed"] for e in evs], [e["event_id"] for e in evs], beam)
