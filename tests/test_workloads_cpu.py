"""The seeded synthetic workloads: deterministic in (seed, ids), absorption
depths from the truncated exponential of the stated attenuation law, entry
points uniform over the central pixel, Poisson arrivals at the stated rate."""
import numpy as np
import pytest
from scipy import stats

import workloads as W


def test_events_are_deterministic_and_seeded():
    a = W.make_events("batch_20keV_320um", n=8)
    b = W.make_events("batch_20keV_320um", n=8)
    assert a == b
    c = W.make_events("batch_20keV_320um", n=8, seed=W.MASTER_SEED + 1)
    assert a != c
    assert [e["event_id"] for e in W.make_events("batch_20keV_320um", n=3, first_id=40)] == [40, 41, 42]


@pytest.mark.parametrize("energy,H", [(8.0, 320.0), (20.0, 320.0), (5.0, 450.0)])
def test_depths_follow_the_truncated_exponential(energy, H):
    rng = np.random.default_rng(3)
    h = W.sample_depths(rng, np.full(20000, energy), H)
    lam = W.attenuation_length_um(energy)
    assert np.all((h >= 0) & (h < H))
    cdf = lambda x: (1 - np.exp(-x / lam)) / (1 - np.exp(-H / lam))
    assert stats.kstest(h, cdf).pvalue > 1e-3
    # the attenuation law of the synthetic workloads: 69.6 um at 8 keV, E^2.9
    assert W.attenuation_length_um(8.0) == pytest.approx(69.6)
    assert W.attenuation_length_um(16.0) / W.attenuation_length_um(8.0) == pytest.approx(2 ** 2.9)


def test_entry_points_cover_the_central_pixel():
    evs = W.make_events("uneven_5_25keV_450um", n=4000)
    x = np.array([e["x_um"] for e in evs])
    y = np.array([e["y_um"] for e in evs])
    assert np.all(np.abs(x) <= 12.5) and np.all(np.abs(y) <= 12.5)
    assert stats.kstest(x, stats.uniform(-12.5, 25.0).cdf).pvalue > 1e-3
    e = np.array([ev["energy_keV"] for ev in evs])
    assert e.min() >= 5.0 and e.max() <= 25.0
    assert stats.kstest(e, stats.uniform(5.0, 20.0).cdf).pvalue > 1e-3


def test_serving_mix_and_arrivals():
    evs = W.make_events("serve_mix_320um", n=6000)
    e = np.array([ev["energy_keV"] for ev in evs])
    for val, share in [(8.0, 0.6), (17.5, 0.3), (25.0, 0.1)]:
        assert (e == val).mean() == pytest.approx(share, abs=0.02)
    t = W.poisson_arrivals(2000.0, 20000, seed=1)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps >= 0)
    assert gaps.mean() == pytest.approx(1 / 2000.0, rel=0.03)
    assert stats.kstest(gaps * 2000.0, "expon").pvalue > 1e-3


def test_committed_json_configs_are_the_presets():
    # workloads/configs/*.json are written by `python -m workloads`; they must
    # stay in step with the presets they mirror
    import glob
    import os
    paths = sorted(glob.glob(os.path.join(W.CONFIG_DIR, "*.json")))
    assert {os.path.basename(p)[:-5] for p in paths} == set(W.PRESETS)
    for path in paths:
        name = os.path.basename(path)[:-5]
        cfg = W.load_config(path)
        assert cfg.pop("name") == name
        assert cfg == W.preset(name)
        a = W.make_events(path, n=5, first_id=3)
        b = W.make_events(name, n=5, first_id=3)
        assert a == b


def test_config_round_trip_and_edits(tmp_path):
    path = str(tmp_path / "w.json")
    W.save_config("plain_3keV_100um", path)
    cfg = W.load_config(path)
    cfg["sensor"]["thickness_um"] = 150.0
    cfg["energies"] = [[8.0, 1.0]]
    evs = W.make_events(cfg, n=20)
    assert all(e["energy_keV"] == 8.0 for e in evs)
    assert all(0.0 <= e["depth_um"] < 150.0 for e in evs)
    assert W.preset(cfg)["sensor"]["thickness_um"] == 150.0


@pytest.mark.parametrize("edit", ["drop_sensor_key", "two_recipes", "unknown_key",
                                  "track_without_pairs", "negative_events", "not_object"])
def test_bad_configs_are_rejected(tmp_path, edit):
    import json
    cfg = json.loads(json.dumps(W.preset("plain_3keV_100um")))
    if edit == "drop_sensor_key":
        del cfg["sensor"]["pitch_um"]
    elif edit == "two_recipes":
        cfg["energy_uniform"] = [5.0, 25.0]
    elif edit == "unknown_key":
        cfg["energy_keV"] = 20.0
    elif edit == "track_without_pairs":
        del cfg["energies"]
        cfg.update(track=True, track_len_um=10.0, theta_max_deg=0.0)
    elif edit == "negative_events":
        cfg["n_events"] = -1
    else:
        cfg = [cfg]
    path = tmp_path / "bad.json"
    path.write_text(json.dumps(cfg))
    with pytest.raises(ValueError):
        W.load_config(str(path))
