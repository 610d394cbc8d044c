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
