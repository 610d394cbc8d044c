"""Pins of the oracle's detector readout (Sec. 4.1 selection, Sec. 4.2 Fano
factor and noise): hand-built pixel maps whose cluster, veto and window
outcome is fixed by construction, and the statistics of the random draws."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle

W = 3.62e-3  # keV per pair


def _map(cells, g=9):
    c = np.zeros((1, g, g), np.int32)
    for (ix, iy), v in cells.items():
        c[0, iy, ix] = v
    return c


def _ro(c, beam, **kw):
    kw.setdefault("noise_keV", 0.0)
    return oracle.readout(c, [7], [3], beam, 300, **kw)


def test_fano_zero_is_the_plain_pair_count():
    for e in (3.0, 8.0, 17.5, 20.0, 25.0):
        for ev in range(5):
            assert oracle.fano_pairs(11, ev, e, 0.0) == oracle.n_pairs(e)


def test_fano_mean_and_variance():
    # N has mean E / w and variance F E / w (normal approximation)
    e, f, n = 20.0, 0.13, 20000
    mean = e / W
    x = np.array([oracle.fano_pairs(20250611, k, e, f) for k in range(n)], float)
    se = math.sqrt(f * mean / n)
    assert abs(x.mean() - mean) < 4 * se
    # the sample variance of n normals has relative sd sqrt(2 / n) = 1 %
    assert x.var() == pytest.approx(f * mean, rel=0.05)
    # a different Fano factor scales the spread by its square root
    y = np.array([oracle.fano_pairs(20250611, k, e, 4 * f) for k in range(4000)], float)
    assert y.std() / x.std() == pytest.approx(2.0, rel=0.06)


def test_single_pixel_event_is_one_full_cluster():
    n = 5525
    r = _ro(_map({(4, 4): n}), beam=20.0)
    assert (r["cx"][0], r["cy"][0]) == (4, 4)
    assert r["e_cluster"][0] == pytest.approx(n * W, rel=1e-12)
    assert r["cluster"][0][4] == pytest.approx(n * W, rel=1e-12)
    assert np.count_nonzero(r["cluster"][0]) == 1
    assert r["accepted"][0] == 1 and r["vetoed"][0] == 0


def test_shared_charge_stays_in_the_cluster_around_the_largest_pixel():
    cells = {(4, 4): 2000, (5, 4): 1500, (4, 5): 1000, (5, 5): 1025}
    r = _ro(_map(cells), beam=20.0)
    assert (r["cx"][0], r["cy"][0]) == (4, 4)
    assert r["e_cluster"][0] == pytest.approx(5525 * W, rel=1e-12)
    # row-major 3 x 3 around (4, 4): (5, 4) is the centre row's right cell
    assert r["cluster"][0][5] == pytest.approx(1500 * W)
    assert r["cluster"][0][8] == pytest.approx(1025 * W)


def test_pileup_veto_annulus():
    # distance 2 or 3 from the centre (outside 3 x 3, inside 7 x 7): vetoed
    for pos in [(6, 4), (4, 1), (7, 7), (1, 2)]:
        r = _ro(_map({(4, 4): 5000, pos: 5}), beam=18.1)
        assert r["vetoed"][0] == 1 and r["accepted"][0] == 0, pos
    # distance 4: neither in the cluster nor in the veto region
    r = _ro(_map({(4, 4): 5000, (8, 4): 5}), beam=18.1)
    assert r["vetoed"][0] == 0 and r["accepted"][0] == 1
    assert r["e_cluster"][0] == pytest.approx(5000 * W)
    # with noise the threshold is veto_factor * noise: 2 pairs = 7.2 eV passes
    r = oracle.readout(_map({(4, 4): 5000, (6, 4): 2}), [7], [3], 18.1, 10,
                       noise_keV=1e-9, veto_factor=3.0)
    assert r["vetoed"][0] == 1
    # 400 pairs (1.45 keV) are 8 sigma above the 0.39 keV threshold
    r = oracle.readout(_map({(4, 4): 5000, (6, 4): 400}), [7], [3], 18.1, 10,
                       noise_keV=0.13, veto_factor=3.0)
    assert r["vetoed"][0] == 1


def test_energy_window_edges():
    n = 5525
    e = n * W
    assert _ro(_map({(4, 4): n}), beam=e + 0.999)["accepted"][0] == 1
    assert _ro(_map({(4, 4): n}), beam=e - 0.999)["accepted"][0] == 1
    assert _ro(_map({(4, 4): n}), beam=e + 1.001)["accepted"][0] == 0
    assert _ro(_map({(4, 4): n}), beam=e - 1.001)["accepted"][0] == 0
    assert _ro(_map({(4, 4): n}), beam=e + 0.5, window_keV=0.4)["accepted"][0] == 0


def test_ties_take_the_first_pixel_in_row_major_order():
    r = _ro(_map({(6, 2): 100, (2, 6): 100, (5, 2): 100}), beam=1.0)
    assert (r["cx"][0], r["cy"][0]) == (5, 2)


def test_corner_centre_clips_the_cluster():
    r = _ro(_map({(0, 0): 3000, (1, 0): 10}), beam=10.9)
    cl = r["cluster"][0]
    assert (r["cx"][0], r["cy"][0]) == (0, 0)
    assert np.isnan(cl[[0, 1, 2, 3, 6]]).all()
    assert cl[4] == pytest.approx(3000 * W) and cl[5] == pytest.approx(10 * W)
    assert r["e_cluster"][0] == pytest.approx(3010 * W)


def test_spectrum_counts_the_accepted_clusters_pixels():
    cells = {(4, 4): 2500, (5, 4): 2000, (4, 3): 1025}
    r = oracle.readout(_map(cells), [1], [0], 20.0, 300, noise_keV=0.0, spec_lo_keV=0.0,
                       spec_bin_keV=0.1)
    h = r["spectrum"]
    # 2500 pairs = 9.05 keV -> bin 90; 2000 -> 7.24 keV -> bin 72; 1025 -> 3.7105 -> 37;
    # the six empty cluster pixels sit at exactly 0 keV -> bin 0
    assert h[90] == 1 and h[72] == 1 and h[37] == 1 and h[0] == 6 and h.sum() == 9
    # a rejected event adds nothing
    r = oracle.readout(_map(cells), [1], [0], 30.0, 300, noise_keV=0.0)
    assert r["accepted"][0] == 0 and r["spectrum"].sum() == 0


def test_noise_is_normal_with_the_stated_width():
    sigma, n_ev = 0.13, 600
    c = np.zeros((n_ev, 9, 9), np.int32)
    r = oracle.readout(c, np.full(n_ev, 5), np.arange(n_ev), 0.0, 10, noise_keV=sigma)
    e = r["e"].reshape(n_ev, -1)
    x = e.ravel()
    assert abs(x.mean()) < 4 * sigma / math.sqrt(x.size)
    assert x.std() == pytest.approx(sigma, rel=0.02)
    assert stats.kstest(x / sigma, "norm").pvalue > 1e-3
    # pixels of an event and events are independent draws
    cc = np.corrcoef(e[:, 0], e[:, 1])[0, 1]
    assert abs(cc) < 4 / math.sqrt(n_ev)
    # the same (seed, event) reproduces the same map; another seed does not
    r2 = oracle.readout(c[:3], [5, 5, 5], [0, 1, 2], 0.0, 10, noise_keV=sigma)
    assert np.array_equal(r2["e"], r["e"][:3])
    r3 = oracle.readout(c[:1], [6], [0], 0.0, 10, noise_keV=sigma)
    assert not np.array_equal(r3["e"][0], r["e"][0])


def test_fano_count_is_continuous_as_the_factor_vanishes():
    # F -> 0 must reach the plain count round(E / w), not a value beside it
    for e in (3.0, 8.0, 17.5, 20.0, 25.0):
        for ev in range(3):
            assert oracle.fano_pairs(11, ev, e, 1e-12) == oracle.n_pairs(e)


def test_noise_alone_rarely_trips_the_3_sigma_veto():
    # 40 noise pixels of the 7 x 7 annulus, each above 3 sigma with
    # probability 0.00135: about 5 % of events are vetoed by noise alone
    # (a 1 sigma threshold would veto nearly all of them)
    n_ev, sigma = 400, 0.13
    c = np.zeros((n_ev, 9, 9), np.int32)
    c[:, 4, 4] = 5525
    r = oracle.readout(c, np.full(n_ev, 3), np.arange(n_ev), 20.0, 300, noise_keV=sigma,
                       veto_factor=3.0)
    assert (r["cx"] == 4).all() and (r["cy"] == 4).all()
    p = 1 - (1 - stats.norm.sf(3.0)) ** 40
    k = int(r["vetoed"].sum())
    assert abs(k - p * n_ev) < 5 * math.sqrt(n_ev * p * (1 - p)), (k, p * n_ev)
