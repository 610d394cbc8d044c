"""The paper's printed results for configurations this library runs, compared
loosely (they depend on the paper's unprinted mobility parameters): Table 1's
absorption-weighted RMS with and without repulsion, and the GGD shape
parameters of Sec. 3.1.  Values and citations: tests/golden/paper_values.json."""
import json
import os

import numpy as np
import pytest

import paper_2506_09712_gb300 as cts
import workloads as W

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _sensor(depletion):
    s = W.preset("batch_20keV_320um")["sensor"]
    return dict(s, depletion_V=depletion, grid_n=17)


def _rms_at(sim, energy, depths, reps, first_id):
    evs = []
    for i, h in enumerate(depths):
        for r in range(reps):
            e = W.make_events("batch_20keV_320um", n=1, first_id=first_id + reps * i + r)[0]
            evs.append(dict(e, energy_keV=float(energy), depth_um=float(h),
                            n_pairs=int(round(energy * 1000 / 3.62))))
    res = sim.run(evs, keep_xy_capacity=int(round(energy * 1000 / 3.62)))
    out = []
    for i in range(len(depths)):
        d = []
        for r, e in zip(res[reps * i:reps * (i + 1)], evs[reps * i:reps * (i + 1)]):
            xy = r["final_xy"]
            d.append((xy[~np.isnan(xy[:, 0])] - [e["x_um"], e["y_um"]]).ravel())
        d = np.concatenate(d)
        out.append((np.sqrt((d ** 2).mean()), d))
    return out


def test_table1_absorption_weighted_rms():
    g = GOLD["table1_weighted_rms_um"]
    s = _sensor(g["sensor"]["depletion_V"])
    m = W.preset("batch_20keV_320um")["mobility"]
    H = s["thickness_um"]
    depths = np.linspace(5.0, H - 5.0, 16)
    ours = {}
    for rep in (0, 1):
        with cts.Simulator(s, m, W.field_switches(repulsion=rep), keep_final_xy=1) as sim:
            vals = []
            for k, e in enumerate(g["energies_keV"]):
                lam = W.attenuation_length_um(e)
                w = np.exp(-depths / lam)
                rms = np.array([v[0] for v in _rms_at(sim, e, depths, 3, 5000 + 100 * k)])
                vals.append(float((w * rms).sum() / w.sum()))
        ours[rep] = np.array(vals)
    paper_no, paper_yes = np.array(g["without_repulsion"]), np.array(g["with_repulsion"])
    # magnitudes within 10 % of the paper's (measured here: 5.69, 4.11, 4.07
    # and 6.19, 5.13, 5.34 um)
    assert np.all(np.abs(ours[0] / paper_no - 1) < 0.1), ours[0]
    assert np.all(np.abs(ours[1] / paper_yes - 1) < 0.1), ours[1]
    # repulsion widens the cloud, relatively more at higher energy
    gain = ours[1] / ours[0]
    assert np.all(gain > 1.02) and gain[2] > gain[0], gain
    # and by amounts close to the paper's (+9 %, +23 %, +30 %)
    assert np.all(np.abs((gain - 1) - (paper_yes / paper_no - 1)) < 0.06), gain


def test_ggd_shape_at_the_paper_depths():
    g = GOLD["ggd_beta_25keV_320um_150V"]
    s = _sensor(GOLD["table1_weighted_rms_um"]["sensor"]["depletion_V"])
    m = W.preset("batch_20keV_320um")["mobility"]
    with cts.Simulator(s, m, keep_final_xy=1) as sim:
        res = _rms_at(sim, 25.0, g["depths_um"], 10, 7000)
    betas = np.array([cts.cts_fit_ggd(d)[1] for _, d in res])
    # flat-topped clouds (beta > 2), flatter after a shorter drift, as printed
    assert np.all(betas > 2.0), betas
    assert betas[0] > betas[2], betas
    # measured here: 2.68, 2.47, 2.41 against the printed 2.63, 2.47, 2.40
    assert np.all(np.abs(betas - np.array(g["beta"])) < 0.12), betas
