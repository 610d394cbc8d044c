"""The stored oracle results of the uneven 5-25 keV / 450 um workload
(tests/golden/uneven_5_25keV_450um_oracle200.json, written by
make_uneven_oracle.py beside it) are the current oracle's: the file names the
oracle source it was made with, and the two shortest events, run again,
give the stored results exactly."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "uneven_5_25keV_450um_oracle200.json")
NAME = "uneven_5_25keV_450um"


def _load():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_golden_file_matches_the_oracle_source_and_workload():
    d = _load()
    with open(oracle._SRC, "rb") as fh:
        assert d["oracle_source_sha256_16"] == hashlib.sha256(fh.read()).hexdigest()[:16], \
            "the oracle changed: rerun tests/golden/make_uneven_oracle.py"
    assert d["workload"] == NAME and d["master_seed"] == W.MASTER_SEED and d["events"] == 200
    evs = W.make_events(NAME, n=200)
    for e, r in zip(evs, d["results"]):
        assert r["event_id"] == e["event_id"]
        assert r["energy_keV"] == pytest.approx(e["energy_keV"], rel=1e-12)
        assert r["depth_um"] == pytest.approx(e["depth_um"], rel=1e-12)
        assert r["n_carriers"] == oracle.n_pairs(e["energy_keV"])
        pix = np.asarray(r["pixels"])
        assert pix.shape == (9, 9) and r["status"] == 0
        # every hole collected, in the grid or outside it
        assert pix.sum() + r["n_outside"] == r["n_collected"] == r["n_carriers"]


def test_golden_file_reproduces_for_its_shortest_events():
    oracle.build()
    d = _load()
    p = W.preset(NAME)
    params = oracle.make_params(p["sensor"], W.field_switches(), p["mobility"])
    evs = W.make_events(NAME, n=200)
    shortest = sorted(d["results"], key=lambda r: r["interactions"])[:2]
    evs = [dict(evs[r["event_id"]], depth_um=r["depth_um"], energy_keV=r["energy_keV"])
           for r in shortest]
    got = oracle.run_events(params, evs)
    for r, g in zip(shortest, got):
        assert g.n_steps == r["n_steps"] and g.interactions == r["interactions"]
        assert np.array_equal(g.pixels, np.asarray(r["pixels"]))
        assert g.n_outside == r["n_outside"] and g.n_collected == r["n_collected"]
