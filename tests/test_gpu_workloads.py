"""Workload-level GPU parity: the uneven 10^4-event batch (KS tests of the
cluster-size and single-pixel-spectrum distributions against the oracle), the
two-species electron-track events, and continuous batching in SERVE mode
(a result is the same alone and in a live mix)."""
import json
import math
import os
import threading
import time

import numpy as np
import pytest
from scipy import stats

import oracle
import paper_2506_09712_gb300 as cts
import workloads as W

pytestmark = pytest.mark.gpu

EV_PER_PAIR_KEV = 3.62e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09712_gb300 import build
    build.build()
    oracle.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _params(name, field=None, **over):
    p = W.preset(name)
    return oracle.make_params(dict(p["sensor"], **over), field or W.field_switches(),
                              p["mobility"])


def cluster_size(pix):
    """Pixels of the grid holding at least 1 keV."""
    return int(np.count_nonzero(pix * EV_PER_PAIR_KEV >= 1.0))


def pixel_spectrum(pix):
    """Energies (keV) >= 1 keV of the 3x3 pixels around the maximum pixel."""
    iy, ix = np.unravel_index(int(np.argmax(pix)), pix.shape)
    win = pix[max(iy - 1, 0):iy + 2, max(ix - 1, 0):ix + 2].reshape(-1) * EV_PER_PAIR_KEV
    return win[win >= 1.0]


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "uneven_5_25keV_450um_oracle200.json")


@pytest.mark.slow
def test_uneven_batch_1e4_events_ks_against_oracle():
    # 10^4 events of E ~ U(5, 25) keV in 450 um Si on the GPU against the FP64
    # oracle's first 200 events (tests/golden/, written by the committed
    # make_uneven_oracle.py): the shared 200 event by event, then the
    # cluster-size and single-pixel-spectrum distributions (Sec. 4.2) by
    # two-sample KS tests.
    name = "uneven_5_25keV_450um"
    p = W.preset(name)
    evs = W.make_events(name, n=10_000)
    with open(GOLDEN) as fh:
        refs = json.load(fh)["results"]
    n_ref = len(refs)
    assert n_ref == 200 and [r["event_id"] for r in refs] == list(range(200))
    # the oracle's events are the workload's 200-event list (its depths are
    # drawn for the list as a whole, so it is not a prefix of the 10^4 list);
    # the energies and depths the oracle ran are taken from the file (another
    # machine's numpy may round the drawn depths differently in the last bit)
    evs_ref = W.make_events(name, n=200)
    for e, r in zip(evs_ref, refs):
        assert e["depth_um"] == pytest.approx(r["depth_um"], rel=1e-12)
        e["depth_um"], e["energy_keV"] = r["depth_um"], r["energy_keV"]
    with cts.Simulator(p["sensor"], p["mobility"], max_slots=512) as sim:
        res = sim.run(evs)
        res_ref = sim.run(evs_ref)
    assert all(r["status"] == 0 for r in res + res_ref)
    # The shared events one by one.  They take up to ~3000 steps; forward
    # Euler is locally unstable for pairs closer than (2 mu k dt)^(1/3) ~
    # 0.05 um, so FP32 and FP64 trajectories part slowly and a few carriers
    # near pixel edges may land differently: every event stays within
    # 1e-2 N per pixel, at least 85 % within the 1e-3 N target (measured on
    # GB300: 184 of 200, the worst 1.7e-3 N), and the distributions are the
    # binding test (measured: KS p = 1.0 for the cluster sizes, 0.86 for the
    # spectrum).
    within, worst = 0, 0.0
    for g, r in zip(res_ref, refs):
        n = g["n_carriers"]
        assert n == r["n_carriers"]
        assert g["n_collected"] == r["n_collected"] == n
        assert abs(g["n_steps"] - r["n_steps"]) <= 2
        dmax = np.abs(g["pixels"] - np.asarray(r["pixels"])).max()
        worst = max(worst, dmax / n)
        assert dmax <= 1e-2 * n
        within += dmax <= 1e-3 * n
    frac = within / n_ref
    # distributions of the 10^4-event run against the oracle's 200 events
    cs_gpu = [cluster_size(r["pixels"]) for r in res]
    cs_ref = [cluster_size(np.asarray(r["pixels"])) for r in refs]
    sp_gpu = np.concatenate([pixel_spectrum(r["pixels"]) for r in res])
    sp_ref = np.concatenate([pixel_spectrum(np.asarray(r["pixels"])) for r in refs])
    p_cs = stats.ks_2samp(cs_gpu, cs_ref).pvalue
    p_sp = stats.ks_2samp(sp_gpu, sp_ref).pvalue
    print(f"\nuneven 1e4 vs oracle 200: {within}/{n_ref} events within 1e-3 N per pixel "
          f"(worst {worst:.2e} N); KS p cluster size {p_cs:.3g}, spectrum {p_sp:.3g}")
    assert frac >= 0.85
    assert p_cs > 0.01
    assert p_sp > 0.01
    # charge conservation over the whole run
    tot = sum(r["pixels"].sum() + r["n_outside"] for r in res)
    assert tot == sum(r["n_carriers"] for r in res)


def _track(n_pairs, k=0):
    e = W.make_events("track_200keV_320um", n=k + 1)[k]
    e["n_pairs"] = n_pairs
    return e


def test_track_event_two_species_parity():
    # a shortened 150 um track (1500 pairs = 3000 carriers): holes and electrons
    # with inter-species attraction, 5 ps steps, stopped when every hole is in
    name = "track_200keV_320um"
    p = W.preset(name)
    ev = _track(1500, k=3)
    ref = oracle.run_event(_params(name), ev)
    with cts.Simulator(p["sensor"], p["mobility"], keep_final_xy=1) as sim:
        g = sim.run([ev], keep_xy_capacity=3000)[0]
    assert g["status"] == 0 == ref.status
    assert g["n_carriers"] == 3000
    assert g["n_collected"] == ref.n_collected == 1500
    assert abs(g["n_steps"] - ref.n_steps) <= 1
    assert np.abs(g["pixels"] - ref.pixels).max() <= 3          # 1e-3 of 3000
    assert abs(g["n_lost"] - ref.n_lost) <= 3
    # collection points of the holes, carrier by carrier
    d = np.abs(g["final_xy"][:1500] - ref.final_xy[:1500])
    assert np.nanmax(d) < 0.05


def test_track_full_size_first_steps():
    # the largest event (2 x 55 250 carriers) for three steps, carrier by carrier
    name = "track_200keV_320um"
    p = W.preset(name)
    ev = _track(55_250, k=1)
    steps = 3
    ref = oracle.run_event(_params(name, max_steps=steps), ev)
    with cts.Simulator(p["sensor"], p["mobility"]) as sim:
        pos, st, done = sim.trajectory(dict(ev, n_carriers=110_500), steps)
    assert done == ref.n_steps == steps
    assert np.array_equal(st, ref.state)
    act = ref.state == oracle.ACTIVE
    d = np.abs(pos[act] - ref.pos[act]).max(axis=1)
    # FP32 displacements: ~1e-7 um per carrier; the few carriers of close
    # electron-hole pairs (r ~ 10 nm, fields ~1 V/um) inherit the FP32 rounding
    # of positions tens of um from the frame anchor and differ by up to ~1e-3 um
    assert np.median(d) < 1e-6
    assert np.quantile(d, 0.999) < 1e-4
    assert d.max() < 1e-2


def test_serving_results_same_alone_and_in_a_live_mix():
    # Requests arrive while others are on the GPU; SERVE admits them at chunk
    # boundaries.  Each result equals the same event run alone.
    name = "serve_mix_320um"
    p = W.preset(name)
    evs = W.make_events(name, n=24, first_id=500)
    with cts.Simulator(p["sensor"], p["mobility"]) as sim:
        alone = {r["event_id"]: r for r in (sim.run([e])[0] for e in evs[:6])}
    got = []
    with cts.Simulator(p["sensor"], p["mobility"], mode=cts.CTS_MODE_SERVE,
                       max_slots=8) as sim:
        def feeder():
            for e in evs:
                rc, _ = sim.submit([e])
                assert rc == 0
                time.sleep(0.01)
        th = threading.Thread(target=feeder)
        th.start()
        deadline = time.time() + 300
        while len(got) < len(evs) and time.time() < deadline:
            got += sim.poll(8, 100)
        th.join()
        st = sim.stats()
    assert len(got) == len(evs)
    assert st["chunks"] > 1 and st["events_done"] == len(evs)
    by_id = {r["event_id"]: r for r in got}
    for eid, a in alone.items():
        b = by_id[eid]
        assert b["status"] == 0
        assert abs(a["n_steps"] - b["n_steps"]) <= 1
        assert np.abs(a["pixels"] - b["pixels"]).max() <= int(1e-3 * a["n_carriers"])
    # continuous batching: events were admitted while others were running, and
    # slots freed by finished events were reused by later arrivals
    first_start = min(r["t_start_ns"] for r in got)
    first_done = min(r["t_done_ns"] for r in got)
    assert any(first_start < r["t_start_ns"] < first_done for r in got)
    assert any(r["t_start_ns"] > first_done for r in got)


def _mip_rms(res, evs):
    """Per-axis RMS of the collected positions about each track's entry point,
    pooled over the events."""
    d = []
    for r, e in zip(res, evs):
        xy = r["final_xy"]
        xy = xy[~np.isnan(xy[:, 0])] - [e["x_um"], e["y_um"]]
        d.append(xy)
    d = np.concatenate(d)
    return float(np.sqrt((d ** 2).mean(axis=0)).mean())


def test_mip_line_source():
    # Sec. 5.1: a minimum-ionising particle crossing 50 um perpendicularly,
    # 80 pairs/um, 1 nm wide.  The paper finds repulsion widens the collected
    # electron distribution by only 2.4 % (1.24 -> 1.27 um); its electron
    # mobility is not printed, so the checks here are the parity with the
    # oracle and the small size of the effect.
    name = "mip_50um"
    p = W.preset(name)
    evs = W.make_events(name)
    n = 2 * p["n_pairs"]
    out = {}
    for label, field, sensor in [("both", W.field_switches(), p["sensor"]),
                                 ("none", W.field_switches(repulsion=0), p["sensor"]),
                                 ("same", W.field_switches(), dict(p["sensor"], species=1))]:
        with cts.Simulator(sensor, p["mobility"], field, keep_final_xy=1) as sim:
            res = sim.run(evs, keep_xy_capacity=n)
        assert all(r["status"] == 0 and r["n_collected"] == p["n_pairs"] for r in res)
        out[label] = _mip_rms(res, evs)
        if label == "both":
            ref = oracle.run_event(oracle.make_params(sensor, field, p["mobility"]), evs[0])
            assert np.abs(res[0]["pixels"] - ref.pixels).max() <= math.floor(1e-3 * n)
            assert _mip_rms([res[0]], evs[:1]) == pytest.approx(
                _mip_rms([dict(final_xy=ref.final_xy)], evs[:1]), rel=2e-3)
    # about a micrometre of diffusion over the 50 um drift
    assert 0.8 < out["none"] < 1.6
    # with both species the attraction of the holes nearly cancels the
    # electrons' mutual repulsion: a change of a few per cent at most
    assert abs(out["both"] / out["none"] - 1) < 0.05
    # electrons alone repel each other visibly
    assert out["same"] / out["none"] > 1.04
