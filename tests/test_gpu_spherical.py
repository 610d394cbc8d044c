"""The simplified spherical model (Sec. 2.2, Eq. 7) on the GPU against the
oracle: trajectories carrier by carrier, whole events pixel by pixel, the
launch modes, the width of the cluster an event is split over, and the size
limit of the keys held in shared memory."""
import math

import numpy as np
import pytest

import oracle
import paper_2506_09712_gb300 as cts
import workloads as W

pytestmark = pytest.mark.gpu

SPH = W.field_switches(spherical=1)


def _sim(name, mode=cts.CTS_MODE_BATCHED, **opt):
    p = W.preset(name)
    return cts.Simulator(p["sensor"], p["mobility"], SPH, mode=mode, **opt)


def _params(name, **sensor_over):
    p = W.preset(name)
    return oracle.make_params(dict(p["sensor"], **sensor_over), SPH, p["mobility"])


@pytest.mark.parametrize("name,n,steps", [("plain_3keV_100um", 829, 40),
                                          ("batch_20keV_320um", 5525, 60)])
def test_spherical_trajectories_match_the_oracle(name, n, steps):
    ev = W.make_events(name, n=1, first_id=11)[0]
    ref = oracle.run_event(_params(name, max_steps=steps), ev)
    with _sim(name) as sim:
        pos, st, done = sim.trajectory(dict(ev, n_carriers=n), steps)
    assert done == ref.n_steps
    assert np.array_equal(st, ref.state)
    act = ref.state == oracle.ACTIVE
    d = np.abs(pos[act] - ref.pos[act]).max(axis=1)
    # FP32 displacements (drift + repulsion + diffusion, 0.3-0.5 um a step)
    # carry ~6e-8 relative rounding each step, ~1e-6 um after tens of steps;
    # the enclosed-charge field is smooth, so no carrier runs away
    assert np.median(d) < 5e-6, np.median(d)
    assert d.max() < 2e-4, d.max()


def _compare(gpu, ref, n):
    assert gpu["status"] == ref.status == 0
    assert gpu["n_collected"] == ref.n_collected
    assert abs(gpu["n_steps"] - ref.n_steps) <= 1
    assert np.abs(gpu["pixels"] - ref.pixels).max() <= math.floor(1e-3 * n)
    assert gpu["interactions"] == pytest.approx(ref.interactions, rel=2e-3)


def test_spherical_events_match_the_oracle():
    # a handle sized to the batch splits each event over a cluster of CTAs
    for name, k in (("plain_3keV_100um", 8), ("batch_20keV_320um", 3)):
        evs = W.make_events(name, n=k, first_id=40)
        refs = oracle.run_events(_params(name), evs)
        with _sim(name, max_slots=k) as sim:
            got = sim.run(evs)
            assert sim.stats()["sph_cluster"] > 1
        for g, r in zip(got, refs):
            _compare(g, r, g["n_carriers"])


def test_spherical_results_do_not_depend_on_the_cluster_width():
    # each event's holes split over 1, 2 or 4 CTAs: the centre's group sums
    # are added in a fixed order and the enclosed counts are exact, so the
    # results agree bit for bit
    name = "batch_20keV_320um"
    evs = W.make_events(name, n=5, first_id=90)
    outs = []
    for c in (1, 2, 4):
        with _sim(name, max_slots=len(evs), sph_cluster=c, keep_final_xy=1) as sim:
            outs.append(sim.run(evs, keep_xy_capacity=5525))
            assert sim.stats()["sph_cluster"] == c
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert a["status"] == b["status"] == 0
            assert a["n_steps"] == b["n_steps"] and a["interactions"] == b["interactions"]
            assert np.array_equal(a["pixels"], b["pixels"])
            assert np.array_equal(a["retire_step"], b["retire_step"])
            assert np.array_equal(a["final_xy"], b["final_xy"])


def test_spherical_cluster_width_option():
    name = "plain_3keV_100um"
    with _sim(name, max_slots=512) as sim:
        assert sim.stats()["sph_cluster"] == 1
    with _sim(name, mode=cts.CTS_MODE_PLAIN) as sim:
        assert sim.stats()["sph_cluster"] == 4
    p = W.preset(name)
    for bad in (3, 8, -1):
        with pytest.raises(cts.SimError) as e:
            cts.Simulator(p["sensor"], p["mobility"], SPH, sph_cluster=bad)
        assert e.value.code == cts.SIM_EINVAL


def test_spherical_modes_agree_exactly():
    name = "plain_3keV_100um"
    evs = W.make_events(name, n=4, first_id=70)
    outs = []
    for mode, opt in [(cts.CTS_MODE_PLAIN, {}), (cts.CTS_MODE_BATCHED, {}),
                      (cts.CTS_MODE_BATCHED, dict(disable_graphs=1)), (cts.CTS_MODE_SERVE, {})]:
        with _sim(name, mode=mode, **opt) as sim:
            outs.append(sim.run(evs))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert a["n_steps"] == b["n_steps"]
            assert np.array_equal(a["pixels"], b["pixels"])
            assert a["interactions"] == b["interactions"]


def test_spherical_rejects_events_beyond_the_sort_size():
    name = "batch_20keV_320um"
    with _sim(name) as sim:
        ev = dict(W.make_events(name, n=1)[0], n_pairs=16385)
        with pytest.raises(cts.SimError) as e:
            sim.run([ev])
        assert e.value.code == cts.SIM_EINVAL
        ok = dict(W.make_events(name, n=1)[0], n_pairs=16384, depth_um=300.0)
        r = sim.run([ok])[0]
        assert r["status"] == 0 and r["n_carriers"] == 16384


@pytest.mark.parametrize("cluster", [1, 2, 4])
def test_spherical_equal_radii_take_the_sorting_path(cluster):
    # 300 holes at one radius and 300 at a larger one (the six axis points
    # (+-a, 0, 0), (0, +-a, 0), (0, 0, +-a) repeated, so the centre is 0 and
    # the squared radii are equal to the bit): the counting pass finds more
    # than 256 holes in one bin and the cluster's first CTA ranks all holes
    # by sorting.  Equal radii do not
    # count each other: the inner shell feels no field, the outer one the
    # inner 300.  One step without drift and diffusion, constant mobility.
    name = "batch_20keV_320um"
    p = W.preset(name)
    mob = dict(p["mobility"], model=W.MOB_CONST)
    field = W.field_switches(spherical=1, drift=0, diffusion=0)
    axes = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                    dtype=float)
    centre = np.array([0.0, 0.0, 160.0])
    xyz = np.concatenate([np.tile(axes * 0.5, (50, 1)), np.tile(axes * 2.0, (50, 1))]) + centre
    ev = W.explicit_event(xyz, seed=5, event_id=7)
    ref = oracle.run_event(oracle.make_params(dict(p["sensor"], max_steps=1), field, mob), ev)
    with cts.Simulator(p["sensor"], mob, field, sph_cluster=cluster) as sim:
        pos, st, done = sim.trajectory(dict(ev, n_carriers=600), 1)
    assert done == ref.n_steps == 1
    assert np.array_equal(st, ref.state)
    moved = np.linalg.norm(ref.pos - xyz, axis=1)
    assert np.all(moved[:300] == 0.0) and np.all(moved[300:] > 0.0)
    d = np.abs(pos - ref.pos).max(axis=1)
    assert d.max() < 1e-6 * moved.max()
