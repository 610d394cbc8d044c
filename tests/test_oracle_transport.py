"""Pins of the oracle's time stepping (Algorithm 1; Eqs. 3, 5, 6; Sec. 2.1) against
closed forms: diffusion variance, drift kinematics and the drift-time integral
(Eq. 9), two-body repulsion and attraction, the expansion of a uniformly charged
ball, charge conservation, translation invariance and the flat-topped profile
that repulsion produces (Sec. 3.1)."""
import math

import numpy as np
import pytest
from scipy import optimize, stats

import workloads as W


def _params(orc, thickness=1000.0, bias=100.0, vdep=0.0, dt_ps=10.0, max_steps=10**6,
            species=1, repulsion=1, drift=1, diffusion=1, mob=None, grid_n=9, T=293.0):
    sensor = dict(thickness_um=thickness, bias_V=bias, depletion_V=vdep, temperature_K=T,
                  eps_r=11.7, pitch_um=25.0, grid_n=grid_n, dt_ps=dt_ps,
                  max_steps=max_steps, species=species)
    mob = dict(W.HOLE_MOBILITY) if mob is None else mob
    return orc.make_params(sensor, W.field_switches(repulsion, drift, diffusion), mob)


def test_diffusion_only_variance(orc):
    # Sec. 1: without repulsion the cloud spreads as a Gaussian of variance 2 D t
    # per axis; with the paper's random walk of variance 2 D dt per step it is
    # exact after any number of steps: Var = sigma0^2 + 2 D n dt.
    n_car, n_steps, dt_ps = 30000, 25, 10.0
    P = _params(orc, thickness=10000.0, dt_ps=dt_ps, max_steps=n_steps, repulsion=0,
                drift=0, mob=dict(W.HOLE_MOBILITY, model=1))
    xyz = np.zeros((n_car, 3)); xyz[:, 2] = 5000.0
    r = orc.run_event(P, W.explicit_event(xyz, seed=99, event_id=3))
    assert r.status == orc.EMAXSTEPS and r.n_steps == n_steps
    D = 48.0 * orc.thermal_voltage(293.0)          # um^2/ns
    var = 2 * D * n_steps * dt_ps * 1e-3
    d = r.pos - xyz
    for axis in range(3):
        v = d[:, axis]
        # chi-square interval for the sample variance (mean known = 0)
        s2 = np.mean(v ** 2)
        lo = stats.chi2.ppf(1e-4, n_car) / n_car * var
        hi = stats.chi2.ppf(1 - 1e-4, n_car) / n_car * var
        assert lo < s2 < hi, (axis, s2, var)
        assert abs(v.mean()) < 5 * math.sqrt(var / n_car)
        assert abs(stats.kurtosis(v)) < 5 * math.sqrt(24 / n_car)


def test_uniform_field_transit_is_exact_kinematics(orc):
    # Vd = 0: E = Vb / H everywhere.  Constant mobility: z decreases by mu E dt per
    # step; the hole is collected in the first step that brings z to <= 0.
    P = _params(orc, thickness=100.0, bias=50.0, vdep=0.0, dt_ps=10.0, repulsion=0,
                diffusion=0, mob=dict(W.HOLE_MOBILITY, model=1))
    z0 = 50.0
    r = orc.run_event(P, W.explicit_event([[1.0, 2.0, z0]]))
    step = 48.0 * 0.5 * 0.01
    assert r.status == 0
    assert r.n_steps == math.ceil(z0 / step)
    assert r.retire_step[0] == r.n_steps - 1
    assert r.pos[0] == pytest.approx([1.0, 2.0, z0 - r.n_steps * step], abs=1e-11)
    assert r.final_xy[0] == pytest.approx([1.0, 2.0], abs=0)
    assert r.n_collected == 1 and r.pixels[4, 4] == 1


def _transit_time(orc, dt_ps, z0, beta=1.0):
    P = _params(orc, thickness=320.0, bias=150.0, vdep=60.0, dt_ps=dt_ps, repulsion=0,
                diffusion=0, mob=dict(W.HOLE_MOBILITY, beta_h=beta))
    r = orc.run_event(P, W.explicit_event([[0.0, 0.0, z0]]))
    # Interpolate the crossing of z = 0 inside the last step.
    zN = r.pos[0, 2]
    v_end = orc.mobility(P, 1, orc.drift_field(P, 0.0)) * orc.drift_field(P, 0.0)
    return r.n_steps * dt_ps * 1e-3 + zN / v_end


def test_drift_time_eq9_closed_form_and_first_order_convergence(orc):
    # Eq. 9: with mu(E) = mu0 / (1 + mu0 E / vsat) (beta = 1) and the linear field
    # of Eq. 6, t = (1/mu0) [ln E / k + z / Ec] between the two end points, Ec =
    # vsat / mu0, k = |dE/dz|.  Forward Euler approaches it at first order.
    H, Vb, Vd = 320.0, 150.0, 60.0
    mu0, vsat = 48.0, 95.0
    k = 2 * Vd / H ** 2
    E = lambda z: (Vb - Vd) / H + 2 * Vd * (H - z) / H ** 2
    z0 = 250.0
    t_exact = (1 / (mu0 * k)) * math.log(E(0.0) / E(z0)) + z0 / vsat
    errs = [abs(_transit_time(orc, dt, z0) - t_exact) for dt in (40.0, 20.0, 10.0, 5.0)]
    assert errs[-1] < 2e-3 * t_exact
    for a, b in zip(errs, errs[1:]):
        assert 1.6 < a / b < 2.5, errs


def test_two_holes_constant_mobility(orc):
    # Two equal charges, repulsion only, constant mu: each moves at mu k / r^2, so
    # d(r^3)/dt = 6 mu k and r^3 = r0^3 + 6 mu k t.
    kc = orc.coulomb_k(11.7)
    mu = 48.0
    r0, n_steps = 0.05, 400
    res = []
    for dt_ps in (0.2, 0.1, 0.05):
        steps = int(round(n_steps * 0.2 / dt_ps))
        P = _params(orc, dt_ps=dt_ps, max_steps=steps, drift=0, diffusion=0,
                    mob=dict(W.HOLE_MOBILITY, model=1))
        r = orc.run_event(P, W.explicit_event([[0, 0, 500.0], [r0, 0, 500.0]]))
        sep = np.linalg.norm(r.pos[1] - r.pos[0])
        t = steps * dt_ps * 1e-3
        res.append(abs(sep - (r0 ** 3 + 6 * mu * kc * t) ** (1 / 3)))
    assert res[-1] < 1e-3 * r0
    assert 1.7 < res[0] / res[1] < 2.3 and 1.7 < res[1] / res[2] < 2.3


def test_two_holes_saturating_mobility_closed_form(orc):
    # beta = 1 mobility: dr/dt = 2 v(E), E = k / r^2 ->
    # t = 1/2 [ (r^3 - r0^3) / (3 mu0 k) + (r - r0) / vsat ].
    kc = orc.coulomb_k(11.7)
    mu0, vsat = 48.0, 95.0
    r0 = 0.01      # E = k / r0^2 ~ 1.2 V/um: mu0 E is comparable with vsat
    t_of = lambda r: 0.5 * ((r ** 3 - r0 ** 3) / (3 * mu0 * kc) + (r - r0) / vsat)
    errs = []
    for dt_ps in (0.004, 0.002, 0.001):
        steps = int(round(2.0 / dt_ps))          # t = 2 ps
        P = _params(orc, dt_ps=dt_ps, max_steps=steps, drift=0, diffusion=0,
                    mob=dict(W.HOLE_MOBILITY, beta_h=1.0))
        r = orc.run_event(P, W.explicit_event([[0, 0, 500.0], [0, r0, 500.0]]))
        sep = np.linalg.norm(r.pos[1] - r.pos[0])
        t = steps * dt_ps * 1e-3
        r_exact = optimize.brentq(lambda x: t_of(x) - t, r0, 10.0, xtol=1e-15)
        errs.append(abs(sep - r_exact))
    assert r_exact > 4 * r0
    assert errs[-1] < 5e-4 * r_exact
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_electron_hole_pair_attracts(orc):
    # Opposite charges with equal constant mobility close as r^3 = r0^3 - 6 mu k t.
    kc = orc.coulomb_k(11.7)
    mu, r0, dt_ps, steps = 48.0, 0.2, 0.1, 1100
    mob = dict(W.HOLE_MOBILITY, model=1, mu0_e=480.0, vsat_e=1e7, beta_e=1.0)
    P = _params(orc, dt_ps=dt_ps, max_steps=steps, drift=0, diffusion=0, species=3, mob=mob)
    r = orc.run_event(P, W.explicit_event([[0, 0, 500.0], [0, 0, 500.0 + r0]], sign=[1, -1]))
    sep = np.linalg.norm(r.pos[1] - r.pos[0])
    t = steps * dt_ps * 1e-3
    expect = (r0 ** 3 - 6 * mu * kc * t) ** (1 / 3)
    assert expect < 0.9 * r0
    assert sep == pytest.approx(expect, rel=2e-3)
    # the pair's centre does not move (equal mobilities, equal and opposite fields)
    assert (r.pos[0] + r.pos[1]) / 2 == pytest.approx([0, 0, 500.0 + r0 / 2], abs=1e-12)


def test_uniform_ball_expansion(orc):
    # A uniformly charged ball under repulsion alone with constant mu stays uniform
    # and its radius follows R^3 = R0^3 + 3 mu k Q t (Q = N - 1 charges act on each
    # carrier).  The RMS radius is sqrt(3/5) R.
    n, R0 = 2000, 1.0
    rng = np.random.default_rng(17)
    pts = rng.standard_normal((n, 3))
    pts *= (R0 * rng.random(n) ** (1 / 3) / np.linalg.norm(pts, axis=1))[:, None]
    pts[:, 2] += 500.0
    kc = orc.coulomb_k(11.7)
    mu, dt_ps, steps = 48.0, 2.0, 350
    P = _params(orc, dt_ps=dt_ps, max_steps=steps, drift=0, diffusion=0,
                mob=dict(W.HOLE_MOBILITY, model=1))
    r = orc.run_event(P, W.explicit_event(pts))
    c0 = pts.mean(axis=0); c1 = r.pos.mean(axis=0)
    rms0 = np.sqrt(((pts - c0) ** 2).sum(axis=1).mean())
    rms1 = np.sqrt(((r.pos - c1) ** 2).sum(axis=1).mean())
    t = steps * dt_ps * 1e-3
    R1 = (R0 ** 3 + 3 * mu * kc * (n - 1) * t) ** (1 / 3)
    assert R1 > 2.5 * R0
    assert rms1 / rms0 == pytest.approx(R1 / R0, rel=0.02)
    assert c1 == pytest.approx(c0, abs=1e-9)


def _event_params(orc, name, **over):
    p = W.preset(name)
    s = dict(p["sensor"], **over)
    return orc.make_params(s, W.field_switches(), p["mobility"])


def test_full_event_charge_conservation_and_translation(orc):
    P = _event_params(orc, "plain_3keV_100um")
    ev = W.make_events("plain_3keV_100um", n=2)
    r0, r1 = orc.run_events(P, ev)
    for r in (r0, r1):
        assert r.status == 0
        assert r.n_collected == 829
        assert r.pixels.sum() + r.n_outside == 829
        assert np.all(r.retire_step >= -1)
        assert r.interactions == orc.count_interactions(r.retire_step, r.n_steps)
    # Shift the entry point by one pitch in x: the map shifts by one column.
    ev_s = dict(ev[0], x_um=ev[0]["x_um"] + 25.0)
    rs = orc.run_event(P, ev_s)
    assert rs.n_steps == r0.n_steps
    assert np.array_equal(rs.pixels[:, 1:], r0.pixels[:, :-1])
    assert rs.pixels[:, 0].sum() == 0


def test_initial_boundaries(orc):
    # Absorbed at the pixel surface: every carrier with z <= 0 is collected before
    # the first step; the others are collected later.  Carriers beyond the back
    # surface are reflected into the sensor.
    P = _params(orc, thickness=100.0, bias=50.0, repulsion=0, diffusion=0)
    r = orc.run_event(P, W.explicit_event([[0, 0, -0.1], [0, 0, 0.0]]))
    assert r.n_steps == 0 and r.n_collected == 2 and np.all(r.retire_step == -1)
    r = orc.run_event(P, W.explicit_event([[0, 0, 101.0]]))
    assert r.n_collected == 1 and r.retire_step[0] >= 0
    P2 = _params(orc, thickness=100.0, bias=50.0, repulsion=0, diffusion=0, max_steps=1)
    r = orc.run_event(P2, W.explicit_event([[0, 0, 101.0]]))
    assert r.status == orc.EMAXSTEPS
    assert r.pos[0, 2] < 100.0


def test_electrons_leave_through_back_and_are_not_binned(orc):
    mob = dict(W.HOLE_MOBILITY, **W.ELECTRON_MOBILITY)
    P = _params(orc, thickness=50.0, bias=50.0, vdep=20.0, species=3, mob=mob)
    r = orc.run_event(P, W.explicit_event([[0, 0, 25.0], [0, 0, 25.0], [3, 0, 49.0]],
                                          sign=[1, -1, -1]))
    assert r.status == 0 and r.n_collected == 1 and r.pixels.sum() == 1
    assert r.state[0] == orc.COLLECTED
    # the electron close to the back contact leaves before the hole is collected
    assert r.state[2] == orc.RETIRED
    assert r.n_lost == int(r.state[1] == orc.ACTIVE)


@pytest.mark.slow
def test_repulsion_flattens_the_profile(orc):
    # Sec. 3.1: with repulsion the collected profile is broader than a Gaussian at
    # the peak (GGD shape beta > 2, i.e. negative excess kurtosis) for shallow
    # collection distances; without repulsion it is Gaussian (beta = 2).
    P = _event_params(orc, "batch_20keV_320um")
    ev = dict(seed=W.MASTER_SEED, event_id=77, kind=W.PHOTON, energy_keV=25.0, n_pairs=0,
              depth_um=300.0, x_um=0.0, y_um=0.0, sigma_um=-1.0)
    r = orc.run_event(P, ev)
    xy = r.final_xy - r.final_xy.mean(axis=0)
    k_rep = stats.kurtosis(xy.reshape(-1))
    P0 = orc.make_params(W.preset("batch_20keV_320um")["sensor"],
                         W.field_switches(repulsion=0), W.HOLE_MOBILITY)
    r0 = orc.run_event(P0, ev)
    xy0 = r0.final_xy - r0.final_xy.mean(axis=0)
    k_free = stats.kurtosis(xy0.reshape(-1))
    assert k_rep < -0.2, k_rep
    assert abs(k_free) < 0.2, k_free
    # repulsion also widens the profile
    assert xy.std() > 1.2 * xy0.std()


def test_induced_charge_on_the_collecting_surface(orc):
    # Shockley-Ramo with the planar weighting potential 1 - z/H: one hole
    # drifting at constant speed induces v t / H, and z0 / H in total
    H, Vb, dt_ps = 200.0, 100.0, 10.0
    P = _params(orc, thickness=H, bias=Vb, vdep=0.0, dt_ps=dt_ps, repulsion=0, diffusion=0,
                mob=dict(W.HOLE_MOBILITY, model=1))
    z0 = 120.0
    r = orc.run_event(P, W.explicit_event(np.array([[0.0, 0.0, z0]])))
    v = 48.0 * Vb / H                            # um/ns (480 cm^2/Vs)
    k = np.arange(1, r.n_steps + 1)
    expect = np.minimum(k * v * dt_ps * 1e-3, z0) / H
    assert np.allclose(r.induced, expect, rtol=1e-12, atol=1e-12)
    # a whole cloud with repulsion, diffusion and the Eq. 6 field: once every
    # hole is in, the sum telescopes to sum(z0) / H whatever the paths were
    P = _params(orc, thickness=H, bias=Vb, vdep=40.0, dt_ps=dt_ps)
    rng = np.random.default_rng(8)
    pts = rng.normal([0.0, 0.0, 150.0], 2.0, (300, 3))
    r = orc.run_event(P, W.explicit_event(pts))
    assert r.status == 0
    assert r.induced[-1] == pytest.approx(pts[:, 2].sum() / H, rel=1e-12)
    assert len(r.induced) == r.n_steps


def test_photon_cloud_starts_at_its_absorption_depth(orc):
    # The absorption depth is measured from the entrance (back) surface, so
    # in this frame (z from the collecting surface) the cloud starts at
    # z = H - depth; with sigma = 0 every pair sits exactly there.
    P = _params(orc, thickness=100.0, max_steps=0)
    ev = dict(seed=5, event_id=1, kind=W.PHOTON, energy_keV=3.0, n_pairs=40, depth_um=30.0,
              x_um=2.0, y_um=-3.0, sigma_um=0.0)
    r = orc.run_event(P, ev)
    assert r.status == orc.EMAXSTEPS and r.n_steps == 0
    assert np.array_equal(r.pos, np.tile([2.0, -3.0, 70.0], (40, 1)))
    # a Gaussian cloud around that point (Eq. 2's sigma given directly)
    r = orc.run_event(P, dict(ev, n_pairs=4000, sigma_um=1.5))
    m, s = r.pos.mean(axis=0), r.pos.std(axis=0)
    assert np.all(np.abs(m - [2.0, -3.0, 70.0]) < 4 * 1.5 / math.sqrt(4000))
    assert np.all(np.abs(s - 1.5) < 0.05)


@pytest.mark.parametrize("theta,phi", [(0.0, 0.0), (60.0, 0.0), (45.0, 90.0), (30.0, 225.0)])
def test_track_runs_inward_from_the_back_surface(orc, theta, phi):
    # sigma = 0: every pair lies on the segment from the entry point (x0, y0, H)
    # along (sin t cos p, sin t sin p, -cos t), uniformly over its length
    # (both species: an electron that started outside would leave through the
    # back contact before the first step, where a hole would be mirrored)
    H, L, n = 300.0, 80.0, 4000
    mob = dict(W.HOLE_MOBILITY, **W.ELECTRON_MOBILITY)
    P = _params(orc, thickness=H, max_steps=0, species=3, mob=mob)
    ev = dict(seed=8, event_id=2, kind=W.TRACK, energy_keV=200.0, n_pairs=n, depth_um=0.0,
              x_um=1.0, y_um=-2.0, sigma_um=0.0, track_len_um=L, theta_deg=theta, phi_deg=phi)
    r = orc.run_event(P, ev)
    assert (r.state == orc.ACTIVE).all()
    assert np.array_equal(r.pos[:n], r.pos[n:])         # a pair's carriers start together
    assert (r.sign[:n] == 1).all() and (r.sign[n:] == -1).all()
    t, p = math.radians(theta), math.radians(phi)
    u = np.array([math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), -math.cos(t)])
    d = r.pos[:n] - np.array([1.0, -2.0, H])
    s = d @ u
    assert np.abs(d - np.outer(s, u)).max() < 1e-9      # on the line
    assert s.min() >= 0.0 and s.max() <= L              # on the segment, inside the sensor
    assert abs(s.mean() - L / 2) < 4 * L / math.sqrt(12 * n)
    assert stats.kstest(s / L, "uniform").pvalue > 1e-4


def test_electrons_below_the_collecting_surface_are_mirrored(orc):
    # Diffusion only, equal constant mobilities: an electron starting just
    # above z = 0 ends its step at |z0 + dz| (reflected), so the end depths
    # follow a folded normal: none exactly at 0 and E[z^2] / E[z]^2 = pi / 2
    # whatever the step's width.  One far hole keeps the event running.
    mob = dict(W.HOLE_MOBILITY, model=1, mu0_e=480.0, vsat_e=0.95e7, beta_e=1.2)
    P = _params(orc, thickness=100.0, max_steps=1, species=3, repulsion=0, drift=0, mob=mob)
    n = 40000
    xyz = np.zeros((n + 1, 3))
    xyz[:, 2] = 1e-12
    xyz[n] = [0.0, 0.0, 50.0]
    sign = np.concatenate([-np.ones(n), [1]]).astype(np.int8)
    r = orc.run_event(P, W.explicit_event(xyz, sign, seed=4, event_id=6))
    assert r.n_steps == 1
    z = r.pos[:n, 2]
    assert (z > 0).all()
    ratio = np.mean(z ** 2) / np.mean(z) ** 2
    assert ratio == pytest.approx(math.pi / 2, rel=0.02)


def test_single_steps_reproduce_the_whole_event(orc):
    # orc.step (one loop body of Algorithm 1 from a given state, the entry
    # the one-step parity tests use) taken 20 times from the initial cloud
    # gives the states and positions of run_event after 20 steps, bit for bit
    p = W.preset("plain_3keV_100um")
    ev = W.make_events("plain_3keV_100um", n=1)[0]
    prm = orc.make_params(dict(p["sensor"], max_steps=20), W.field_switches(), p["mobility"])
    ref = orc.run_event(prm, ev)
    pos, sign = orc.init_event(prm, ev)
    st = np.zeros(len(sign), dtype=np.int8)
    for k in range(20):
        pos, st = orc.step(prm, ev["seed"], ev["event_id"], k, pos, sign, st)
    act = st == orc.ACTIVE
    assert np.array_equal(st, ref.state)
    assert np.array_equal(pos[act], ref.pos[act])
