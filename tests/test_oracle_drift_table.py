"""Pins of the oracle's sampled (non-uniform) drift field: a two-sample table
that lies on Eq. 6 reproduces Eq. 6, and a piecewise-linear profile gives the
transit time of its closed-form integral."""
import math

import numpy as np
import pytest

import workloads as W


def _sensor(H=100.0, dt_ps=1.0, steps=10**6, table=None):
    s = dict(thickness_um=H, bias_V=50.0, depletion_V=20.0, temperature_K=293.0, eps_r=11.7,
             pitch_um=25.0, grid_n=5, dt_ps=dt_ps, max_steps=steps, species=1)
    if table is not None:
        s["drift_table_Vum"] = table
    return s


def test_two_samples_on_eq6_reproduce_eq6(orc):
    s = _sensor(steps=300)
    P0 = orc.make_params(s, W.field_switches(0, 1, 0), dict(W.HOLE_MOBILITY))
    H = s["thickness_um"]
    E0, EH = orc.drift_field(P0, 0.0), orc.drift_field(P0, H)
    P1 = orc.make_params(_sensor(steps=300, table=[E0, EH]), W.field_switches(0, 1, 0),
                         dict(W.HOLE_MOBILITY))
    for z in (0.0, 17.0, 63.2, H):
        assert orc.drift_field(P1, z) == pytest.approx(orc.drift_field(P0, z), rel=1e-14)
    ev = W.explicit_event(np.array([[0.0, 0.0, 80.0], [1.0, 2.0, 40.0]]))
    r0, r1 = orc.run_event(P0, ev), orc.run_event(P1, ev)
    assert np.allclose(r0.pos, r1.pos, atol=1e-9)


def test_piecewise_linear_profile_transit_time(orc):
    # constant mobility, drift only: t = sum over segments of
    # dz ln(E1 / E0) / (mu (E1 - E0)) from the start depth to the surface
    H, mu = 100.0, 48.0                         # um, um^2/(V ns) (480 cm^2/Vs)
    table = [2.0, 0.5, 0.5, 1.5, 0.3]           # V/um at z = 0, 25, 50, 75, 100
    dz = H / (len(table) - 1)
    z0 = 90.0
    t = 0.0
    for k in range(len(table) - 1):
        a, b = k * dz, min((k + 1) * dz, z0)
        if b <= a:
            break
        e_a = table[k]
        e_b = table[k] + (table[k + 1] - table[k]) * (b - a) / dz
        t += (b - a) * (math.log(e_b / e_a) / (e_b - e_a) if e_b != e_a else 1.0 / e_a) / mu
    dt_ps = 1.0
    P = orc.make_params(_sensor(H=H, dt_ps=dt_ps, table=table), W.field_switches(0, 1, 0),
                        dict(W.HOLE_MOBILITY, model=1))
    r = orc.run_event(P, W.explicit_event(np.array([[0.0, 0.0, z0]])))
    assert r.status == 0
    assert r.n_steps * dt_ps * 1e-3 == pytest.approx(t, rel=0.01)
