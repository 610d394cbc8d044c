"""Pins of the oracle's simplified spherical model (Sec. 2.2, Eq. 7): a
hand-built symmetric configuration, Newton's shell theorem against the
pairwise field (Eq. 4) on a uniform ball, and the expansion law of a
uniformly charged ball, which the spherical model follows shell by shell."""
import numpy as np
import pytest

import workloads as W


def _ball(n, R, rng):
    p = rng.standard_normal((n, 3))
    return p * (R * rng.random(n) ** (1 / 3) / np.linalg.norm(p, axis=1))[:, None]


def test_symmetric_configuration_by_hand(orc):
    # holes at +-1 on x, +-2 on y, +-3 on z: centre 0; a hole at r = 2 has the
    # two at r = 1 inside, one at r = 3 the four at r = 1 and 2
    pts = np.array([[1, 0, 0], [-1, 0, 0], [0, 2, 0], [0, -2, 0], [0, 0, 3], [0, 0, -3]], float)
    e = orc.field_spherical(pts + [10.0, -4.0, 7.0], kc=1.0)
    expect = np.array([[0, 0, 0], [0, 0, 0], [0, 2 * 2 / 8, 0], [0, -2 * 2 / 8, 0],
                       [0, 0, 4 * 3 / 27], [0, 0, -4 * 3 / 27]])
    np.testing.assert_allclose(e, expect, atol=1e-15)
    # equal radii do not count each other; a single hole feels nothing
    e = orc.field_spherical(np.array([[1.0, 0, 0], [-1.0, 0, 0]]), kc=1.0)
    assert np.all(e == 0)
    assert np.all(orc.field_spherical(np.array([[3.0, 4.0, 5.0]]), kc=1.0) == 0)


def test_shell_theorem_against_the_pairwise_field(orc):
    # inside a uniformly charged ball the pairwise Coulomb field (Eq. 4) and
    # the enclosed-charge field of Eq. 7 agree up to sampling noise
    rng = np.random.default_rng(3)
    pts = _ball(6000, 5.0, rng)
    es = orc.field_spherical(pts, kc=1.0)
    ep = orc.field(pts, kc=1.0)
    r = np.linalg.norm(pts - pts.mean(0), axis=1)
    sel = (r > 1.5) & (r < 4.5)
    rad_s = (es[sel] * (pts[sel] - pts.mean(0))).sum(1) / r[sel]
    rad_p = (ep[sel] * (pts[sel] - pts.mean(0))).sum(1) / r[sel]
    # per carrier the pairwise field carries the graininess of its neighbours,
    # so compare shell averages
    edges = np.linspace(1.5, 4.5, 7)
    k = np.digitize(r[sel], edges) - 1
    for b in range(6):
        ms, mp = rad_s[k == b].mean(), rad_p[k == b].mean()
        assert ms == pytest.approx(mp, rel=0.03), b
        # and both follow the continuum N r / R^3 at the shell's mean radius
        assert ms == pytest.approx(6000 * r[sel][k == b].mean() / 125.0, rel=0.04), b


def test_uniform_ball_expansion_law(orc):
    # R^3 = R0^3 + 3 mu k_C Q t for the ball's edge; with the spherical model a
    # uniform ball stays uniform, so the RMS radius scales the same way
    n, R0 = 2000, 1.0
    pts = _ball(n, R0, np.random.default_rng(17))
    pts[:, 2] += 500.0
    kc = orc.coulomb_k(11.7)
    mu, dt_ps, steps = 48.0, 2.0, 350
    sensor = dict(thickness_um=1000.0, bias_V=100.0, depletion_V=0.0, temperature_K=293.0,
                  eps_r=11.7, pitch_um=25.0, grid_n=9, dt_ps=dt_ps, max_steps=steps, species=1)
    P = orc.make_params(sensor, W.field_switches(1, 0, 0, spherical=1),
                        dict(W.HOLE_MOBILITY, model=1))
    r = orc.run_event(P, W.explicit_event(pts))
    assert r.status == orc.EMAXSTEPS and r.n_steps == steps
    c0, c1 = pts.mean(0), r.pos.mean(0)
    rms0 = np.sqrt(((pts - c0) ** 2).sum(1).mean())
    rms1 = np.sqrt(((r.pos - c1) ** 2).sum(1).mean())
    t = steps * dt_ps * 1e-3
    R1 = (R0 ** 3 + 3 * mu * kc * n * t) ** (1 / 3)
    assert R1 > 2.5 * R0
    assert rms1 / rms0 == pytest.approx(R1 / R0, rel=0.02)
    # the model's forces are not pairwise (no momentum conservation), yet the
    # field is radial about the centre: the centre moves by a tiny fraction of
    # the radius only
    assert np.linalg.norm(c1 - c0) < 1e-3 * R1
    # one field evaluation per active hole and step is counted
    assert r.interactions == n * steps
