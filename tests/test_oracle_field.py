"""Pins of the oracle's repulsion field (Eq. 4 read as a field, Sec. 2.1) and of its
material constants, against closed forms, library constants and invariants."""
import math

import numpy as np
import pytest
from scipy import constants as K
from scipy import integrate, special

import workloads as W


def test_constants_against_scipy(orc):
    kc = K.e / (4 * math.pi * K.epsilon_0 * 11.7) * 1e6   # V um
    assert orc.coulomb_k(11.7) == pytest.approx(kc, rel=1e-9)
    assert orc.thermal_voltage(293.0) == pytest.approx(K.k * 293.0 / K.e, rel=1e-12)


@pytest.mark.parametrize("e_kev,n", [(3.0, 829), (5.0, 1381), (8.0, 2210), (17.5, 4834),
                                     (20.0, 5525), (25.0, 6906)])
def test_pair_count_3p62_eV(orc, e_kev, n):
    # Sec. 2: one pair per 3.62 eV; these counts are the ones the workloads quote.
    assert orc.n_pairs(e_kev) == n


def test_sigma_power_law(orc):
    # Eq. 2: sigma = 0.0044 E^1.75 -> value at 1 keV and the scaling exponent.
    assert orc.sigma_um(1.0) == pytest.approx(0.0044, rel=1e-15)
    assert orc.sigma_um(20.0) / orc.sigma_um(10.0) == pytest.approx(2 ** 1.75, rel=1e-14)


def test_drift_field_integrates_to_bias(orc):
    s = W.preset("batch_20keV_320um")
    P = orc.make_params(s["sensor"], None, s["mobility"])
    H, Vb, Vd = 320.0, 150.0, 60.0
    # Highest field at the junction (pixel) side, lowest at the back.
    assert orc.drift_field(P, 0.0) == pytest.approx((Vb + Vd) / H, rel=1e-14)
    assert orc.drift_field(P, H) == pytest.approx((Vb - Vd) / H, rel=1e-14)
    # The potential drop across the sensor equals the bias voltage.
    v, _ = integrate.quad(lambda z: orc.drift_field(P, z), 0.0, H)
    assert v == pytest.approx(Vb, rel=1e-12)
    # Uniform doping: E is linear with slope 2 Vd / H^2 (Poisson equation).
    slope = (orc.drift_field(P, 100.0) - orc.drift_field(P, 200.0)) / 100.0
    assert slope == pytest.approx(2 * Vd / H ** 2, rel=1e-12)


def test_mobility_limits(orc):
    mob = dict(W.HOLE_MOBILITY)
    P = orc.make_params(W.preset("batch_20keV_320um")["sensor"], None, mob)
    mu0 = 480.0 * 0.1      # um^2/(V ns)
    vsat = 0.95e7 * 1e-5   # um/ns
    assert orc.mobility(P, 1, 0.0) == pytest.approx(mu0, rel=1e-15)
    # saturation: v = mu E -> vsat at high field
    assert orc.mobility(P, 1, 1e6) * 1e6 == pytest.approx(vsat, rel=1e-5)
    # monotone decreasing
    e = np.linspace(0, 10, 200)
    m = [orc.mobility(P, 1, x) for x in e]
    assert np.all(np.diff(m) < 0)
    # beta = 1: the textbook form mu0 / (1 + mu0 E / vsat)
    P1 = orc.make_params(W.preset("batch_20keV_320um")["sensor"], None, dict(mob, beta_h=1.0))
    for x in (0.1, 1.0, 3.0):
        assert orc.mobility(P1, 1, x) == pytest.approx(mu0 / (1 + mu0 * x / vsat), rel=1e-14)
    # constant-mobility switch
    Pc = orc.make_params(W.preset("batch_20keV_320um")["sensor"], None, dict(mob, model=1))
    assert orc.mobility(Pc, 1, 5.0) == pytest.approx(mu0, rel=1e-15)


def test_two_charges_coulomb(orc):
    kc = orc.coulomb_k(11.7)
    E = orc.field([[0, 0, 0], [0.3, 0.4, 0.0]])
    # |r| = 0.5: field magnitude k/r^2, pointing from the source to the target.
    assert E[1] == pytest.approx([kc / 0.25 * 0.6, kc / 0.25 * 0.8, 0.0], rel=1e-14)
    assert E[0] == pytest.approx(-E[1], rel=1e-14)


def test_opposite_charges_attract(orc):
    kc = orc.coulomb_k(11.7)
    E = orc.field([[0, 0, 0], [1.0, 0, 0]], sign=[1, -1])
    # Field at the hole (x=0) from the electron at x=1 points toward the electron
    # (+x); the field at the electron from the hole points away from the hole (+x)
    # and the electron moves against it, i.e. toward the hole.
    assert E[0] == pytest.approx([kc, 0, 0], rel=1e-14)
    assert E[1] == pytest.approx([kc, 0, 0], rel=1e-14)


def test_cube_vertices_closed_form(orc):
    a = 0.7
    kc = orc.coulomb_k(11.7)
    v = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float) * a
    E = orc.field(v)
    per_axis = kc / a ** 2 * (1 + 1 / math.sqrt(2) + 1 / (3 * math.sqrt(3)))
    centre = np.full(3, a / 2)
    for i in range(8):
        out = np.sign(v[i] - centre)
        assert E[i] == pytest.approx(per_axis * out, rel=1e-13)


def test_regular_tetrahedron(orc):
    kc = orc.coulomb_k(11.7)
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float)  # edge 2*sqrt(2)
    E = orc.field(v)
    edge = 2 * math.sqrt(2)
    # Three equal charges at distance `edge`, 109.47 deg apart as seen from the
    # centre: the resultant is radial with magnitude sqrt(6) k / edge^2.
    for i in range(4):
        rhat = v[i] / np.linalg.norm(v[i])
        assert E[i] == pytest.approx(math.sqrt(6) * kc / edge ** 2 * rhat, rel=1e-13)


def test_newton_third_law(orc):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((300, 3))
    s = np.where(rng.random(300) < 0.5, 1, -1).astype(np.int8)
    E = orc.field(x, sign=s)
    # Sum over carriers of q_i E_i = total internal force = 0.
    F = (s[:, None] * E).sum(axis=0)
    scale = np.abs(s[:, None] * E).sum(axis=0)
    assert np.all(np.abs(F) <= 1e-13 * scale)
    # The field changes sign when every charge flips only through q_i (it is a
    # field, not a force): flipping all signs flips every field.
    E2 = orc.field(x, sign=-s)
    assert np.allclose(E2, -E, rtol=1e-14, atol=0)


def test_inactive_carriers_are_not_sources(orc):
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 2, 0]], float)
    E_all = orc.field(x)
    E_two = orc.field(x[:2])
    E_mask = orc.field(x, active=[0, 0, 1])
    assert E_mask[:2] == pytest.approx(E_two, rel=1e-15)
    assert not np.allclose(E_all[:2], E_two)


def test_softening_form(orc):
    kc = orc.coulomb_k(11.7)
    eps = 0.1
    E = orc.field([[0, 0, 0], [0.2, 0, 0]], eps=eps)
    assert E[1][0] == pytest.approx(kc * 0.2 / (0.04 + eps ** 2) ** 1.5, rel=1e-14)
    # coincident carriers contribute nothing, with or without softening
    assert orc.field([[1, 1, 1], [1, 1, 1]])[0] == pytest.approx([0, 0, 0], abs=0)


def test_gauss_law_gaussian_cloud(orc):
    # Eq. 7 (the enclosed-charge field of a spherically symmetric cloud) applied to
    # a Gaussian cloud gives E(r) = k N / r^2 [erf(r / (sqrt2 s)) - sqrt(2/pi) (r/s)
    # exp(-r^2 / 2 s^2)].  The brute-force field of a sample approaches it.
    n, s = 20000, 1.0
    x = W.random_cloud(n, s, seed=11)
    rng = np.random.default_rng(5)
    rows = rng.choice(n, 300, replace=False)
    E = orc.field(x, rows=rows)
    kc = orc.coulomb_k(11.7)
    r = np.linalg.norm(x[rows], axis=1)
    keep = r > 0.8
    er = (E * x[rows]).sum(axis=1)[keep] / r[keep]
    rr = r[keep]
    enclosed = special.erf(rr / (math.sqrt(2) * s)) - math.sqrt(2 / math.pi) * rr / s * np.exp(-rr ** 2 / (2 * s ** 2))
    model = kc * (n - 1) / rr ** 2 * enclosed
    ratio = er / model
    assert abs(np.median(ratio) - 1.0) < 0.03
    assert abs(np.mean(ratio) - 1.0) < 0.05


def test_rows_equal_full(orc):
    x = W.random_cloud(200, 0.5, seed=2)
    full = orc.field(x)
    part = orc.field(x, rows=[5, 77, 199])
    assert part == pytest.approx(full[[5, 77, 199]], rel=0, abs=0)


def test_pixel_index_rule(orc):
    s = W.preset("batch_20keV_320um")
    P = orc.make_params(s["sensor"], None, s["mobility"])   # 9x9, 25 um
    assert orc.pixel_of(P, 0.0, 0.0) == (4, 4)
    assert orc.pixel_of(P, 12.5, -12.5) == (5, 4)      # lower edges belong to the pixel
    assert orc.pixel_of(P, 12.499999, -12.500001) == (4, 3)
    assert orc.pixel_of(P, -112.5, 112.4999) == (0, 8)
    assert orc.pixel_of(P, 112.5, 0.0) is None          # one past the last edge
    assert orc.pixel_of(P, -112.5000001, 0.0) is None
    pix, out = orc.bin_positions(P, [0.0, 30.0, 500.0, -30.0], [0.0, 0.0, 0.0, 60.0])
    assert out == 1 and pix.sum() == 3
    assert pix[4, 4] == 1 and pix[4, 5] == 1 and pix[6, 3] == 1
