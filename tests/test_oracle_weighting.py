"""Pins of the oracle's pixel weighting potential (Shockley-Ramo; the weighting
field the paper names as the step towards transient signals, Sec. 5.3) and of
the per-pixel induced charge its transport run records.

The potential solves Laplace's equation in the slab 0 < z < H with 1 on the
pixel, 0 on the rest of the collecting surface and on the back surface.  The
oracle writes it as an image series of rectangle solid angles; the pins below
come from other representations and from identities of the boundary problem:
the Fourier-integral solution, direct quadrature of the half-space Poisson
kernel, the sum over all pixels (the planar potential 1 - z/H), boundary
values, symmetry and the end values of the recorded signals."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
import workloads as W

H = 100.0
P = 25.0
PIX = (-P / 2, P / 2, -P / 2, P / 2)


def phi(x, y, z, rect=PIX, h=H):
    return oracle.weighting_potential(x, y, z, rect, h)


def _fourier(x, y, z, a, b, h):
    """The slab solution by Fourier transform in (x, y): the boundary data's
    transform (a product of sinc's) times sinh(k (H - z)) / sinh(k H)."""
    def f(ky, kx):
        k = math.hypot(kx, ky)
        g = math.sinh(k * (h - z)) / math.sinh(k * h) if k * h < 700 else math.exp(-k * z)
        return (2 * math.sin(kx * a / 2) / kx) * (2 * math.sin(ky * b / 2) / ky) * \
            math.cos(kx * x) * math.cos(ky * y) * g
    kmax = 60.0 / z
    val, _ = integrate.dblquad(f, 1e-12, kmax, 1e-12, kmax, epsabs=1e-11, epsrel=1e-10)
    return val / math.pi ** 2


@pytest.mark.parametrize("pt", [(0.0, 0.0, 30.0), (20.0, 5.0, 60.0), (40.0, -30.0, 90.0)])
def test_matches_the_fourier_integral_solution(pt):
    x, y, z = pt
    assert phi(x, y, z) == pytest.approx(_fourier(x, y, z, P, P, H), abs=2e-9)


@pytest.mark.parametrize("pt", [(0.0, 0.0, 5.0), (30.0, 4.0, 12.0), (-7.0, 11.0, 2.0),
                                (60.0, -45.0, 40.0)])
def test_half_space_term_is_the_poisson_kernel_integral(pt):
    # solid angle / 2 pi = integral of zeta / (2 pi r^3) over the rectangle
    x, y, zeta = pt
    rect = (-10.0, 15.0, -5.0, 20.0)
    val, _ = integrate.dblquad(
        lambda yp, xp: zeta / (2 * math.pi * ((xp - x) ** 2 + (yp - y) ** 2 + zeta ** 2) ** 1.5),
        rect[0], rect[1], rect[2], rect[3], epsabs=1e-13, epsrel=1e-12)
    assert oracle.rect_solid_angle(x, y, zeta, rect) == pytest.approx(val, abs=1e-11)
    # odd in zeta
    assert oracle.rect_solid_angle(x, y, -zeta, rect) == -oracle.rect_solid_angle(x, y, zeta, rect)


@pytest.mark.parametrize("z", [7.0, 50.0, 93.0])
def test_sum_over_all_pixels_is_the_planar_potential(z):
    # the pixels tile the collecting surface: their potentials add up to the
    # potential of the whole surface, 1 - z / H; the slab confines a pixel's
    # potential laterally (decay exp(-pi r / H)), so +-40 pitches suffice.
    # Pixels 14 H away need more image pairs before the two-term tail is
    # exact to 1e-9 (its next term grows like r^4 and z^4): 200 pairs leave
    # 2e-10, while a dropped n^-5 tail term would leave 2e-8 - 2e-7 and a
    # wrong tail sign 1e-5 - 1e-4
    x, y = 3.0, 7.0
    n = 40
    tot = 0.0
    for i in range(-n, n + 1):
        for j in range(-n, n + 1):
            tot += oracle.weighting_potential(
                x, y, z, (i * P - P / 2, i * P + P / 2, j * P - P / 2, j * P + P / 2), H, 200)
    assert tot == pytest.approx(1.0 - z / H, abs=5e-9)


def test_boundary_values_and_bounds():
    assert phi(3.0, -4.0, 0.0) == 1.0
    assert phi(13.0, 0.0, 0.0) == 0.0
    assert phi(3.0, -4.0, H) == 0.0
    # the limits from inside the slab
    assert phi(3.0, -4.0, 1e-7) == pytest.approx(1.0, abs=1e-6)
    assert phi(13.0, 0.0, 1e-7) == pytest.approx(0.0, abs=1e-6)
    assert abs(phi(3.0, -4.0, H - 1e-7)) < 1e-8
    # the mid-edge of the pixel at the surface: one half
    assert phi(12.5, 0.0, 1e-9) == pytest.approx(0.5, abs=1e-6)
    # maximum principle and monotone decay below the pixel centre
    rng = np.random.default_rng(5)
    pts = np.column_stack([rng.uniform(-80, 80, 300), rng.uniform(-80, 80, 300),
                           rng.uniform(0.01, H - 0.01, 300)])
    vals = np.array([phi(*p) for p in pts])
    assert (vals >= -1e-12).all() and (vals <= 1 + 1e-12).all()
    col = [phi(0.0, 0.0, z) for z in np.linspace(0.5, H - 0.5, 40)]
    assert np.all(np.diff(col) < 0)


def test_laplace_residual_is_at_the_finite_difference_level():
    h = 0.5
    for (x, y, z) in [(5.0, 3.0, 20.0), (14.0, -9.0, 45.0), (31.0, 27.0, 70.0)]:
        c = phi(x, y, z)
        d2 = [phi(x + h, y, z) + phi(x - h, y, z) - 2 * c,
              phi(x, y + h, z) + phi(x, y - h, z) - 2 * c,
              phi(x, y, z + h) + phi(x, y, z - h) - 2 * c]
        scale = max(abs(v) for v in d2)
        assert abs(sum(d2)) < 2e-3 * scale, (x, y, z, d2)


def test_symmetry_and_translation():
    for (x, y, z) in [(4.0, 9.0, 17.0), (-30.0, 12.0, 66.0)]:
        v = phi(x, y, z)
        assert phi(-x, y, z) == pytest.approx(v, rel=1e-12, abs=1e-15)
        assert phi(x, -y, z) == pytest.approx(v, rel=1e-12, abs=1e-15)
        assert phi(y, x, z) == pytest.approx(v, rel=1e-12, abs=1e-15)
        sh = (P * 3, P * -2)
        moved = (PIX[0] + sh[0], PIX[1] + sh[0], PIX[2] + sh[1], PIX[3] + sh[1])
        assert phi(x + sh[0], y + sh[1], z, moved) == pytest.approx(v, rel=1e-12, abs=1e-15)


def test_thick_sensor_limit_is_the_half_space_solution():
    for (x, y, z) in [(0.0, 0.0, 10.0), (20.0, -5.0, 3.0)]:
        assert phi(x, y, z, h=1e7) == pytest.approx(oracle.rect_solid_angle(x, y, z, PIX),
                                                    abs=1e-9)


def test_more_image_pairs_converge():
    # the two-term tail leaves an error far below the test tolerances
    for (x, y, z) in [(0.0, 0.0, 30.0), (80.0, 80.0, 50.0)]:
        ref = phi(x, y, z)
        assert oracle.weighting_potential(x, y, z, PIX, H, 200) == pytest.approx(ref, abs=1e-12)
        assert abs(oracle.weighting_potential(x, y, z, PIX, H, 4) - ref) < 1e-7


def _params(name="plain_3keV_100um", **sensor_over):
    p = W.preset(name)
    sensor = dict(p["sensor"], **sensor_over)
    return oracle.make_params(sensor, W.field_switches(), p["mobility"])


def test_window_layout_and_surface_rule():
    pr = _params()              # grid 5 x 5, centre pixel (2, 2), pitch 25
    g, pitch = pr.grid_n, pr.pitch_um
    x, y, z = 9.0, -21.0, 37.0
    w = oracle.window_potentials(pr, x, y, z)
    for b in range(3):
        for a in range(3):
            ix, iy = g // 2 - 1 + a, g // 2 - 1 + b
            x1, y1 = (ix - g / 2) * pitch, (iy - g / 2) * pitch
            assert w[b, a] == phi(x, y, z, (x1, x1 + pitch, y1, y1 + pitch), pr.thickness_um)
    # on the collecting surface: one-hot on the readout's own pixel
    for (x, y) in [(0.0, 0.0), (13.0, -20.0), (-37.4, 37.4), (70.0, 0.0)]:
        w = oracle.window_potentials(pr, x, y, 0.0)
        exp = np.zeros((3, 3))
        ix, iy = oracle.pixel_of(pr, x, y) or (-9, -9)
        if abs(ix - g // 2) <= 1 and abs(iy - g // 2) <= 1:
            exp[iy - g // 2 + 1, ix - g // 2 + 1] = 1.0
        assert np.array_equal(w, exp), (x, y)
    assert not oracle.window_potentials(pr, 1.0, 2.0, pr.thickness_um).any()


def _pairs_event(n, seed=3):
    rng = np.random.default_rng(seed)
    xyz = np.column_stack([rng.normal(4.0, 6.0, n), rng.normal(-3.0, 6.0, n),
                           rng.uniform(15.0, 40.0, n)])
    return xyz


def test_two_species_signal_ends_at_the_pixel_counts():
    # holes and electrons start at the same points: their start potentials
    # cancel, electrons end on the back surface (potential 0) and holes on a
    # pixel (potential 1 there), so each pixel's final signal is its count.
    # Both mobilities (electrons are faster); pairs near the back surface so
    # that every electron leaves before the last hole arrives.
    p = W.preset("track_200keV_320um")
    sensor = dict(p["sensor"], thickness_um=50.0, bias_V=50.0, depletion_V=20.0, dt_ps=5.0,
                  grid_n=9)
    pr = oracle.make_params(sensor, W.field_switches(), p["mobility"])
    xyz = _pairs_event(30)
    xyz[:, 2] += 10.0
    both = np.concatenate([xyz, xyz])
    sign = np.concatenate([np.ones(30), -np.ones(30)]).astype(np.int8)
    r = oracle.run_event(pr, W.explicit_event(both, sign, event_id=7), induced_px=True)
    assert r.status == 0 and r.n_lost == 0
    c = pr.grid_n // 2
    win = r.pixels[c - 1:c + 2, c - 1:c + 2]
    assert win.sum() > 20
    assert np.abs(r.induced_px[-1] - win).max() < 1e-9
    # the whole-surface signal of the same run ends at the collected count
    assert r.induced[-1] == pytest.approx(30.0, abs=1e-9)


def test_hole_signal_telescopes_from_the_start_potentials():
    pr = _params()
    xyz = _pairs_event(40, seed=4)
    r = oracle.run_event(pr, W.explicit_event(xyz, event_id=9), induced_px=True)
    assert r.status == 0
    c = pr.grid_n // 2
    start = sum(oracle.window_potentials(pr, *p) for p in xyz)
    win = r.pixels[c - 1:c + 2, c - 1:c + 2]
    assert np.abs(r.induced_px[-1] - (win - start)).max() < 1e-9
    assert r.induced_px.shape == (r.n_steps, 3, 3)
    # the first step alone, from the recorded end positions of a one-step run
    one = oracle.run_event(_params(max_steps=1), W.explicit_event(xyz, event_id=9),
                           induced_px=True)
    moved = one.pos.copy()
    moved[:, 2] = np.clip(moved[:, 2], 0.0, pr.thickness_um)
    end = sum(oracle.window_potentials(pr, *p) for p in moved)
    assert np.abs(one.induced_px[0] - (end - start)).max() < 1e-9
    assert np.abs(r.induced_px[0] - one.induced_px[0]).max() < 1e-12
