"""Pins of the oracle's generalised-Gaussian model (Sec. 3.1, Eq. 8) and fast
generation (Sec. 4.2): the density's normalisation and its Gaussian and
Laplace special cases, the sampler against the distribution (KS and the
closed-form moment), the maximum-likelihood fit against scipy's, and the
generator's charge bookkeeping."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle


@pytest.mark.parametrize("alpha,beta", [(1.0, 2.0), (2.5, 2.6), (0.7, 1.0), (4.0, 6.0)])
def test_density_is_normalised(alpha, beta):
    v, _ = integrate.quad(lambda x: oracle.ggd_pdf(x, alpha, beta), -60 * alpha, 60 * alpha,
                          points=[0.0], limit=200)
    assert v == pytest.approx(1.0, abs=1e-9)


def test_density_special_cases():
    # beta = 2: a Gaussian of sigma = alpha / sqrt(2); beta = 1: a Laplace law
    for x in (0.0, 0.3, 1.7, -2.2):
        assert oracle.ggd_pdf(x, 1.5, 2.0) == pytest.approx(
            stats.norm.pdf(x, scale=1.5 / math.sqrt(2)), rel=1e-12)
        assert oracle.ggd_pdf(x, 0.8, 1.0) == pytest.approx(
            stats.laplace.pdf(x, scale=0.8), rel=1e-12)


@pytest.mark.parametrize("alpha,beta", [(3.0, 2.5), (1.2, 2.0), (5.0, 3.3), (2.0, 1.5)])
def test_sampler_follows_the_density(alpha, beta):
    x = oracle.ggd_samples(20250611, 7, 20000, alpha, beta)
    assert stats.kstest(x, stats.gennorm(beta, scale=alpha).cdf).pvalue > 1e-3
    # E|X|^beta = alpha^beta / beta, relative sd sqrt(beta / n) ~ 1 %
    m = (np.abs(x) ** beta).mean()
    assert m == pytest.approx(alpha ** beta / beta, rel=0.05)
    # signs are balanced and the two axes are independent draws
    assert abs((x > 0).mean() - 0.5) < 0.02
    y = oracle.ggd_samples(20250611, 7, 20000, alpha, beta, axis=1)
    assert abs(np.corrcoef(x, y)[0, 1]) < 0.03


def test_ml_fit_matches_scipy_and_recovers_the_truth():
    x = oracle.ggd_samples(3, 4, 40000, 2.2, 2.7)
    a, b = oracle.fit_ggd(x)
    sb, _, sa = stats.gennorm.fit(x, floc=0)
    assert a == pytest.approx(sa, rel=1e-4) and b == pytest.approx(sb, rel=1e-4)
    assert a == pytest.approx(2.2, rel=0.02) and b == pytest.approx(2.7, rel=0.03)
    # the profile likelihood is largest at the fitted beta
    def loglik(al, be):
        return np.log([oracle.ggd_pdf(v, al, be) for v in x[:2000]]).sum()
    a2, b2 = oracle.fit_ggd(x[:2000])
    for db in (-0.05, 0.05):
        assert loglik(a2, b2) >= loglik(a2, b2 + db)
    with pytest.raises(ValueError):
        oracle.fit_ggd(np.zeros(10))


def test_generator_bookkeeping():
    ev = dict(seed=1, event_id=5, n_pairs=5525, x_um=3.0, y_um=-4.0, alpha=6.0, beta=2.5)
    pix, out = oracle.generate([ev], 25.0, 9)
    assert pix.sum() + out[0] == 5525
    # the entry pixel (4, 4) holds the largest count; the cloud is symmetric
    # about the entry point, so the x marginal peaks there too
    assert np.unravel_index(pix[0].argmax(), pix[0].shape) == (4, 4)
    # a cloud much narrower than a pixel lands in one pixel
    pix, out = oracle.generate([dict(ev, alpha=1e-3)], 25.0, 9)
    assert pix[0, 4, 4] == 5525 and out[0] == 0
    # a wide cloud spills out of a 3 x 3 grid; pixel shares follow the GGD
    # cell probabilities
    big = dict(ev, x_um=0.0, y_um=0.0, alpha=30.0, beta=2.0, n_pairs=50000)
    pix, out = oracle.generate([big], 25.0, 3)
    cdf = stats.gennorm(2.0, scale=30.0).cdf
    p1 = np.array([cdf(-12.5) - cdf(-37.5), cdf(12.5) - cdf(-12.5), cdf(37.5) - cdf(12.5)])
    expect = 50000 * np.outer(p1, p1)
    assert np.all(np.abs(pix[0] - expect) < 5 * np.sqrt(expect) + 1)
    assert pix.sum() + out[0] == 50000


def test_parameterisation_functions_and_fits():
    pa = [1.5, 2.0, -0.3, 0.02]
    pb = [0.4, 2.0, 0.5, 1.2, -0.8]
    t = np.linspace(0.2, 20.0, 60)
    # Eq. 10 by hand at t = 4: 1.5 + 2 * 2 - 1.2 + 0.32
    assert oracle.alpha_of_t(pa, 4.0) == pytest.approx(4.62, abs=1e-12)
    # Eq. 11 before p1 is the exponential term alone; after it both terms add
    assert oracle.beta_of_t(pb, 1.0) == pytest.approx(2 + 1.2 * math.exp(-0.8), abs=1e-12)
    assert oracle.beta_of_t(pb, 6.0) == pytest.approx(2 + 0.4 * 2.0 + 1.2 * math.exp(-4.8),
                                                      abs=1e-12)
    # noise-free data give back the parameters
    assert np.allclose(oracle.fit_alpha_of_t(t, oracle.alpha_of_t(pa, t)), pa, atol=1e-9)
    q = oracle.fit_beta_of_t(t, oracle.beta_of_t(pb, t), [0.3, 1.8, 0.6, 1.0, -0.6])
    assert np.allclose(q, pb, rtol=1e-4, atol=1e-6)


def test_weighted_eq10_fit_is_weighted_least_squares():
    # Rows scaled by w minimise sum w^2 r^2: exact data come back for any
    # weights, and integer weights equal repeating each point w^2 times
    pa = [1.5, 2.0, -0.3, 0.02]
    t = np.linspace(0.2, 20.0, 40)
    rng = np.random.default_rng(12)
    w = rng.integers(1, 4, t.size).astype(float)
    assert np.allclose(oracle.fit_alpha_of_t(t, oracle.alpha_of_t(pa, t), w), pa, atol=1e-9)
    noisy = oracle.alpha_of_t(pa, t) + rng.normal(0, 0.05, t.size)
    rep = np.repeat(np.arange(t.size), (w ** 2).astype(int))
    a = oracle.fit_alpha_of_t(t, noisy, w)
    b = oracle.fit_alpha_of_t(t[rep], noisy[rep])
    assert np.allclose(a, b, rtol=1e-9, atol=1e-10)
    assert not np.allclose(a, oracle.fit_alpha_of_t(t, noisy), rtol=1e-6, atol=1e-8)
