"""KS pins of every oracle sampler against the CDF of its analytic differential
distribution (numerical quadrature), plus per-interaction energy/momentum conservation.
Sample layout (or_sample): [happened, parent_T, parent_dir(3), T0, dir0(3), T1, dir1_z, dir1.dir0];
the incoming particle moves along +z."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle

ME = 0.51099895
PB = 0
N = 6000


def cdf_from_pdf(pdf, a, b, n=4001):
    x = np.linspace(a, b, n)
    y = np.array([pdf(v) for v in x])
    c = integrate.cumulative_trapezoid(y, x, initial=0.0)
    # refine with Simpson-accurate total via quad
    tot = integrate.quad(pdf, a, b, epsrel=1e-10, limit=400)[0]
    c *= tot / c[-1]
    return lambda v: np.interp(v, x, c / tot)


def ks(samples, cdf):
    return stats.kstest(samples, cdf).pvalue


@pytest.mark.parametrize("E", [0.02, 0.5, 5.0, 500.0])
def test_compton(slab_oracle, E):
    s = slab_oracle.sample(oracle.S_COMPTON, PB, E, N)
    kap = E / ME
    e0 = 1 / (1 + 2 * kap)
    eps = s[:, 1] / E

    def pdf(e):
        c = 1 - (1 / e - 1) / kap
        return e + 1 / e - (1 - c * c)
    assert ks(eps, cdf_from_pdf(pdf, e0, 1.0)) > 1e-3
    # photon angle from Compton kinematics
    cth = s[:, 4]
    assert np.allclose(cth, 1 - (1 / eps - 1) / kap, rtol=0, atol=1e-12)
    # momentum conservation: E z = E' u' + p_e u_e with |p_e| from the electron energy
    Te = s[:, 5]
    assert np.all(Te + s[:, 1] == E)
    pe = np.sqrt(Te * (Te + 2 * ME))
    pvec = np.array([0, 0, E]) - s[:, 1:2] * s[:, 2:5]
    assert np.allclose(np.linalg.norm(pvec, axis=1), pe, rtol=1e-9)
    assert np.allclose(pvec / np.linalg.norm(pvec, axis=1)[:, None], s[:, 6:9], atol=1e-12)
    # azimuth uniform
    phi = np.arctan2(s[:, 3], s[:, 2])
    assert ks((phi + np.pi) / (2 * np.pi), "uniform") > 1e-3


@pytest.mark.parametrize("E", [1.2, 10.0, 1e4])
def test_pair(slab_oracle, E):
    s = slab_oracle.sample(oracle.S_PAIR, PB, E, N)
    assert np.all(s[:, 0] == 1) and np.all(s[:, 1] == -1)  # parent absorbed
    a = ME / E
    x = (s[:, 5] + ME) / E  # positron total-energy fraction
    assert ks(x, cdf_from_pdf(lambda v: 1 - 4 / 3 * v * (1 - v), a, 1 - a)) > 1e-3
    assert np.allclose(s[:, 5] + s[:, 9] + 2 * ME, E, rtol=1e-15)
    assert np.all(s[:, 5] >= -1e-12) and np.all(s[:, 9] >= -1e-12)
    # characteristic angles m/E+-
    assert np.allclose(s[:, 8], np.cos(ME / (s[:, 5] + ME)), atol=1e-12)
    assert np.allclose(s[:, 10], np.cos(ME / (s[:, 9] + ME)), atol=1e-12)
    assert not np.any(np.isnan(s))


def test_pair_below_threshold_does_nothing(slab_oracle):
    s = slab_oracle.sample(oracle.S_PAIR, PB, 1.0, 10)
    assert np.all(s[:, 0] == 0)


def moller_pdf(T, e):
    g = T / ME + 1
    gg = (2 * g - 1) / g**2
    return (1 - gg) + 1 / e**2 + 1 / (1 - e) ** 2 - gg / (e * (1 - e))


def bhabha_pdf(T, e):
    g = T / ME + 1
    b2 = 1 - 1 / g**2
    y = 1 / (g + 1)
    y12 = 1 - 2 * y
    B1, B2, B4 = 2 - y * y, y12 * (3 + y * y), y12**3
    B3 = B4 + y12**2
    return 1 / (b2 * e**2) - B1 / e + B2 - B3 * e + B4 * e**2


def check_two_body(s, T):
    Td = s[:, 5]
    Tp = s[:, 1]
    assert np.allclose(Td + Tp, T, rtol=1e-15)
    p0 = math.sqrt(T * (T + 2 * ME))
    pd = np.sqrt(Td * (Td + 2 * ME))
    pp = np.sqrt(Tp * (Tp + 2 * ME))
    rest = np.array([0, 0, p0]) - pd[:, None] * s[:, 6:9]
    # the primary's momentum from conservation must have the on-shell magnitude
    assert np.allclose(np.linalg.norm(rest, axis=1), pp, rtol=1e-9)
    assert np.allclose(rest / np.linalg.norm(rest, axis=1)[:, None], s[:, 2:5], atol=1e-10)


@pytest.mark.parametrize("T", [2.5, 20.0, 2e3])
def test_moller(slab_oracle, T):
    Tc, _ = slab_oracle.cuts(PB)
    s = slab_oracle.sample(oracle.S_MOLLER, PB, T, N)
    eps = s[:, 5] / T
    a = Tc / T
    # compare in u = 1/eps where the density is smooth
    cdf = cdf_from_pdf(lambda u: moller_pdf(T, 1 / u) / u**2, 2.0, 1 / a, n=20001)
    assert ks(1 / eps, cdf) > 1e-3
    assert np.all((eps >= a - 1e-15) & (eps <= 0.5 + 1e-15))
    check_two_body(s, T)


@pytest.mark.parametrize("T", [2.5, 20.0, 2e3])
def test_bhabha(slab_oracle, T):
    Tc, _ = slab_oracle.cuts(PB)
    s = slab_oracle.sample(oracle.S_BHABHA, PB, T, N)
    eps = s[:, 5] / T
    a = Tc / T
    cdf = cdf_from_pdf(lambda u: bhabha_pdf(T, 1 / u) / u**2, 1.0, 1 / a, n=20001)
    assert ks(1 / eps, cdf) > 1e-3
    assert np.all((eps >= a - 1e-15) & (eps <= 1 + 1e-15))
    check_two_body(s, T)


def test_bhabha_rejection_function_bounded():
    # the acceptance 1 - b2 eps (B1 - eps (B2 - eps (B3 - eps B4))) must stay in [0, 1]
    for T in np.exp(np.linspace(math.log(1e-3), math.log(1e6), 60)):
        g = T / ME + 1
        b2 = 1 - 1 / g**2
        e = np.linspace(1e-6, 1.0, 2001)
        val = b2 * e**2 * bhabha_pdf(T, e)
        assert np.all(val <= 1 + 1e-12) and np.all(val >= -1e-12)


def test_moller_rejection_bound():
    for T in np.exp(np.linspace(math.log(1e-3), math.log(1e6), 60)):
        g = T / ME + 1
        gg = (2 * g - 1) / g**2
        e = np.linspace(1e-6, 0.5, 2001)
        assert np.all(e**2 * moller_pdf(T, e) <= 2 + 0.25 * (1 - gg) + 1e-12)


@pytest.mark.parametrize("T", [0.5, 30.0, 3e4])
def test_brem(slab_oracle, T):
    _, kc = slab_oracle.cuts(PB)
    s = slab_oracle.sample(oracle.S_BREM, PB, T, N)
    k = s[:, 5]
    E = T + ME
    cdf = cdf_from_pdf(lambda lk: 4 / 3 - 4 / 3 * math.exp(lk) / E + (math.exp(lk) / E) ** 2,
                       math.log(kc), math.log(T), n=20001)
    assert ks(np.log(k), cdf) > 1e-3
    assert np.all(s[:, 1] + k == T)
    assert np.allclose(s[:, 4], 1.0)  # lepton keeps its direction
    assert np.allclose(s[:, 8], math.cos(ME / E), atol=1e-12)


@pytest.mark.parametrize("T", [0.01, 1.0, 300.0])
def test_annihilation_in_flight(slab_oracle, T):
    s = slab_oracle.sample(oracle.S_ANNIH, PB, T, N)
    g = T / ME + 1
    sq = math.sqrt((g - 1) / (g + 1))
    emin, emax = (1 - sq) / 2, (1 + sq) / 2
    Etot = T + 2 * ME
    eps = s[:, 5] / Etot
    S = lambda e: -(g + 1) ** 2 + (g * g + 4 * g + 1) / e - 1 / e**2
    cdf = cdf_from_pdf(lambda le: S(math.exp(le)) * math.exp(le), math.log(emin), math.log(emax), n=20001)
    assert ks(np.log(eps), cdf) > 1e-3
    assert np.allclose(s[:, 5] + s[:, 9], Etot, rtol=1e-15)
    # photon 2 from momentum conservation must be massless: |p+ z - E1 u1| = E2
    pp = math.sqrt(T * (T + 2 * ME))
    rest = np.array([0, 0, pp]) - s[:, 5:6] * s[:, 6:9]
    assert np.allclose(np.linalg.norm(rest, axis=1), s[:, 9], rtol=1e-9)


def test_annihilation_at_rest(slab_oracle):
    s = slab_oracle.sample(oracle.S_ANNIH_REST, PB, 0.0, N)
    assert np.all(s[:, 5] == ME) and np.all(s[:, 9] == ME)
    assert np.allclose(s[:, 11], -1.0)  # back to back
    assert ks((s[:, 8] + 1) / 2, "uniform") > 1e-3  # isotropic: cos theta uniform
    phi = np.arctan2(s[:, 7], s[:, 6])
    assert ks((phi + np.pi) / (2 * np.pi), "uniform") > 1e-3
