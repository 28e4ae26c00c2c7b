"""The seeded input recipes against their stated distributions (CPU).

Both the CUDA path and the oracle take their primaries and layouts from
paper_2209_15445_gb300.workloads; these tests check that each recipe draws what it states:
the slab and barrel layouts, the beam of the headline workload, the log-uniform energies,
the species fractions, the |eta| < 1.5 directions and the E^-2 serving spectrum on the inner
barrel face.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2209_15445_gb300 import workloads as W

N = 20000
P_MIN = 1e-3  # KS p-value floor (fixed seeds: the draws are the same every run)


def ks_uniform(x, lo, hi):
    return stats.kstest(x, "uniform", args=(lo, hi - lo)).pvalue


def species_fractions(pdg):
    return {p: np.mean(pdg == p) for p in (22, 11, -11)}


def within_binomial(f, p, n, k=5.0):
    return abs(f - p) <= k * math.sqrt(p * (1 - p) / n)


def test_slab_layout():
    g = W.slab_calorimeter()
    assert g.kind == 0 and g.n_layers == 50 and g.n_bins == 100
    assert [g.materials[m].name for m in g.sub_materials] == ["Pb", "lAr"]
    assert g.sub_thickness == [2.3, 5.7] and g.half_xy == 200.0
    assert g.n_layers * sum(g.sub_thickness) == pytest.approx(400.0, abs=1e-9)


def test_barrel_layout():
    g = W.barrel_calorimeter()
    assert g.kind == 1 and g.n_layers == 20 and g.half_z == 3000.0
    assert [g.materials[m].name for m in g.sub_materials] == ["Si", "Fe", "Pb", "lAr"]
    depth = sum(g.sub_thickness)
    assert depth == pytest.approx(28.3, abs=1e-12)
    r = np.array(g.layer_r)
    assert r[0] == 300.0 and r[-1] + depth == pytest.approx(1800.0, abs=1e-9)
    pitch = np.diff(r)
    np.testing.assert_allclose(pitch, (1500.0 - depth) / 19, rtol=1e-12)
    assert (pitch > depth).all()  # a vacuum gap between consecutive layers


def test_paper_calorimeter_is_the_slab_with_lead_tungstate():
    g, s = W.pbwo4_calorimeter(), W.slab_calorimeter()
    assert g.materials[0].elements and g.materials[1] == s.materials[1]
    assert g.sub_thickness == s.sub_thickness and g.n_layers == s.n_layers


def test_headline_beam():
    p = W.electrons(1000, 1e4, first_event=7)
    assert (p.pdg == 11).all() and (p.E == 1e4).all()
    assert (p.pos == 0).all() and (p.dir == [0, 0, 1]).all()
    np.testing.assert_array_equal(p.event, np.arange(7, 1007))


def test_mixed_recipe():
    p = W.mixed(N)
    assert p.E.min() >= 100.0 and p.E.max() <= 1e5
    assert ks_uniform(np.log(p.E), math.log(100.0), math.log(1e5)) > P_MIN
    f = species_fractions(p.pdg)
    for sp, want in ((22, 0.5), (11, 0.4), (-11, 0.1)):
        assert within_binomial(f[sp], want, N), (sp, f[sp])
    assert (p.pos == 0).all() and (p.dir == [0, 0, 1]).all()
    assert len(np.unique(p.event)) == N


def test_barrel_recipe():
    p = W.barrel_primaries(N)
    assert p.E.min() >= 1e3 and p.E.max() <= 5e4
    assert ks_uniform(np.log(p.E), math.log(1e3), math.log(5e4)) > P_MIN
    f = species_fractions(p.pdg)
    assert within_binomial(f[11], 0.5, N) and within_binomial(f[22], 0.5, N) and f[-11] == 0
    np.testing.assert_allclose(np.linalg.norm(p.dir, axis=1), 1.0, rtol=1e-12)
    c = p.dir[:, 2]
    assert ks_uniform(c, -math.tanh(1.5), math.tanh(1.5)) > P_MIN
    eta = np.arctanh(c)
    assert np.abs(eta).max() < 1.5
    phi = np.arctan2(p.dir[:, 1], p.dir[:, 0])
    assert ks_uniform(phi, -math.pi, math.pi) > P_MIN
    assert (p.pos == 0).all()


def test_serving_recipe():
    p = W.serving_batch(N, seed=11, event=5)
    assert (p.event == 5).all()
    assert p.E.min() >= 10.0 and p.E.max() <= 2e4
    # E^-2 on [10 MeV, 20 GeV]: 1/E is uniform
    assert ks_uniform(1.0 / p.E, 1.0 / 2e4, 1.0 / 10.0) > P_MIN
    f = species_fractions(p.pdg)
    for sp in (22, 11, -11):
        assert within_binomial(f[sp], 1 / 3, N), (sp, f[sp])
    # on the inner barrel face, on the ray from the origin along the direction
    np.testing.assert_allclose(np.hypot(p.pos[:, 0], p.pos[:, 1]), 300.0, rtol=1e-12)
    rhat = p.pos / np.linalg.norm(p.pos, axis=1, keepdims=True)
    np.testing.assert_allclose(rhat, p.dir, atol=1e-12)
    assert np.abs(np.arctanh(p.dir[:, 2])).max() < 1.5


def test_serving_batch_sizes():
    rng = np.random.default_rng(2)
    n = np.array([W.serving_batch_size(rng) for _ in range(N)])
    assert n.min() >= 10 and n.max() <= 10000
    # int() of a log-uniform draw x on [10, 10^4]: P(n <= k) = P(x < k + 1), exactly
    k = np.unique(n)
    cdf_want = np.log((k + 1) / 10.0) / math.log(1e3)
    cdf_got = np.searchsorted(np.sort(n), k, side="right") / N
    assert np.abs(cdf_got - cdf_want).max() < 1.95 / math.sqrt(N)  # KS bound at 0.1 %


def test_recipes_are_seeded():
    a, b = W.mixed(100, seed=9), W.mixed(100, seed=9)
    np.testing.assert_array_equal(a.E, b.E)
    np.testing.assert_array_equal(a.pdg, b.pdg)
    c = W.mixed(100, seed=10)
    assert not np.array_equal(a.E, c.E)
