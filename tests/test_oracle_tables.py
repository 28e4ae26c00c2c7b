"""Pins of the oracle's energy grid, tables, range integration, inverse range and cuts."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2209_15445_gb300 import workloads as w

PB, LAR = 0, 1


def test_grid():
    E = oracle.node_energies()
    assert len(E) == 289
    assert E[0] == pytest.approx(1e-3, rel=1e-15, abs=0) and E[-1] == pytest.approx(1e6, rel=1e-13, abs=0)
    assert np.allclose(np.diff(np.log(E)), math.log(10) / 32, rtol=1e-12, atol=0)


def test_tables_equal_closed_forms_at_nodes(slab_oracle):
    E = oracle.node_energies()
    o = slab_oracle
    for m in (PB, LAR):
        Tc, kc = o.cuts(m)
        g = [o.table(0, t, m) for t in range(3)]
        for i in range(0, 289, 7):
            assert g[0][i] == o.mu_compton(m, E[i])
            assert g[1][i] == o.mu_pair(m, E[i])
            assert g[2][i] == o.mu_photo(m, E[i])
            # interpolation reproduces the nodes
            assert o.interp(0, 0, m, E[i]) == pytest.approx(g[0][i], rel=1e-13, abs=0)
        e = [o.table(1, t, m) for t in range(4)]
        p = [o.table(2, t, m) for t in range(5)]
        for i in range(0, 289, 7):
            assert e[0][i] == o.dedx_col(m, E[i], Tc, 0) + o.dedx_rad(m, E[i], kc)
            assert e[2][i] == o.lambda_ioni(m, E[i], Tc, 0)
            assert e[3][i] == o.lambda_brem(m, E[i], kc)
            assert p[0][i] == o.dedx_col(m, E[i], Tc, 1) + o.dedx_rad(m, E[i], kc)
            assert p[2][i] == o.lambda_ioni(m, E[i], Tc, 1)
            assert p[4][i] == o.lambda_annih(m, E[i])


def test_interpolation_is_linear_in_lnE(slab_oracle):
    E = oracle.node_energies()
    v = slab_oracle.table(1, 2, PB)
    for i in (10, 100, 200):
        for t in (0.25, 0.5, 0.9):
            e = math.exp(math.log(E[i]) + t * (math.log(E[i + 1]) - math.log(E[i])))
            assert slab_oracle.interp(1, 2, PB, e) == pytest.approx(v[i] + t * (v[i + 1] - v[i]), rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("species,positron", [(1, 0), (2, 1)])
def test_range_is_integral_of_inverse_stopping_power(slab_oracle, species, positron):
    o = slab_oracle
    E = oracle.node_energies()
    for m in (PB, LAR):
        Tc, kc = o.cuts(m)
        S = lambda T: o.dedx_col(m, T, Tc, positron) + o.dedx_rad(m, T, kc)
        R = o.table(species, 1, m)
        assert R[0] == pytest.approx(E[0] / (2 * S(E[0])), rel=1e-14, abs=0)
        assert np.all(np.diff(R) > 0)
        for i in (1, 40, 120, 200, 288):
            pts = [math.log(x) for x in (2 * Tc, kc) if E[0] < x < E[i]]
            v, _ = integrate.quad(lambda t: math.exp(t) / S(math.exp(t)), math.log(E[0]), math.log(E[i]),
                                  epsabs=0, epsrel=1e-11, limit=500, points=pts or None)
            assert R[i] == pytest.approx(R[0] + v, rel=2e-6, abs=0)


def test_inverse_range_closure(slab_oracle):
    rng = np.random.default_rng(1)
    for sp in (1, 2):
        for m in (PB, LAR):
            for E in np.exp(rng.uniform(math.log(1.001e-3), math.log(9e5), 200)):
                R = slab_oracle.interp(sp, 1, m, E)
                assert slab_oracle.inverse_range(sp, m, R) == pytest.approx(E, rel=1e-12, abs=0)
            R0 = slab_oracle.table(sp, 1, m)[0]
            assert slab_oracle.inverse_range(sp, m, 0.5 * R0) == 0.0


def test_cuts_solve_their_definitions(slab_oracle):
    o = slab_oracle
    for m in (PB, LAR):
        Tc, kc = o.cuts(m)
        assert 0.99e-3 <= Tc <= 1e4 and 0.99e-3 <= kc <= 1e4
        assert o.interp(3, 0, m, Tc) == pytest.approx(0.7, rel=1e-12, abs=0)
        mu = o.interp(0, 0, m, kc) + o.interp(0, 1, m, kc) + o.interp(0, 2, m, kc)
        assert 5.0 / mu == pytest.approx(0.7, rel=1e-12, abs=0)
    # lead stops electrons faster than argon: a higher threshold for the same range
    assert o.cuts(PB)[0] > o.cuts(LAR)[0] and o.cuts(PB)[1] > o.cuts(LAR)[1]


def test_cut_clamps():
    g = w.Geometry(kind=0, n_layers=1, materials=[w.LAR], sub_materials=[0], sub_thickness=[10.0], half_xy=100.0)
    tiny = oracle.Oracle(g, range_cut_mm=1e-9)
    # below the first grid node the inversion stops at the node (1 keV)
    e0 = oracle.node_energies()[0]
    assert tiny.cuts(0) == (e0, e0)
    huge = oracle.Oracle(g, range_cut_mm=1e9)
    assert huge.cuts(0)[0] == 1e4
