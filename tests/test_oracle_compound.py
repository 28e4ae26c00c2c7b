"""Pins of compound materials in the oracle (the paper's PbWO4, Sec. 2.2).

* PDG values for lead tungstate: X0 = 7.39 g/cm^2 and <Z/A> = 0.41315.
* A "compound" of one element is that element: every table equal to the elemental one.
* Mixture rules, checked against separate elemental oracles: mass attenuation for Compton
  and photoabsorption and 1/X0 per g/cm^2 are the mass-fraction-weighted sums.
* Full transport in the paper's PbWO4 / lAr calorimeter conserves energy per event.
"""
import numpy as np
import pytest

import oracle
from paper_2209_15445_gb300 import workloads as W
from published import published

ELEMENTS = {82: ("Pb", 207.2, 11.35, 823.0), 74: ("W", 183.84, 19.3, 727.0), 8: ("O", 15.999, 1.141, 95.0)}


def slab_of(mat):
    return W.Geometry(kind=0, n_layers=2, materials=[mat, W.LAR], sub_materials=[0, 1], sub_thickness=[2.3, 5.7],
                      half_xy=200.0)


def mass_fractions(m):
    tot = sum(a * n for _, a, n in m.elements)
    return {z: a * n / tot for z, a, n in m.elements}


@pytest.fixture(scope="module")
def pbwo4():
    return oracle.Oracle(slab_of(W.PBWO4))


def test_pdg_radiation_length_of_lead_tungstate(pbwo4):
    x0_g_cm2 = 1.0 / pbwo4.inv_X0(0) / 10.0 * W.PBWO4.density
    assert abs(x0_g_cm2 / published("x0_PbWO4") - 1.0) < 0.01, x0_g_cm2


def test_pdg_z_over_a_of_lead_tungstate():
    w = mass_fractions(W.PBWO4)
    zoa = sum(w[z] * z / a for z, a, _ in W.PBWO4.elements)
    assert abs(zoa - published("ZoA_PbWO4")) < 2e-4


def test_one_element_compound_is_the_element():
    pb = W.PB
    pb_c = W.Material("Pb as a compound", 0, 0.0, pb.density, pb.I_eV, elements=((82, 207.2, 1.0),))
    a, b = oracle.Oracle(slab_of(pb)), oracle.Oracle(slab_of(pb_c))
    for sp, nt in ((0, 3), (1, 4), (2, 5)):
        for t in range(nt):
            np.testing.assert_allclose(b.table(sp, t, 0), a.table(sp, t, 0), rtol=1e-14, atol=0)
    assert a.cuts(0) == pytest.approx(b.cuts(0), rel=1e-14, abs=0)


def elemental(z, density=1.0):
    name, A, _, I = ELEMENTS[z]
    return oracle.Oracle(slab_of(W.Material(name, z, A, density, I)))


@pytest.mark.parametrize("E", [0.05, 0.3, 2.0, 50.0])
def test_mixture_rules(pbwo4, E):
    w = mass_fractions(W.PBWO4)
    rho = W.PBWO4.density
    els = {z: elemental(z) for z in w}  # density 1 g/cm^3: values per g/cm^2
    for f in ("mu_compton", "mu_photo"):
        mix = sum(w[z] * getattr(els[z], f)(0, E) for z in w)
        assert getattr(pbwo4, f)(0, E) / rho == pytest.approx(mix, rel=1e-12, abs=0), f
    mix = sum(w[z] * els[z].inv_X0(0) for z in w)
    assert pbwo4.inv_X0(0) / rho == pytest.approx(mix, rel=1e-12, abs=0)


def test_transport_in_the_papers_calorimeter():
    geom = W.pbwo4_calorimeter()
    o = oracle.Oracle(geom)
    prim = W.electrons(20, 1e4)
    r = o.transport(prim)
    tot = r["edep"].sum(1) + r["leaked"] + r["killed"]
    np.testing.assert_allclose(tot, prim.E, rtol=1e-12)
    # 13 X0 of PbWO4 (X0 = 8.9 mm) and 2 X0 of argon: the shower peaks in the first half
    e = r["edep"].sum(0)
    assert e[: geom.n_bins // 2].sum() > 0.5 * e.sum()
