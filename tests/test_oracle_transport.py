"""Transport-level pins of the oracle: per-event energy conservation, thread-count
independence, the exponential attenuation law, CSDA depth, positron annihilation at rest,
looper caps, and consistency of the generation histogram."""
import math

import numpy as np
import pytest

import oracle
from paper_2209_15445_gb300 import workloads as w

ME = 0.51099895


def primary_energy(prim):
    return prim.E + np.where(prim.pdg == -11, 2 * ME, 0.0)


def ledger(res):
    return res["edep"].sum(axis=1) + res["leaked"] + res["killed"]


def test_energy_conservation_slab(slab_oracle):
    p = w.mixed(300, seed=11)
    r = slab_oracle.transport(p, n_threads=4)
    E0 = primary_energy(p)
    assert np.allclose(ledger(r), E0, rtol=1e-12, atol=0)
    assert r["steps"].sum() > 0 and np.all(r["killed"] == 0)


def test_energy_conservation_barrel_field(barrel_oracle):
    p = w.barrel_primaries(40, seed=12)
    p = p.take(np.arange(40))
    p.E[:] = np.minimum(p.E, 3000.0)
    r = barrel_oracle.transport(p, n_threads=4)
    assert np.allclose(ledger(r), primary_energy(p), rtol=1e-12, atol=0)


def test_results_independent_of_thread_count(slab_oracle):
    p = w.mixed(64, seed=13)
    a = slab_oracle.transport(p, n_threads=1, max_gen=2000)
    b = slab_oracle.transport(p, n_threads=7, max_gen=2000)
    assert np.array_equal(a["edep"], b["edep"])
    assert np.array_equal(a["gen_hist"], b["gen_hist"])
    assert np.array_equal(a["steps"], b["steps"])
    assert a["gen_hist"].sum() == a["steps"].sum()


def test_exponential_attenuation_compton_only():
    """With only Compton scattering and no field, a pencil beam of N photons crossing a
    slab of thickness L interacts in its first step with probability 1 - exp(-mu L);
    interacting photons survive to step again (generation 1), the others leave."""
    L = 20.0
    g = w.Geometry(kind=0, n_layers=1, materials=[w.PB], sub_materials=[0], sub_thickness=[L], half_xy=1e7)
    o = oracle.Oracle(g)
    n = 20000
    E = 1.0
    p = w.Primaries(np.full(n, 22, np.int32), np.full(n, E), np.zeros((n, 3)),
                    np.tile([0.0, 0.0, 1.0], (n, 1)), np.arange(n, dtype=np.uint32))
    r = o.transport(p, process_mask=oracle.P_COMPT, max_gen=4, n_threads=8)
    mu = o.mu_compton(0, E)
    # the table interpolates mu linearly in ln E; at a node-exact energy it is exact
    mu_tab = o.interp(0, 0, 0, E)
    pint = 1 - math.exp(-mu_tab * L)
    k = int(r["gen_hist"][1, 0])
    sd = math.sqrt(n * pint * (1 - pint))
    assert abs(k - n * pint) < 5 * sd
    assert abs(mu_tab / mu - 1) < 2e-3


def test_csda_depth_without_discrete_processes():
    """With the discrete processes off and no field an electron runs straight and loses its
    energy continuously: everything is deposited and the deepest deposit lies at R(E)."""
    L = 100.0
    g = w.Geometry(kind=0, n_layers=200, materials=[w.PB], sub_materials=[0], sub_thickness=[0.5], half_xy=1e7)
    o = oracle.Oracle(g)
    E = 50.0
    p = w.electrons(4, E)
    r = o.transport(p, process_mask=0x80000000, n_threads=1)
    assert np.allclose(r["edep"].sum(axis=1), E, rtol=1e-13)
    R = o.interp(1, 1, 0, E)
    deepest = np.nonzero(r["edep"][0])[0].max()
    assert deepest == int(R / 0.5)


def test_positron_below_cut_annihilates_at_rest(slab_oracle):
    n = 50
    p = w.Primaries(np.full(n, -11, np.int32), np.full(n, 5e-4), np.tile([0.0, 0.0, 1.0], (n, 1)),
                    np.tile([0.0, 0.0, 1.0], (n, 1)), np.arange(n, dtype=np.uint32))
    r = slab_oracle.transport(p, max_gen=3)
    assert int(r["gen_hist"][0, 2]) == n and int(r["gen_hist"][1, 0]) == 2 * n  # two photons each
    assert np.allclose(ledger(r), 5e-4 + 2 * ME, rtol=1e-13)


def test_step_cap_kills_and_accounts():
    p = w.electrons(5, 1000.0)
    o = oracle.Oracle(w.slab_calorimeter())
    r = o.transport(p, max_steps=3)
    assert np.all(r["killed"] > 0)
    assert np.allclose(ledger(r), 1000.0, rtol=1e-12)


def test_vacuum_looper_cap_barrel():
    """A low-p_T electron launched in the inner vacuum along phi with no z motion circles
    forever: the vacuum-step cap must kill it and account its energy."""
    o = oracle.Oracle(w.barrel_calorimeter(), field_T=3.8)
    p = w.Primaries(np.array([11], np.int32), np.array([5.0]), np.array([[100.0, 0.0, 0.0]]),
                    np.array([[0.0, 1.0, 0.0]]), np.array([0], np.uint32))
    r = o.transport(p, max_vacuum_steps=50)
    assert r["killed"][0] == pytest.approx(5.0, abs=0)
    assert int(r["steps"][1]) == 51


def test_straight_gamma_leaks_through_vacuum_barrel():
    o = oracle.Oracle(w.barrel_calorimeter(), field_T=3.8)
    p = w.Primaries(np.array([22], np.int32), np.array([100.0]), np.zeros((1, 3)),
                    np.array([[0.0, 0.0, 1.0]]), np.array([0], np.uint32))
    r = o.transport(p)
    assert r["leaked"][0] == 100.0 and int(r["steps"][0]) == 1


def test_a_step_cut_short_by_the_step_limit_does_not_interact():
    """Stepping reading (C9): a discrete interaction happens only where the sampled
    interaction length ends the step; a step cut short by the range-based limit
    s_max = max(0.2 R, min(R, 1 mm)) or by a boundary only loses energy continuously.
    e- of 3.9 T_c in bulk Pb with Moller ionisation alone: delta rays (at most T/2 < 2 T_c)
    cannot ionise in turn, so the delta rays counted are the primaries' interactions. Along
    the primary's interaction-free slowing-down steps s_k, with the cross section at each
    pre-step energy, I = sum Sigma(T_k) s_k; the mean count per primary lies between
    1 - exp(-I) (a first interaction) and I (an interaction only lowers the cross section).
    Interacting at the end of every limited step would give about one per 1 mm step."""
    g = w.Geometry(kind=0, n_layers=1, materials=[w.PB], sub_materials=[0], sub_thickness=[1000.0], half_xy=1e6)
    o = oracle.Oracle(g)
    Tc = o.cuts(0)[0]
    T0 = 3.9 * Tc

    def energy_at_range(R):
        lo, hi = 1e-3, T0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if o.interp(1, 1, 0, mid) < R else (lo, mid)
        return 0.5 * (lo + hi)

    I, T = 0.0, T0
    while T > 2.0 * Tc:
        R = o.interp(1, 1, 0, T)
        s = R if R <= 1.0 else max(0.2 * R, 1.0)
        I += o.interp(1, 2, 0, T) * s
        if s >= R:
            break
        T = energy_at_range(R - s)
    n = 4000
    r = o.transport(w.electrons(n, T0), process_mask=oracle.P_EIONI)
    mean = int(r["created"][1]) / n
    sd = math.sqrt(I / n)
    assert 1.0 - math.exp(-I) - 4 * sd <= mean <= I + 4 * sd, (mean, I)


def test_fraction_of_positrons_annihilating_in_flight():
    """Stepping reading (C9), with a process that ends the track: 10 MeV e+ in bulk Pb with
    annihilation as the only discrete process (photons do not interact, so all of them
    leave). The positron survives its k-th interaction-free slowing-down step s_k with
    probability exp(-Sigma(T_k) s_k), Sigma at the pre-step energy, so it annihilates in flight
    with probability 1 - exp(-I), I = sum Sigma(T_k) s_k; otherwise at rest, into two photons
    of exactly m_e c^2 each."""
    g = w.Geometry(kind=0, n_layers=1, materials=[w.PB], sub_materials=[0], sub_thickness=[1000.0], half_xy=1e6)
    o = oracle.Oracle(g)
    T0 = 10.0

    def energy_at_range(R, hi):
        lo = 1e-6
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if o.interp(2, 1, 0, mid) < R else (lo, mid)
        return 0.5 * (lo + hi)

    I, T = 0.0, T0
    while T >= 1e-3:
        R = o.interp(2, 1, 0, T)
        s = R if R <= 1.0 else max(0.2 * R, 1.0)
        I += o.interp(2, 4, 0, T) * s
        if s >= R:
            break
        T = energy_at_range(R - s, T)
    n = 4000
    p = w.Primaries(np.full(n, -11, np.int32), np.full(n, T0), np.zeros((n, 3)), np.tile([0.0, 0.0, 1.0], (n, 1)),
                    np.arange(n, dtype=np.uint32))
    r = o.transport(p, process_mask=oracle.P_ANNIH, outgoing=4 * n)
    photons = r["outgoing"][r["outgoing"][:, 1] == 22]
    assert len(photons) == 2 * n
    in_flight = np.count_nonzero(np.abs(photons[:, 2] - ME) > 1e-9) / 2 / n
    want = 1.0 - math.exp(-I)
    assert abs(in_flight - want) <= 4 * math.sqrt(want * (1 - want) / n), (in_flight, want)
