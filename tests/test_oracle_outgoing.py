"""Pins of the oracle's outgoing-particle list (the particles the calorimeter hands back,
paper Sec. 4): it accounts for the leaked energy of every event exactly, every record sits
on the world boundary heading out, primaries submitted outside come back unchanged, and
the list does not depend on the thread count."""
import numpy as np

import oracle
from paper_2209_15445_gb300 import workloads as W

ME = 0.51099895


def per_event_energy(out, n_events):
    e = out[:, 2] + np.where(out[:, 1] == -11, 2 * ME, 0.0)
    return np.bincount(out[:, 0].astype(int), weights=e, minlength=n_events)


def test_outgoing_list_accounts_for_leaked_energy():
    o = oracle.Oracle(W.slab_calorimeter())
    prim = W.mixed(60, seed=41)
    r = o.transport(prim, outgoing=100000)
    out = r["outgoing"]
    assert len(out) > 50
    np.testing.assert_allclose(per_event_energy(out, len(r["leaked"])), r["leaked"], rtol=1e-12, atol=1e-12)


def test_outgoing_particles_leave_through_the_world_boundary():
    geom = W.slab_calorimeter()
    o = oracle.Oracle(geom)
    r = o.transport(W.electrons(50, 1e4), outgoing=100000)
    out = r["outgoing"]
    pos, d = out[:, 3:6], out[:, 6:9]
    zmax = sum(geom.sub_thickness) * geom.n_layers
    back = np.isclose(pos[:, 2], zmax, atol=1e-9) & (d[:, 2] > 0)
    front = np.isclose(pos[:, 2], 0.0, atol=1e-9) & (d[:, 2] < 0)
    side_x = np.isclose(np.abs(pos[:, 0]), geom.half_xy, atol=1e-6) & (pos[:, 0] * d[:, 0] > 0)
    side_y = np.isclose(np.abs(pos[:, 1]), geom.half_xy, atol=1e-6) & (pos[:, 1] * d[:, 1] > 0)
    assert np.all(back | front | side_x | side_y)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)


def test_primaries_outside_come_back_unchanged():
    o = oracle.Oracle(W.slab_calorimeter())
    n = 5
    prim = W.Primaries(np.array([22, 11, -11, 22, 11], np.int32), np.array([1.0, 2.0, 3.0, 4.0, 5.0]),
                       np.array([[0.0, 0.0, -10.0 - k] for k in range(n)]),
                       np.tile([0.0, 0.0, -1.0], (n, 1)), np.arange(n, dtype=np.uint32))
    r = o.transport(prim, outgoing=100)
    out = r["outgoing"]
    out = out[np.argsort(out[:, 0])]
    assert len(out) == n
    np.testing.assert_array_equal(out[:, 1], prim.pdg)
    np.testing.assert_array_equal(out[:, 2], prim.E)
    np.testing.assert_array_equal(out[:, 3:6], prim.pos)


def test_outgoing_list_is_thread_independent():
    o = oracle.Oracle(W.barrel_calorimeter(), field_T=3.8)
    prim = W.barrel_primaries(40, seed=2)
    a = o.transport(prim, outgoing=100000, n_threads=1)["outgoing"]
    b = o.transport(prim, outgoing=100000, n_threads=4)["outgoing"]
    key = lambda x: x[np.lexsort(x.T[::-1])]
    np.testing.assert_array_equal(key(a), key(b))
