"""Pins of the oracle's navigation (slab and tube stacks) and helix propagation:
brute-force marching with the point locator, chord sums, and analytic helix facts."""
import math

import numpy as np
import pytest

import oracle
from paper_2209_15445_gb300 import workloads as w


def test_locate_slab(slab_oracle):
    o = slab_oracle
    z = np.array([0.0, 0.0, 1.0])
    assert o.locate([0, 0, 1.0], z) == 0
    assert o.locate([0, 0, 3.0], z) == 1
    assert o.locate([0, 0, 2.3], z) == 1 and o.locate([0, 0, 2.3], -z) == 0
    assert o.locate([0, 0, 0.0], z) == 0 and o.locate([0, 0, 0.0], -z) == -1
    assert o.locate([0, 0, 399.0], z) == 99
    assert o.locate([0, 0, -1.0], z) == -1 and o.locate([250.0, 0, 5.0], z) == -1
    assert o.locate([0, 0, 8.0 * 10 + 1.0], z) == 20


def test_locate_barrel(barrel_oracle):
    o = barrel_oracle
    assert o.n_vol == 1 + 20 * 4 + 19
    x = np.array([1.0, 0.0, 0.0])
    assert o.locate([100.0, 0, 0], x) == 0
    assert o.locate([300.1, 0, 0], x) == 1       # Si of layer 0
    assert o.locate([310.0, 0, 0], x) == 2       # Fe
    assert o.locate([300.0, 0, 0], x) == 1 and o.locate([300.0, 0, 0], -x) == 0
    assert o.locate([330.0, 0, 0], x) == 5       # gap after layer 0
    assert o.locate([1799.0, 0, 0], x) == o.n_vol - 1
    assert o.locate([1801.0, 0, 0], x) == -1 and o.locate([500.0, 0, 3001.0], x) == -1


def brute_first_exit(o, p, u, vol, smax=5000.0, h=0.01):
    p = np.asarray(p, float); u = np.asarray(u, float)
    s = 0.0
    while s < smax:
        s1 = s + h
        if o.locate(p + s1 * u, u) != vol:
            lo, hi = s, s1
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                if o.locate(p + mid * u, u) != vol:
                    hi = mid
                else:
                    lo = mid
            return hi, o.locate(p + hi * u + 1e-9 * u, u)
        s = s1
    return None, None


def rand_dir(rng):
    c = rng.uniform(-1, 1); ph = rng.uniform(0, 2 * math.pi); s = math.sqrt(1 - c * c)
    return np.array([s * math.cos(ph), s * math.sin(ph), c])


def test_slab_distance_vs_brute_force(slab_oracle):
    rng = np.random.default_rng(2)
    o = slab_oracle
    for _ in range(60):
        p = np.array([rng.uniform(-190, 190), rng.uniform(-190, 190), rng.uniform(0.1, 399.9)])
        u = rand_dir(rng)
        vol = o.locate(p, u)
        s, nx = o.distance(p, u, vol)
        sb, nb = brute_first_exit(o, p, u, vol, h=0.05)
        assert s == pytest.approx(sb, abs=1e-9)
        assert nx == nb


def test_barrel_distance_vs_brute_force(barrel_oracle):
    rng = np.random.default_rng(3)
    o = barrel_oracle
    g = w.barrel_calorimeter()
    radii = []
    for r0 in g.layer_r:
        radii.append(r0)
        for t in np.cumsum(g.sub_thickness):
            radii.append(r0 + t)
    for _ in range(60):
        r = rng.uniform(10, 1790); ph = rng.uniform(0, 2 * math.pi)
        p = np.array([r * math.cos(ph), r * math.sin(ph), rng.uniform(-2900, 2900)])
        u = rand_dir(rng)
        vol = o.locate(p, u)
        s, nx = o.distance(p, u, vol)
        sb, nb = brute_first_exit(o, p, u, vol, h=0.05)
        q = p + s * u
        r = math.hypot(q[0], q[1])
        # the locator's on-surface band (1e-9 relative in r) blurs the march by
        # band / |dr/ds| along the ray
        drds = abs(q[0] * u[0] + q[1] * u[1]) / r
        assert s == pytest.approx(sb, abs=1e-9 + 4e-9 * 1800.0 / max(drds, 1e-6))
        assert nx == nb
        surfaces = [abs(r - b) for b in radii] + [abs(abs(q[2]) - 3000.0)]
        assert min(surfaces) < 1e-9 * 3000.0


def test_chord_sum(slab_oracle):
    o = slab_oracle
    c = 0.95  # stays inside the 200 mm half width over 400 mm of depth
    u = np.array([math.sqrt(1 - c * c), 0.0, c])
    p = np.zeros(3)
    vol = o.locate(p, u)
    total = 0.0
    while vol >= 0:
        s, nx = o.distance(p, u, vol)
        p = p + s * u
        total += s
        vol = nx
    assert total == pytest.approx(400.0 / c, rel=1e-12, abs=0)


def test_helix_radius_turn_and_sense():
    B = 1.0
    T = 2000.0
    pm = math.sqrt(T * (T + 2 * 0.51099895))
    rho = pm / (0.299792458 * B)  # p_T[GeV] = 0.3 B[T] R[m]
    u = np.array([1.0, 0.0, 0.0])
    p0 = np.zeros(3)
    # electron (q = -1) in B along +z: F = q v x B points along +y
    p1, u1 = oracle.helix_move(B, T, -1, 1.0, p0, u)
    assert p1[1] > 0 and np.sign(np.cross(u, [0, 0, B])[1] * -1) > 0
    # quarter turn: displacement rho * sqrt(2), direction rotated by 90 degrees
    p1, u1 = oracle.helix_move(B, T, -1, 0.5 * math.pi * rho, p0, u)
    assert np.linalg.norm(p1) == pytest.approx(rho * math.sqrt(2), rel=1e-12, abs=0)
    assert np.allclose(u1, [0, 1, 0], atol=1e-12)
    # full turns with a z component: xy returns, z advances linearly, p_T conserved
    c = 0.3
    u = np.array([math.sqrt(1 - c * c), 0.0, c])
    s_turn = 2 * math.pi * rho  # transverse radius rho*u_T, covered at rate u_T per unit path
    p1, u1 = oracle.helix_move(B, T, 1, 3 * s_turn, p0, u)
    assert np.allclose(p1[:2], 0.0, atol=1e-9 * rho)
    assert p1[2] == pytest.approx(3 * s_turn * c, rel=1e-14, abs=0)
    assert np.allclose(u1, u, atol=1e-12)
    # many small steps equal one large step (the helix is exact)
    q = p0.copy(); v = u.copy()
    for _ in range(100):
        q, v = oracle.helix_move(B, T, 1, 10.0, q, v)
    p1, u1 = oracle.helix_move(B, T, 1, 1000.0, p0, u)
    assert np.allclose(q, p1, atol=1e-9) and np.allclose(v, u1, atol=1e-12)
    assert math.hypot(v[0], v[1]) == pytest.approx(math.sqrt(1 - c * c), rel=1e-12, abs=0)


def brute_helix_exit(o, T, q, B, p, u, vol, smax, h):
    s = 0.0
    pp, uu = np.array(p, float), np.array(u, float)
    while s < smax:
        p1, u1 = oracle.helix_move(B, T, q, s + h, p, u)
        if o.locate(p1, u1) != vol:
            lo, hi = s, s + h
            for _ in range(70):
                mid = 0.5 * (lo + hi)
                pm, um = oracle.helix_move(B, T, q, mid, p, u)
                if o.locate(pm, um) != vol:
                    hi = mid
                else:
                    lo = mid
            return hi
        s += h
    return None


@pytest.mark.parametrize("geom,B", [("barrel", 3.8), ("slab", 1.0)])
def test_helix_distance_vs_brute_force(geom, B):
    g = w.barrel_calorimeter() if geom == "barrel" else w.slab_calorimeter()
    o = oracle.Oracle(g, field_T=B)
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(200):
        if geom == "barrel":
            r = rng.uniform(290, 1790); ph = rng.uniform(0, 2 * math.pi)
            p = np.array([r * math.cos(ph), r * math.sin(ph), rng.uniform(-2900, 2900)])
        else:
            p = np.array([rng.uniform(-190, 190), rng.uniform(-190, 190), rng.uniform(0.1, 399.9)])
        u = rand_dir(rng)
        T = math.exp(rng.uniform(math.log(0.5), math.log(500.0)))
        q = int(rng.choice([-1, 1]))
        vol = o.locate(p, u)
        s, nx = o.helix_distance(T, q, p, u, vol)
        if s > 400.0:
            continue
        sb = brute_helix_exit(o, T, q, B, p, u, vol, s + 5.0, h=min(0.05, s / 4 + 1e-3))
        qq, uq = oracle.helix_move(B, T, q, s, p, u)
        r = math.hypot(qq[0], qq[1])
        rate = abs(qq[0] * uq[0] + qq[1] * uq[1]) / r if geom == "barrel" else 1.0
        assert sb is not None and s == pytest.approx(sb, abs=1e-8 + 4e-9 * 1800.0 / max(rate, 1e-6))
        pe, ue = oracle.helix_move(B, T, q, s + 1e-7, p, u)
        assert o.locate(pe, ue) == nx
        checked += 1
    assert checked > 50
