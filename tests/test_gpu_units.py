"""Parity of the CUDA building blocks with the FP64 oracle, through the C ABI probes:
Philox words (bit-exact), tables and cuts (1e-12 FP64 / 1e-6 FP32 relative), inverse
range, navigation distances, and the samplers (FP64 to rounding, FP32 in distribution)."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2209_15445_gb300 import workloads as W

from gpu_common import make, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slab():
    need_gpu()
    return make(W.slab_calorimeter(), precision=0)


@pytest.fixture(scope="module")
def slab_o():
    return oracle.Oracle(W.slab_calorimeter())


@pytest.fixture(scope="module")
def barrel():
    need_gpu()
    return make(W.barrel_calorimeter(), field_T=3.8, precision=0)


@pytest.fixture(scope="module")
def barrel_o():
    return oracle.Oracle(W.barrel_calorimeter(), field_T=3.8)


def test_philox_bit_exact(slab):
    from paper_2209_15445_gb300 import adept as A
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, (5000, 4), dtype=np.uint64).astype(np.uint32)
    for key in [(0, 0), (1, 7), (0xFFFFFFFF, 0x12345678)]:
        rc, out = A.adept_probe_philox(slab.h, key, ctr)
        assert rc == 0
        for i in range(0, 5000, 97):
            assert np.array_equal(out[i], oracle.philox(ctr[i], key))


def test_cuts_match(slab, slab_o):
    from paper_2209_15445_gb300 import adept as A
    for m in range(2):
        rc, tc, kc = A.adept_get_cuts(slab.h, m)
        assert rc == 0
        otc, okc = slab_o.cuts(m)
        assert tc == pytest.approx(otc, rel=1e-12, abs=0) and kc == pytest.approx(okc, rel=1e-12, abs=0)


TABLES = [(0, 3), (1, 4), (2, 5)]


def test_table_nodes_fp64_and_fp32(slab, slab_o):
    from paper_2209_15445_gb300 import adept as A
    for s, nt in TABLES:
        for t in range(nt):
            for m in range(2):
                ref = slab_o.table(s, t, m)
                rc, g64 = A.adept_get_table(slab.h, s, t, m, 0)
                assert rc == 0
                np.testing.assert_allclose(g64, ref, rtol=1e-12, atol=1e-300)
                rc, g32 = A.adept_get_table(slab.h, s, t, m, 1)
                np.testing.assert_allclose(g32, ref.astype(np.float32).astype(np.float64), rtol=1.2e-7, atol=1e-300)


def test_interpolation_fp64_and_fp32(slab, slab_o):
    from paper_2209_15445_gb300 import adept as A
    rng = np.random.default_rng(2)
    E = np.exp(rng.uniform(math.log(1.001e-3), math.log(9.9e5), 4000))
    E = np.concatenate([E, oracle.node_energies()[1:-1]])
    for s, nt in TABLES:
        for t in range(nt):
            for m in range(2):
                ref = np.array([slab_o.interp(s, t, m, e) for e in E])
                rc, v64 = A.adept_probe_interp(slab.h, s, t, m, 0, E)
                assert rc == 0
                np.testing.assert_allclose(v64, ref, rtol=1e-12, atol=1e-300 + 1e-12 * np.abs(ref).max() * 1e-6)
                rc, v32 = A.adept_probe_interp(slab.h, s, t, m, 1, E)
                # FP32 lookup error relative to the magnitude of the bin's two nodes (a
                # relative error is undefined where an interval starts at zero, e.g. at the
                # pair threshold)
                node = slab_o.table(s, t, m)
                b = np.clip(np.floor((np.log(E) - math.log(1e-3)) * 32 / math.log(10)).astype(int), 0, 287)
                scale = np.maximum(np.abs(ref), np.maximum(np.abs(node[b]), np.abs(node[b + 1])))
                err = np.abs(v32 - ref) / np.maximum(scale, 1e-300)
                assert err.max() < 1e-6, (s, t, m, err.max())


def test_inverse_range(slab, slab_o):
    from paper_2209_15445_gb300 import adept as A
    rng = np.random.default_rng(3)
    for s in (1, 2):
        for m in range(2):
            Rn = slab_o.table(s, 1, m)
            R = np.exp(rng.uniform(math.log(Rn[0] * 0.5), math.log(Rn[-1]), 3000))
            ref = np.array([slab_o.inverse_range(s, m, r) for r in R])
            rc, g = A.adept_probe_inverse_range(slab.h, s, m, 0, R)
            assert rc == 0
            np.testing.assert_allclose(g, ref, rtol=1e-12, atol=0)
            rc, g32 = A.adept_probe_inverse_range(slab.h, s, m, 1, R)
            clear = R > Rn[0] * (1 + 1e-5)
            # FP32 range nodes: the inversion is accurate to a few float ulps of R / (dR/dlnE)
            np.testing.assert_allclose(g32[clear], ref[clear], rtol=2e-5)
            assert np.all(g32[R < Rn[0] * (1 - 1e-5)] == 0.0)


def rand_dirs(rng, n):
    c = rng.uniform(-1, 1, n)
    ph = rng.uniform(0, 2 * math.pi, n)
    s = np.sqrt(1 - c * c)
    return np.stack([s * np.cos(ph), s * np.sin(ph), c], 1)


def check_distances(tr, orc, pos, d, T, q, prec, tol):
    from paper_2209_15445_gb300 import adept as A
    vol = np.array([orc.locate(p, u) for p, u in zip(pos, d)], np.int32)
    keep = vol >= 0
    pos, d, T, q, vol = pos[keep], d[keep], T[keep], q[keep], vol[keep]
    rc, s, nx = A.adept_probe_distance(tr.h, prec, pos, d, vol, T, q)
    assert rc == 0
    ref = [orc.helix_distance(t_, int(q_), p, u, v) if q_ != 0 else orc.distance(p, u, v)
           for p, u, v, t_, q_ in zip(pos, d, vol, T, q)]
    rs = np.array([r[0] for r in ref])
    rn = np.array([r[1] for r in ref])
    agree = np.abs(s - rs) <= tol * np.maximum(1.0, rs)
    if prec == 1 and np.any(q != 0):
        # FP32 helix: phases good to ~1e-7 rad, i.e. 1e-6 of rho/u_T in path, plus rounding
        uT = np.hypot(d[:, 0], d[:, 1])
        rho = np.sqrt(T * (T + 2 * 0.51099895)) * uT / (0.299792458 * orc.field_T)
        agree |= np.abs(s - rs) <= 1e-6 * rho / np.maximum(uT, 1e-9) + 1e-5 * np.maximum(1.0, rs)
    assert agree.mean() > 0.999, (np.abs(s - rs) / np.maximum(1, rs)).max()
    assert (nx[agree] == rn[agree]).all()
    return len(vol)


def test_distances_slab_straight(slab, slab_o):
    rng = np.random.default_rng(4)
    n = 4000
    pos = np.stack([rng.uniform(-190, 190, n), rng.uniform(-190, 190, n), rng.uniform(0.01, 399.99, n)], 1)
    d = rand_dirs(rng, n)
    assert check_distances(slab, slab_o, pos, d, np.ones(n), np.zeros(n, np.int32), 0, 1e-12) > 3000
    assert check_distances(slab, slab_o, pos, d, np.ones(n), np.zeros(n, np.int32), 1, 2e-6) > 3000


def test_distances_barrel_straight_and_helix(barrel, barrel_o):
    rng = np.random.default_rng(5)
    n = 4000
    r = rng.uniform(10, 1790, n)
    ph = rng.uniform(0, 2 * math.pi, n)
    pos = np.stack([r * np.cos(ph), r * np.sin(ph), rng.uniform(-2900, 2900, n)], 1)
    d = rand_dirs(rng, n)
    T = np.exp(rng.uniform(math.log(0.05), math.log(5e3), n))
    q0 = np.zeros(n, np.int32)
    assert check_distances(barrel, barrel_o, pos, d, T, q0, 0, 1e-11) > 3000
    q = rng.choice([-1, 1], n).astype(np.int32)
    assert check_distances(barrel, barrel_o, pos, d, T, q, 0, 1e-9) > 3000
    assert check_distances(barrel, barrel_o, pos, d, T, q, 1, 1e-4) > 3000


SAMPLERS = [(0, 0, 2.0), (0, 0, 0.05), (1, 0, 50.0), (2, 0, 30.0), (3, 0, 30.0), (4, 0, 100.0), (5, 0, 3.0),
            (6, 0, 0.0), (4, 1, 5.0), (2, 1, 3.0)]


@pytest.mark.parametrize("which,m,E", SAMPLERS)
def test_samplers_fp64_match_oracle(slab, slab_o, which, m, E):
    from paper_2209_15445_gb300 import adept as A
    n = 3000
    rc, g = A.adept_probe_sample(slab.h, which, m, 0, E, 7, n)
    assert rc == 0
    ref = slab_o.sample(which, m, E, n, seed=1, event=7)
    # same Philox words, FP64 on both sides: equal up to libm rounding
    np.testing.assert_allclose(g, ref, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("which,m,E", SAMPLERS)
def test_samplers_fp32_same_distribution(slab, slab_o, which, m, E):
    from paper_2209_15445_gb300 import adept as A
    n = 20000
    rc, g = A.adept_probe_sample(slab.h, which, m, 1, E, 9, n)
    assert rc == 0
    ref = slab_o.sample(which, m, E, n, seed=1, event=11)  # an independent stream
    for col in (1, 5, 8):  # parent energy, secondary energy, secondary polar cosine
        a, b = g[:, col], ref[:, col]
        if np.ptp(b) == 0:
            assert np.allclose(a, b, rtol=1e-6)
            continue
        assert stats.ks_2samp(a, b).pvalue > 1e-4, col
    # energy bookkeeping stays FP64-exact in the split form
    if which in (0, 2, 3, 4):
        np.testing.assert_allclose(g[:, 1] + g[:, 5], E, rtol=1e-15)
