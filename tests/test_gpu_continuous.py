"""Parity of the optional continuous physics (multiple scattering, loss fluctuations) with
the FP64 oracle: the device samplers draw by draw, then full transport (per-generation
queue sizes exactly in FP64, showers per layer in both forms, secondaries and step-length
distributions)."""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2209_15445_gb300 import workloads as W

from gpu_common import make, need_gpu
from test_gpu_transport import gen_log, gpu_run, layer_check, primary_energy

pytestmark = pytest.mark.gpu
BOTH = 3  # ADEPT_PHYS_MSC | ADEPT_PHYS_FLUCT


@pytest.fixture(scope="module")
def slab():
    need_gpu()
    tr = make(W.slab_calorimeter(), precision=0)
    yield tr
    tr.close()


@pytest.fixture(scope="module")
def slab_o():
    return oracle.Oracle(W.slab_calorimeter())


DEFLECT = [(0, 50.0, 0.05), (0, 5.0, 0.01), (1, 1.0, 0.3), (0, 0.01, 1.0)]
FLUCT = [(1, 0, 1000.0, 1.0), (1, 0, 2.0, 0.02), (2, 0, 0.2, 0.005), (2, 1, 30.0, 2.0)]


@pytest.mark.parametrize("m,T,s", DEFLECT)
def test_deflection_fp64_matches_oracle(slab, slab_o, m, T, s):
    from paper_2209_15445_gb300 import adept as A
    n = 4000
    rc, g = A.adept_probe_continuous(slab.h, 0, 1, m, 0, T, s, 7, n)
    assert rc == 0
    ref = slab_o.sample_continuous(0, 1, m, T, s, n, seed=1, event=7)
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("m,T,s", DEFLECT)
def test_deflection_fp32_follows_the_same_draws(slab, slab_o, m, T, s):
    """the split form uses the same Philox words (23-bit uniforms, fast intrinsics)"""
    from paper_2209_15445_gb300 import adept as A
    n = 4000
    rc, g = A.adept_probe_continuous(slab.h, 0, 1, m, 1, T, s, 7, n)
    assert rc == 0
    ref = slab_o.sample_continuous(0, 1, m, T, s, n, seed=1, event=7)
    assert np.allclose(np.linalg.norm(g, axis=1), 1.0, atol=1e-6)
    close = np.all(np.abs(g - ref) < 2e-4, axis=1)
    assert close.mean() > 0.999, close.mean()


@pytest.mark.parametrize("sp,m,T,s", FLUCT)
def test_fluctuation_fp64_matches_oracle(slab, slab_o, sp, m, T, s):
    from paper_2209_15445_gb300 import adept as A
    n = 4000
    rc, g = A.adept_probe_continuous(slab.h, 1, sp, m, 0, T, s, 9, n)
    assert rc == 0
    ref = slab_o.sample_continuous(1, sp, m, T, s, n, seed=1, event=9)
    np.testing.assert_allclose(g, ref, rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("sp,m,T,s", FLUCT)
def test_fluctuation_fp32_same_distribution(slab, slab_o, sp, m, T, s):
    from paper_2209_15445_gb300 import adept as A
    n = 20000
    rc, g = A.adept_probe_continuous(slab.h, 1, sp, m, 1, T, s, 9, n)
    assert rc == 0
    ref = slab_o.sample_continuous(1, sp, m, T, s, n, seed=1, event=13)  # independent draws
    mean = ref[0, 1]
    assert abs(g[0, 1] / mean - 1) < 1e-4  # the mean loss from the FP32 tables
    assert (g[:, 0] >= 0).all() and (g[:, 0] <= 2 * g[0, 1] * (1 + 1e-12)).all()
    assert stats.ks_2samp(g[:, 0] / g[0, 1], ref[:, 0] / mean).pvalue > 1e-4


def run_generations(geom, prim, mask):
    from paper_2209_15445_gb300 import adept as A
    tr = make(geom, precision=0, process_mask=mask, graph_generations=16, physics=BOTH, tuned=False)
    A.adept_reset_generation_log(tr.h)
    gpu_run(tr, prim)
    log = gen_log(tr)
    tr.close()
    ref = oracle.Oracle(geom).transport(prim, process_mask=mask, max_gen=20000, physics=BOTH)["gen_hist"]
    ref = ref.astype(np.int64)
    last = np.nonzero(ref.sum(axis=1))[0].max()
    got = np.zeros_like(ref)
    got[0] = [np.sum(prim.pdg == 22), np.sum(prim.pdg == 11), np.sum(prim.pdg == -11)]
    k = min(len(log), len(ref) - 1)
    got[1:k + 1] = log[:k]
    return got[: last + 2], ref[: last + 2]


def test_generation_counts_with_msc_and_fluctuations_ioni_only():
    """Ionisation alone, with a deflection on every charged step: as with full physics below,
    the last bits of CUDA's and glibc's FP64 log/cos/sqrt can flip one boundary decision
    (seen: 2 of 933 entries off by one track in 40 events, once steps cut short by the step
    limit stopped interacting and the tracks took more deflected steps)."""
    need_gpu()
    got, ref = run_generations(W.slab_calorimeter(), W.electrons(40, 300.0), oracle.P_EIONI)
    d = np.abs(got - ref)
    assert d.max() <= 2, d.max()
    assert d.sum() <= 1e-3 * ref.sum() + 4, (d.sum(), ref.sum())


def test_generation_counts_with_msc_and_fluctuations_full_physics():
    """With a deflection on every charged step, the last-bit differences between CUDA's and
    glibc's FP64 log/cos/sqrt reach the positions, and over ~1e5 steps one boundary decision
    can flip (seen: one e- one generation late out of 4 events). The histories otherwise
    agree: every generation within one track."""
    need_gpu()
    prim = W.mixed(4, seed=23)
    prim.E[:] = np.minimum(prim.E, 1000.0)
    got, ref = run_generations(W.slab_calorimeter(), prim, 0)
    d = np.abs(got - ref)
    assert d.max() <= 2, d.max()
    assert d.sum() <= 1e-3 * ref.sum() + 4, (d.sum(), ref.sum())


@pytest.mark.parametrize("precision,phys", [(0, BOTH), (1, BOTH), (1, 1), (1, 2)])
def test_showers_with_msc_and_fluctuations(precision, phys):
    need_gpu()
    geom = W.slab_calorimeter()
    prim = W.electrons(300 if precision else 100, 1e4 if precision else 1000.0)
    tr = make(geom, precision=precision, arena_bytes=4 << 30, physics=phys)
    edep, meta = gpu_run(tr, prim)
    tr.close()
    E0 = primary_energy(prim)
    assert abs(meta.deposited_MeV + meta.leaked_MeV + meta.killed_MeV - E0.sum()) <= 1e-9 * E0.sum()
    ref = oracle.Oracle(geom).transport(prim, physics=phys)
    assert np.allclose(ref["edep"].sum(1) + ref["leaked"] + ref["killed"], E0, rtol=1e-12)
    layer_check(edep, ref["edep"])
    if precision == 0:
        # the same histories event by event, but for last-bit divergences, whose chance grows
        # with the number of deflected steps (seen: 89 % of 1 GeV showers identical)
        same = np.all(np.isclose(edep, ref["edep"], rtol=1e-9, atol=1e-9), axis=1)
        assert same.mean() > 0.75, same.mean()


def test_msc_barrel_field():
    need_gpu()
    geom = W.barrel_calorimeter()
    prim = W.barrel_primaries(200, seed=8)
    ref = oracle.Oracle(geom, field_T=3.8).transport(prim, physics=BOTH)
    tr = make(geom, precision=1, field_T=3.8, arena_bytes=2 << 30, physics=BOTH, tuned=False)
    edep, meta = gpu_run(tr, prim)
    tr.close()
    layer_check(edep, ref["edep"], rel=0.03)


def test_msc_with_chords_matches_oracle():
    """both optional parts at once (the V = 3 kernels)"""
    need_gpu()
    geom = W.barrel_calorimeter()
    prim = W.barrel_primaries(150, seed=9)
    ref = oracle.Oracle(geom, field_T=3.8).transport(prim, physics=BOTH, field_max_iter=100)
    tr = make(geom, precision=1, field_T=3.8, arena_bytes=2 << 30, physics=BOTH, field_max_iterations=100,
              tuned=False)
    edep, meta = gpu_run(tr, prim)
    tr.close()
    layer_check(edep, ref["edep"], rel=0.03)


def test_secondaries_and_step_lengths_with_msc_fp64():
    """counts within 1e-4 of the oracle's (FP64, same streams, libm last bits aside)"""
    need_gpu()
    from paper_2209_15445_gb300 import adept as A
    geom = W.slab_calorimeter()
    prim = W.electrons(200, 3000.0)
    tr = make(geom, precision=0, arena_bytes=2 << 30, flags=A.FLAG_STEP_HISTOGRAM, physics=BOTH)
    gpu_run(tr, prim)
    st = tr.stats()
    rc, hist = A.adept_get_step_histogram(tr.h)
    tr.close()
    ref = oracle.Oracle(geom).transport(prim, steplen=True, physics=BOTH)
    def near(a, b, rel=1e-4):
        a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        assert np.all(np.abs(a - b) <= rel * np.maximum(b, 1) + 2), (a, b)
    near(list(st.secondaries), ref["created"])
    near(list(st.steps), ref["steps"])
    near(hist, ref["steplen"], rel=1e-3)


def test_invalid_physics_options_rejected():
    need_gpu()
    from paper_2209_15445_gb300 import adept as A
    with pytest.raises(A.AdeptError):
        make(W.slab_calorimeter(), precision=1, physics=4)
    with pytest.raises(A.AdeptError):
        make(W.slab_calorimeter(), precision=1, physics=1, msc_range_factor=-1.0)
    with pytest.raises(A.AdeptError):  # the fused kernel has no physics variant
        make(W.slab_calorimeter(), precision=1, physics=1, fused=1, tuned=False)
