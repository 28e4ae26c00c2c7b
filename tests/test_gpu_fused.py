"""The fused mode (one kernel per generation for all three species) against the FP64
oracle and against the concurrent species kernels.

The random streams are keyed per track, so the set of tracks in each generation does not
depend on which kernel or warp ran them: per-generation queue sizes must equal the
oracle's exactly in FP64, whichever mode runs.
"""
import numpy as np
import pytest

import oracle
from paper_2209_15445_gb300 import workloads as W

from gpu_common import make, need_gpu
from test_gpu_transport import SINGLE, compare_generations, gpu_run, layer_check, shower_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,pdg,E,mask", SINGLE)
def test_fused_single_interaction_generation_counts_bit_exact(name, pdg, E, mask):
    need_gpu()
    geom = W.slab_calorimeter()
    tr = make(geom, precision=0, process_mask=mask, graph_generations=8, fused=1, tuned=False)
    n = 200
    prim = W.Primaries(np.full(n, pdg, np.int32), np.full(n, E), np.zeros((n, 3)),
                       np.tile([0.0, 0.0, 1.0], (n, 1)), np.arange(n, dtype=np.uint32))
    compare_generations(tr, oracle.Oracle(geom), prim, mask)
    tr.close()


@pytest.mark.parametrize("bps", [1, 2])
def test_fused_full_physics_generation_counts_bit_exact(bps):
    need_gpu()
    geom = W.slab_calorimeter()
    tr = make(geom, precision=0, graph_generations=16, fused=1, blocks_per_sm=bps, tuned=False)
    prim = W.mixed(6, seed=21)
    prim.E[:] = np.minimum(prim.E, 2000.0)
    compare_generations(tr, oracle.Oracle(geom), prim, 0)
    tr.close()


def test_fused_shower_fp64_matches_oracle():
    need_gpu()
    worst, g, o = shower_parity(W.slab_calorimeter(), W.electrons(100, 1000.0), precision=0, fused=1, tuned=False)
    assert worst < 1e-6


@pytest.mark.parametrize("bps", [2, 3])
def test_fused_split_equals_concurrent_split(bps):
    """same inputs, split form: the fused and the concurrent kernels give the same showers"""
    need_gpu()
    geom = W.slab_calorimeter()
    prim = W.electrons(300, 1e4)
    out = []
    for fused in (0, 1):
        kw = dict(fused=1, blocks_per_sm=bps) if fused else dict(fused=0)
        tr = make(geom, precision=1, arena_bytes=2 << 30, tuned=False, **kw)
        edep, meta = gpu_run(tr, prim)
        st = tr.stats()
        out.append((edep, list(st.steps), list(st.secondaries)))
        tr.close()
    (e0, s0, c0), (e1, s1, c1) = out
    # the same device code per track, compiled into two kernels: step and secondary totals
    # match exactly, and each event's deposit to rounding. FP32 contraction (FMA or not)
    # can differ between the two compilations: a few FP32 ulps (eps 6e-8) in one sampled
    # fraction change a leaking track's energy and the event's deposit by ~1e-7 of it
    # (seen: 1.7e-6 MeV and 1.1e-4 MeV in one of 300 events), and can move a few eV of one
    # step across a layer boundary. Bound: 16 FP32 ulps of the event total.
    assert s0 == s1 and c0 == c1
    np.testing.assert_allclose(e1.sum(axis=1), e0.sum(axis=1), rtol=16 * 2.0**-24)
    assert (np.abs(e1 - e0) <= 1e-6 * e0.sum(axis=1, keepdims=True)).all()


def test_fused_barrel_field_matches_oracle():
    need_gpu()
    prim = W.barrel_primaries(200, seed=5)
    for prec in (0, 1):
        shower_parity(W.barrel_calorimeter(), prim, precision=prec, field_T=3.8, fused=1, tuned=False)


def test_fused_rejects_species_timing():
    need_gpu()
    from paper_2209_15445_gb300 import adept as A
    with pytest.raises(A.AdeptError):
        make(W.slab_calorimeter(), precision=1, fused=1, flags=A.FLAG_TIME_SPECIES, tuned=False)
