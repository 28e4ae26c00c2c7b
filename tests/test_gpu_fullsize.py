"""Full-size parity on the configurations of the study, in the launch configuration that
bench.py times (CUDA-graph chunks of 32 generations, default kernel variants).

* 10,000 x 10 GeV e- (the headline workload): every event on both sides, split and plain
  FP64 forms; per-layer means within 3 combined SE and 1 % (layers above 1 % of the total).
* 20,000 mixed primaries in 1 T and 100,000 barrel primaries in 3.8 T: the GPU runs the
  whole batch, the oracle recomputes a seeded sample of 2,000 events (an event's result
  depends only on its own random streams), compared event by event and per layer.
* The headline workload with multiple scattering and fluctuations, and in the paper's PbWO4
  calorimeter, sampled the same way.
The worst per-layer relative difference of each form against the FP64 oracle is printed.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2209_15445_gb300 import workloads as W

from gpu_common import make, need_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
ME = 0.51099895


def per_layer(g, o, frac=0.01, rel=0.01, nsig=3.0):
    mg, mo = g.mean(0), o.mean(0)
    sg = g.std(0, ddof=1) / math.sqrt(len(g))
    so = o.std(0, ddof=1) / math.sqrt(len(o))
    big = mo > frac * mo.sum()
    d = np.abs(mg - mo)
    ok = (d <= nsig * np.sqrt(sg**2 + so**2)) & (d <= rel * mo)
    worst = float((d[big] / mo[big]).max())
    assert ok[big].all(), list(zip(np.nonzero(big & ~ok)[0], mg[big & ~ok], mo[big & ~ok]))
    return worst


def run_gpu(geom, prim, precision, field, chunks=1, arena=12 << 30, **kw):
    tr = make(geom, precision=precision, field_T=field, arena_bytes=arena, graph_generations=32,
              max_events=200000, tracks_per_MeV=0.1, **kw)
    n = len(prim)
    parts = [np.arange(k * n // chunks, (k + 1) * n // chunks) for k in range(chunks)]
    ids = [tr.submit(prim.take(ix)) for ix in parts]
    tr.transport()
    out = []
    tot = 0.0
    for rid, ix in zip(ids, parts):
        e, meta = tr.result(rid, len(ix))
        assert meta.killed_MeV == 0.0
        tot += meta.deposited_MeV + meta.leaked_MeV
        out.append(e)
    tr.close()
    E0 = (prim.E + np.where(prim.pdg == -11, 2 * ME, 0.0)).sum()
    assert abs(tot - E0) <= 1e-9 * E0
    return np.concatenate(out)


@pytest.fixture(scope="module")
def c2_oracle():
    prim = W.electrons(10000, 1e4)
    return prim, oracle.Oracle(W.slab_calorimeter()).transport(prim)["edep"]


@pytest.mark.parametrize("precision", [1, 0])
def test_c2_full_size(c2_oracle, precision):
    need_gpu()
    prim, ref = c2_oracle
    g = run_gpu(W.slab_calorimeter(), prim, precision, 0.0)
    worst = per_layer(g, ref)
    paired = np.abs(g.sum(1) - ref.sum(1)) / ref.sum(1)
    print(f"\n10k x 10 GeV e-, {'split' if precision else 'FP64'}: worst per-layer rel. diff {worst:.2e}, "
          f"events with total deposit within 1e-6: {np.mean(paired < 1e-6):.4f}")
    if precision == 0:
        assert worst < 1e-6


def sampled(geom, field, prim, chunks, arena, precision, n_sample=2000, physics=0):
    need_gpu()
    g = run_gpu(geom, prim, precision, field, chunks=chunks, arena=arena, **({"physics": physics} if physics else {}))
    rng = np.random.default_rng(99)
    idx = np.sort(rng.choice(len(prim), n_sample, replace=False))
    ref = oracle.Oracle(geom, field_T=field).transport(prim.take(idx), physics=physics)["edep"]
    gs = g[idx]
    worst = per_layer(gs, ref, rel=0.03)
    paired = np.abs(gs.sum(1) - ref.sum(1)) / np.maximum(ref.sum(1), 1e-300)
    return worst, float(np.mean(paired < 1e-6))


@pytest.mark.parametrize("precision", [1, 0])
def test_c3_full_size_sampled(precision):
    prim = W.mixed(20000, seed=3)
    worst, frac = sampled(W.slab_calorimeter(), 1.0, prim, 1, 12 << 30, precision)
    print(f"\n20k mixed, 1 T, {'split' if precision else 'FP64'}: worst per-layer rel. diff on 2000 sampled "
          f"events {worst:.2e}; events equal to 1e-6: {frac:.4f}")


def test_c4_full_size_sampled():
    prim = W.barrel_primaries(100000, seed=4)
    worst, frac = sampled(W.barrel_calorimeter(), 3.8, prim, 100, 40 << 30, 1)
    print(f"\n100k barrel, 3.8 T, split: worst per-layer rel. diff on 2000 sampled events {worst:.2e}; "
          f"events equal to 1e-6: {frac:.4f}")


def test_c2_with_msc_and_fluctuations_full_size_sampled():
    """the headline workload with multiple scattering and loss fluctuations (bench
    --physics 3): 10,000 showers on the GPU, 1,000 sampled events in the oracle"""
    prim = W.electrons(10000, 1e4)
    worst, frac = sampled(W.slab_calorimeter(), 0.0, prim, 1, 60 << 30, 1, n_sample=1000, physics=3)
    print(f"\n10k x 10 GeV e- with MSC + fluctuations, split: worst per-layer rel. diff on 1000 sampled events "
          f"{worst:.2e}")


def test_papers_calorimeter_full_size_sampled():
    """10,000 x 10 GeV e- in the paper's PbWO4 / lAr calorimeter, split"""
    prim = W.electrons(10000, 1e4)
    worst, frac = sampled(W.pbwo4_calorimeter(), 0.0, prim, 1, 12 << 30, 1)
    print(f"\n10k x 10 GeV e- in PbWO4/lAr, split: worst per-layer rel. diff on 2000 sampled events {worst:.2e}; "
          f"events equal to 1e-6: {frac:.4f}")
