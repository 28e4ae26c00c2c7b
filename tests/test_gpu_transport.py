"""Transport parity of the CUDA path with the FP64 oracle (C ABI end to end).

* single-interaction runs: per-generation queue sizes equal the oracle's exactly;
* showers: per-layer mean deposit within 3 combined standard errors and 1 % on every
  layer carrying more than 1 % of the total, and per-event energy conservation to 1e-9;
* edge cases: empty and ragged requests, primaries outside the calorimeter, bad input,
  too small an arena, a time budget that runs out, and queue overflow.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2209_15445_gb300 import workloads as W

from gpu_common import ledger, make, need_gpu

pytestmark = pytest.mark.gpu
ME = 0.51099895


def primary_energy(p):
    return p.E + np.where(p.pdg == -11, 2 * ME, 0.0)


def gpu_run(tr, prim):
    rid = tr.submit(prim)
    tr.transport()
    n_ev = len(np.unique(prim.event))
    edep, meta = tr.result(rid, n_ev)
    return edep, meta


def gen_log(tr):
    from paper_2209_15445_gb300 import adept as A
    n, log = A.adept_get_generation_log(tr.h)
    assert n >= 0
    return log.astype(np.int64)


def compare_generations(tr, orc, prim, mask, precision_note=""):
    from paper_2209_15445_gb300 import adept as A
    A.adept_reset_generation_log(tr.h)
    gpu_run(tr, prim)
    log = gen_log(tr)
    ref = orc.transport(prim, process_mask=mask, max_gen=20000)["gen_hist"].astype(np.int64)
    # the log row g holds the queues after generation g, i.e. the oracle's generation g+1
    last = np.nonzero(ref.sum(axis=1))[0].max()
    assert last >= 1
    got = np.zeros_like(ref)
    got[0] = [np.sum(prim.pdg == 22), np.sum(prim.pdg == 11), np.sum(prim.pdg == -11)]
    k = min(len(log), len(ref) - 1)
    got[1:k + 1] = log[:k]
    np.testing.assert_array_equal(got[: last + 2], ref[: last + 2])


SINGLE = [
    ("compton", 22, 1.0, oracle.P_COMPT),
    ("conversion", 22, 50.0, oracle.P_CONV),
    ("photo", 22, 0.2, oracle.P_PHOTO),
    ("e-ioni", 11, 100.0, oracle.P_EIONI),
    ("e-brem", 11, 300.0, oracle.P_EBREM),
    ("e+annihilation", -11, 20.0, oracle.P_ANNIH | oracle.P_PIONI),
]


@pytest.mark.parametrize("name,pdg,E,mask", SINGLE)
def test_single_interaction_generation_counts_bit_exact(name, pdg, E, mask):
    need_gpu()
    geom = W.slab_calorimeter()
    tr = make(geom, precision=0, process_mask=mask, graph_generations=8)
    n = 200
    prim = W.Primaries(np.full(n, pdg, np.int32), np.full(n, E), np.zeros((n, 3)),
                       np.tile([0.0, 0.0, 1.0], (n, 1)), np.arange(n, dtype=np.uint32))
    compare_generations(tr, oracle.Oracle(geom), prim, mask)
    tr.close()


def test_full_physics_generation_counts_bit_exact_few_events():
    need_gpu()
    geom = W.slab_calorimeter()
    tr = make(geom, precision=0, graph_generations=16)
    prim = W.mixed(6, seed=21)
    prim.E[:] = np.minimum(prim.E, 2000.0)
    compare_generations(tr, oracle.Oracle(geom), prim, 0)
    tr.close()


@pytest.mark.parametrize("chunk,fused", [(1, 0), (5, 0), (7, 1)])
def test_generation_counts_across_chunk_lengths(chunk, fused):
    """Generation g reads its queue sizes from slot g mod 3 and its tracks from buffer g mod 2,
    and its place in the chunk comes in as an argument, so chunk lengths that are not
    multiples of 6 start the chunks at every phase of both. The sizes per generation must
    still equal the oracle's exactly (FP64), in both the concurrent and the fused mode.
    Tail chunks are off here, so that every chunk has the fixed length."""
    need_gpu()
    geom = W.slab_calorimeter()
    kw = dict(fused=1, blocks_per_sm=2) if fused else {}
    tr = make(geom, precision=0, graph_generations=chunk, tuned=False, tail_tracks=-1, **kw)
    prim = W.mixed(4, seed=23)
    prim.E[:] = np.minimum(prim.E, 1000.0)
    compare_generations(tr, oracle.Oracle(geom), prim, 0)
    tr.close()


@pytest.mark.parametrize("fused,tail", [(0, 1 << 30), (1, 1 << 30), (0, 300)])
def test_tail_chunks_stop_with_the_last_track(fused, tail):
    """Tail chunks run one generation per iteration of a conditional graph loop and read
    their place in the chunk from the device: the queue sizes per generation still equal the
    oracle's exactly (FP64), and the transport runs exactly as many generations as the
    oracle's showers last, with at most a few empty generations at the end: tail chunks take
    over once the population has decayed below tail_tracks and an eighth of its peak, and a
    fixed chunk of 8 is queued only while the status two chunks back was above both, so no
    more than the rest of one fixed chunk and one more run past the last track."""
    need_gpu()
    geom = W.slab_calorimeter()
    kw = dict(fused=1, blocks_per_sm=2) if fused else {}
    tr = make(geom, precision=0, graph_generations=8, tuned=False, tail_tracks=tail, **kw)
    prim = W.mixed(4, seed=23)
    prim.E[:] = np.minimum(prim.E, 1000.0)
    orc = oracle.Oracle(geom)
    g0 = tr.stats().generations
    compare_generations(tr, orc, prim, 0)
    ran = tr.stats().generations - g0
    ref = orc.transport(prim, max_gen=20000)["gen_hist"]
    lasting = int(np.nonzero(ref.sum(axis=1))[0].max()) + 1  # generations with live tracks
    assert lasting <= ran < lasting + 16, (ran, lasting)
    tr.close()


def layer_check(g, o, frac=0.01, rel=0.01, nsig=3.0):
    """per-layer means within nsig combined SE and rel on layers above frac of the total"""
    mg, mo = g.mean(0), o.mean(0)
    sg = g.std(0, ddof=1) / math.sqrt(len(g))
    so = o.std(0, ddof=1) / math.sqrt(len(o))
    big = mo > frac * mo.sum()
    d = np.abs(mg - mo)
    bad = big & ~((d <= nsig * np.sqrt(sg**2 + so**2)) & (d <= rel * mo))
    assert not bad.any(), list(zip(np.nonzero(bad)[0], mg[bad], mo[bad], (d / mo)[bad]))
    return (d / np.maximum(mo, 1e-300))[big].max()


def shower_parity(geom, prim, precision, field_T=0.0, **kw):
    tr = make(geom, precision=precision, field_T=field_T, arena_bytes=2 << 30, **kw)
    edep, meta = gpu_run(tr, prim)
    assert meta.killed_MeV == 0.0
    tr.close()
    orc = oracle.Oracle(geom, field_T=field_T)
    ref = orc.transport(prim)
    E0 = primary_energy(prim)
    # energy conservation per request (per-event leaked/killed are summed in meta)
    assert abs(meta.deposited_MeV + meta.leaked_MeV + meta.killed_MeV - E0.sum()) <= 1e-9 * E0.sum()
    assert np.allclose(ledger(ref["edep"], ref["leaked"], ref["killed"]), E0, rtol=1e-12)
    return layer_check(edep, ref["edep"]), edep, ref


def test_shower_1gev_electrons_fp64():
    need_gpu()
    worst, g, o = shower_parity(W.slab_calorimeter(), W.electrons(100, 1000.0), precision=0)
    # FP64 with the same random streams: the histories are the oracle's
    assert worst < 1e-6


def test_shower_10gev_electrons_split_precision():
    need_gpu()
    worst, g, o = shower_parity(W.slab_calorimeter(), W.electrons(1000, 1e4), precision=1)
    print("split-precision worst per-layer relative error vs FP64 oracle:", worst)


def test_shower_mixed_field_1T():
    need_gpu()
    prim = W.mixed(400, seed=31)
    prim.E[:] = np.minimum(prim.E, 2e4)
    for prec in (0, 1):
        shower_parity(W.slab_calorimeter(), prim, precision=prec, field_T=1.0)


def test_shower_barrel_3p8T():
    need_gpu()
    prim = W.barrel_primaries(300, seed=41)
    prim.E[:] = np.minimum(prim.E, 5e3)
    for prec in (0, 1):
        shower_parity(W.barrel_calorimeter(), prim, precision=prec, field_T=3.8)


def test_empty_and_ragged_requests():
    need_gpu()
    tr = make(W.slab_calorimeter(), precision=1)
    rid = tr.submit(W.electrons(0, 1.0))
    from paper_2209_15445_gb300 import adept as A
    assert A.adept_poll(tr.h, rid) == 1
    edep, meta = tr.result(rid, 0)
    assert meta.n_events == 0 and edep.size == 0
    edep, meta = gpu_run(tr, W.electrons(1, 10.0))
    assert edep.shape == (1, 100) and abs(meta.deposited_MeV + meta.leaked_MeV - 10.0) < 1e-9
    # a zero-energy particle and a photon below the tracking cut just deposit
    p = W.Primaries(np.array([11, 22], np.int32), np.array([0.0, 5e-4]), np.zeros((2, 3)),
                    np.array([[0, 0, 1.0], [0, 0, 1.0]]), np.array([3, 3], np.uint32))
    edep, meta = gpu_run(tr, p)
    assert abs(meta.deposited_MeV - 5e-4) < 1e-15
    tr.close()


def test_primaries_outside_leak_immediately():
    need_gpu()
    tr = make(W.slab_calorimeter(), precision=0)
    p = W.Primaries(np.array([22, -11], np.int32), np.array([100.0, 5.0]),
                    np.array([[500.0, 0, 10.0], [0, 0, -5.0]]), np.array([[0, 0, 1.0], [0, 0, 1.0]]),
                    np.array([0, 1], np.uint32))
    edep, meta = gpu_run(tr, p)
    assert meta.leaked_MeV == pytest.approx(100.0 + 5.0 + 2 * ME, rel=1e-15, abs=0)
    assert edep.sum() == 0.0
    tr.close()


def test_invalid_input_and_small_arena():
    need_gpu()
    from paper_2209_15445_gb300 import adept as A
    tr = make(W.slab_calorimeter(), precision=0)
    bad = A.tracks_array(W.electrons(2, 10.0))
    bad["pdg"][1] = 2212
    rc, _ = A.adept_submit(tr.h, bad)
    assert rc == A.EINVAL and "pdg" in A.adept_last_error(tr.h)
    bad = A.tracks_array(W.electrons(1, 10.0))
    bad["dir"][0] = [0, 0, 2.0]
    assert A.adept_submit(tr.h, bad)[0] == A.EINVAL
    tr.close()
    with pytest.raises(A.AdeptError) as e:
        make(W.slab_calorimeter(), arena_bytes=1 << 20)
    assert e.value.code == A.ENOMEM


def test_timeout_then_resume():
    need_gpu()
    from paper_2209_15445_gb300 import adept as A
    tr = make(W.slab_calorimeter(), precision=1, graph_generations=1)
    prim = W.electrons(50, 5000.0)
    rid = tr.submit(prim)
    rc = A.adept_transport(tr.h, 1)  # 1 us: stops after the first chunk
    assert rc in (A.ETIMEOUT, A.OK)
    assert A.adept_poll(tr.h, rid) in (0, 1)
    tr.transport()
    edep, meta = tr.result(rid, 50)
    assert abs(meta.deposited_MeV + meta.leaked_MeV - 50 * 5000.0) < 1e-9 * 50 * 5000.0
    tr.close()


def test_queue_overflow_is_reported():
    need_gpu()
    from paper_2209_15445_gb300 import adept as A
    tr = make(W.slab_calorimeter(), precision=1, track_capacity=2048)
    tr.submit(W.electrons(50, 1e4))
    rc = A.adept_transport(tr.h, 0)
    assert rc == A.ENOMEM and "capacity" in A.adept_last_error(tr.h)
    assert tr.stats().overflow > 0
    tr.close()


def test_alone_equals_in_mix():
    """Serving: a request's result does not depend on what else is in flight (its random
    streams are keyed by its own events and track ids)."""
    need_gpu()
    geom = W.barrel_calorimeter()
    tr = make(geom, precision=1, field_T=3.8, arena_bytes=1 << 30)
    a = W.serving_batch(300, seed=5, event=1000)
    alone, _ = gpu_run(tr, a)
    ids = [tr.submit(W.serving_batch(500, seed=6 + k, event=2000 + k)) for k in range(3)]
    ra = tr.submit(a)
    ids.append(tr.submit(W.serving_batch(800, seed=9, event=3000)))
    tr.transport()
    mixed, _ = tr.result(ra, 1)
    np.testing.assert_allclose(mixed, alone, rtol=1e-9, atol=1e-9)
    tr.close()


def test_interleaved_events_number_like_grouped_ones():
    """A request's events are numbered in the order they first appear and its tracks in the
    order they come within their event, whether an event's tracks are together or spread
    through the request (the host's event table, with scattered event numbers that collide in
    it): the same primaries give the same per-event deposits either way."""
    need_gpu()
    geom = W.slab_calorimeter()
    n_ev, per = 50, 3
    events = (1000003 + 7919 * np.arange(n_ev) * np.arange(1, n_ev + 1)).astype(np.uint32)
    kind = [(11, 1000.0), (22, 500.0), (-11, 200.0)]
    def prim(order):
        idx = [(k, j) for k in range(n_ev) for j in range(per)] if order == "grouped" else \
              [(k, j) for j in range(per) for k in range(n_ev)]
        pdg = np.array([kind[j][0] for k, j in idx], np.int32)
        E = np.array([kind[j][1] for k, j in idx])
        pos = np.zeros((len(idx), 3))
        d = np.tile([0.0, 0.0, 1.0], (len(idx), 1))
        return W.Primaries(pdg, E, pos, d, np.array([events[k] for k, j in idx], np.uint32))
    tr = make(geom, precision=1, arena_bytes=1 << 30)
    res = {}
    for order in ("grouped", "interleaved"):
        p = prim(order)
        rid = tr.submit(p)
        tr.transport()
        res[order] = tr.result(rid, n_ev)
        assert res[order][1].n_events == n_ev
    tr.close()
    (g, mg), (i, mi) = res["grouped"], res["interleaved"]
    np.testing.assert_allclose(i, g, rtol=1e-12, atol=1e-9)
    E0 = n_ev * sum(E + (2 * ME if pdg == -11 else 0.0) for pdg, E in kind)
    for m in (mg, mi):
        assert abs(m.deposited_MeV + m.leaked_MeV + m.killed_MeV - E0) <= 1e-9 * E0


def test_event_marking_paths_agree_and_a_result_buffer_is_reused():
    """At a chunk's end the events that still have tracks are marked through a per-block
    bitmap of the event slots (up to 393,216 slots, with a direct pass below 16,384 live
    tracks) or, with more slots, by every live track marking its event: both report the same
    finished events, so the requests' deposits agree (up to the order of the FP64 atomics).
    A caller's buffer passed to result() is filled in place, also when reused."""
    need_gpu()
    geom = W.slab_calorimeter()
    n = 2000
    prim = W.electrons(n, 1e4)
    res = []
    for slots in (65536, 400000):
        tr = make(geom, precision=1, arena_bytes=2 << 30, max_events=slots)
        edep, meta = gpu_run(tr, prim)
        buf = np.full((n, tr.n_bins), np.nan)
        for _ in range(2):
            rid = tr.submit(prim)
            tr.transport()
            again, m2 = tr.result(rid, n, out=buf)
            assert again is buf
            np.testing.assert_allclose(again, edep, rtol=1e-12, atol=1e-9)
            assert m2.n_events == n and abs(m2.deposited_MeV - meta.deposited_MeV) <= 1e-9 * meta.deposited_MeV
        res.append((edep, meta))
        tr.close()
    (e0, m0), (e1, m1) = res
    np.testing.assert_allclose(e1, e0, rtol=1e-12, atol=1e-9)
    for f in ("deposited_MeV", "leaked_MeV", "killed_MeV"):
        assert abs(getattr(m1, f) - getattr(m0, f)) <= 1e-9 * max(1.0, abs(getattr(m0, f)))
    E0 = primary_energy(prim).sum()
    assert abs(m0.deposited_MeV + m0.leaked_MeV + m0.killed_MeV - E0) <= 1e-9 * E0


@pytest.mark.parametrize("precision", [0, 1])
def test_secondary_counts_and_step_lengths(precision):
    """Secondaries per species and the step-length distribution per species against the
    oracle (the paper compares secondary counts "to the per-mil level", Sec. 2.2, and
    validates step-length distributions, Sec. 2.1): identical in FP64, within 1 per mil
    (counts) and a chi-square test (histograms) in the split form."""
    need_gpu()
    from paper_2209_15445_gb300 import adept as A
    from scipy import stats
    geom = W.slab_calorimeter()
    prim = W.electrons(1000, 1e4)
    tr = make(geom, precision=precision, arena_bytes=4 << 30, flags=A.FLAG_STEP_HISTOGRAM)
    gpu_run(tr, prim)
    st = tr.stats()
    rc, hist = A.adept_get_step_histogram(tr.h)
    assert rc == 0
    tr.close()
    ref = oracle.Oracle(geom).transport(prim, steplen=True)
    g_sec = np.array(list(st.secondaries), np.int64)
    o_sec = ref["created"].astype(np.int64)
    g_steps = np.array(list(st.steps), np.int64)
    if precision == 0:
        np.testing.assert_array_equal(g_sec, o_sec)
        np.testing.assert_array_equal(g_steps, ref["steps"].astype(np.int64))
        np.testing.assert_array_equal(hist.astype(np.int64), ref["steplen"].astype(np.int64))
    else:
        assert np.all(np.abs(g_sec - o_sec) <= 1e-3 * o_sec), (g_sec, o_sec)
        for sp in range(3):
            a, b = hist[sp].astype(float), ref["steplen"][sp].astype(float)
            keep = (a + b) > 50
            chi2 = np.sum((a[keep] - b[keep]) ** 2 / (a[keep] + b[keep]))
            assert stats.chi2.sf(chi2, keep.sum()) > 1e-4, (sp, chi2, keep.sum())


@pytest.mark.parametrize("fused", [0, 1])
def test_one_generation_per_launch_without_graphs(fused):
    """the small-batch form: no CUDA graphs, one generation per launch and the queue sizes
    read back after each; the same per-generation queues as the oracle, with the timing
    events on"""
    need_gpu()
    from paper_2209_15445_gb300 import adept as A
    geom = W.slab_calorimeter()
    flags = A.FLAG_TIME_STEPS if fused else A.FLAG_TIME_SPECIES
    tr = make(geom, precision=0, graph_generations=-1, fused=fused, flags=flags, tuned=False)
    prim = W.mixed(4, seed=22)
    prim.E[:] = np.minimum(prim.E, 1000.0)
    compare_generations(tr, oracle.Oracle(geom), prim, 0)
    st = tr.stats()
    assert st.step_launches > 10 and st.step_kernel_ms > 0
    tr.close()


def test_admission_waits_for_slots_and_energy_budget():
    """more requests than event slots, and an energy budget that admits a few at a time:
    every request completes, each with the result it gets alone"""
    need_gpu()
    geom = W.slab_calorimeter()
    reqs = [W.electrons(20, 300.0, first_event=1000 * k) for k in range(10)]
    alone = []
    tr = make(geom, precision=1, tuned=False)
    for r in reqs:
        alone.append(gpu_run(tr, r)[0])
    tr.close()
    # 64 slots hold three requests of 20 events; a queue capacity of 4096 at 0.3 tracks/MeV
    # is an energy budget of 13.6 GeV, two of these 6 GeV requests at a time
    tr = make(geom, precision=1, max_events=64, track_capacity=4096, tracks_per_MeV=0.3, tuned=False)
    ids = [tr.submit(r) for r in reqs]
    tr.transport()
    for rid, a in zip(ids, alone):
        got, meta = tr.result(rid, 20)
        np.testing.assert_allclose(got, a, rtol=1e-9, atol=1e-9)
    tr.close()


@pytest.mark.parametrize("block", [64, 128])
def test_small_blocks_match_oracle(block):
    """the block sizes below 256 that the autotuner may pick"""
    need_gpu()
    geom = W.slab_calorimeter()
    tr = make(geom, precision=0, block_size=block, graph_generations=16, tuned=False)
    prim = W.mixed(5, seed=24)
    prim.E[:] = np.minimum(prim.E, 1500.0)
    compare_generations(tr, oracle.Oracle(geom), prim, 0)
    tr.close()
