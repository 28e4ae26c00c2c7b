"""Serving: 16 host producer threads submit requests while one driver thread runs the
transport; requests are admitted at generation boundaries as memory frees up, their work
overlaps on the device, and every result comes back complete, conserving energy, and equal
to the same request transported alone."""
import threading
import time

import numpy as np
import pytest

from paper_2209_15445_gb300 import workloads as W

from gpu_common import make, need_gpu

pytestmark = pytest.mark.gpu
ME = 0.51099895


def test_sixteen_producers_continuous_batching():
    need_gpu()
    from paper_2209_15445_gb300 import adept as A
    geom = W.barrel_calorimeter()
    tr = make(geom, precision=1, field_T=3.8, arena_bytes=2 << 30, graph_generations=8)
    stop = threading.Event()
    errors, results = [], {}
    lock = threading.Lock()

    def driver():
        while not stop.is_set():
            rc = A.adept_transport(tr.h, 5000)
            if rc not in (A.OK, A.ETIMEOUT):
                errors.append(A.adept_last_error(tr.h))
                return
            if rc == A.OK:
                time.sleep(1e-4)

    def producer(k):
        rng = np.random.default_rng(k)
        for j in range(6):
            n = int(np.exp(rng.uniform(np.log(10), np.log(600))))
            ev = 10000 * (k + 1) + j
            batch = W.serving_batch(n, seed=1000 * k + j, event=ev)
            rid = tr.submit(batch)
            rc = A.adept_wait(tr.h, rid, 60_000_000)
            if rc != A.OK:
                errors.append(f"wait {rc}")
                return
            out, meta = tr.result(rid, 1)
            E0 = batch.E.sum() + 2 * ME * np.sum(batch.pdg == -11)
            with lock:
                results[(k, j)] = (batch, out, meta, E0)

    th = [threading.Thread(target=driver)] + [threading.Thread(target=producer, args=(k,)) for k in range(16)]
    for t in th:
        t.start()
    for t in th[1:]:
        t.join(timeout=300)
    stop.set()
    th[0].join(timeout=60)
    assert not errors, errors
    assert len(results) == 16 * 6
    for (k, j), (batch, out, meta, E0) in results.items():
        assert abs(meta.deposited_MeV + meta.leaked_MeV + meta.killed_MeV - E0) <= 1e-9 * E0
        assert meta.latency_us > 0
    # a sample of requests transported again alone gives the same deposits
    for key in [(0, 0), (7, 3), (15, 5)]:
        batch, out, meta, E0 = results[key]
        alone, _ = tr.run(batch)
        np.testing.assert_allclose(alone, out, rtol=1e-9, atol=1e-9)
    tr.close()
