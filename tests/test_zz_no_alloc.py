"""The allocation-free table build (adept_build_tables_noalloc) against the regular one.

Callers that cannot allocate device memory (a host framework owning every allocation,
or a path that must not add allocation latency or failures) use an entry point whose
working memory is a static device array. Two calls in a row must each reproduce the
tables and thresholds that adept_build_tables leaves in a context's arena, and those of
the FP64 CPU oracle, within the 1e-12 relative tolerance of the FP64 table tests. This file is collected last so that a
run stopping at the first failure has run everything else before it.
"""
import numpy as np
import pytest

import oracle
from paper_2209_15445_gb300 import workloads as W

from gpu_common import make, need_gpu

pytestmark = pytest.mark.gpu

NTAB = [(0, 3), (1, 4), (2, 5)]


def test_noalloc_tables_match_regular_build_twice():
    torch = need_gpu()
    from paper_2209_15445_gb300 import adept as A
    for geom in (W.slab_calorimeter(), W.barrel_calorimeter()):
        mats = geom.materials
        tr = make(geom, precision=0, arena_bytes=256 << 20)
        o = oracle.Oracle(geom)
        ref = np.zeros((len(mats), 12, A.NNODE))
        ora = np.zeros((len(mats), 12, A.NNODE))
        ref_cuts = np.zeros((len(mats), 2))
        ora_cuts = np.zeros((len(mats), 2))
        for m in range(len(mats)):
            r = 0
            for s, nt in NTAB:
                for t in range(nt):
                    rc, v = A.adept_get_table(tr.h, s, t, m, 0)
                    assert rc == 0
                    ref[m, r] = v
                    ora[m, r] = o.table(s, t, m)
                    r += 1
            rc, tc, kc = A.adept_get_cuts(tr.h, m)
            ref_cuts[m] = (tc, kc)
            ora_cuts[m] = o.cuts(m)
        tr.close()
        stream = torch.cuda.Stream()
        for call in range(2):
            # filled on the stream the entry point runs on, so the fill is ordered before it
            with torch.cuda.stream(stream):
                out = torch.full((len(mats), 12, A.NNODE), float("nan"), dtype=torch.float64, device="cuda")
                cuts = torch.full((len(mats), 2), float("nan"), dtype=torch.float64, device="cuda")
            rc = A.adept_build_tables_noalloc(mats, 0.7, out.data_ptr(), cuts.data_ptr(), stream.cuda_stream)
            assert rc == A.OK, call
            stream.synchronize()
            got, got_cuts = out.cpu().numpy(), cuts.cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
            np.testing.assert_allclose(got_cuts, ref_cuts, rtol=1e-12, atol=0)
            np.testing.assert_allclose(got, ora, rtol=1e-12, atol=1e-300)
            np.testing.assert_allclose(got_cuts, ora_cuts, rtol=1e-12, atol=0)


def test_noalloc_rejects_more_materials_than_its_scratch_holds():
    torch = need_gpu()
    from paper_2209_15445_gb300 import adept as A
    out = torch.zeros(8 * 12 * A.NNODE, dtype=torch.float64, device="cuda")
    cuts = torch.zeros(16, dtype=torch.float64, device="cuda")
    mats = [W.PB] * 5
    assert A.adept_build_tables_noalloc(mats, 0.7, out.data_ptr(), cuts.data_ptr(), 0) == A.EINVAL
    assert A.adept_build_tables_noalloc([], 0.7, out.data_ptr(), cuts.data_ptr(), 0) == A.EINVAL
