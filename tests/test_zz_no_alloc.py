"""The allocation-free table build (adept_build_tables_noalloc) against the regular one.

Callers that cannot allocate device memory (a host framework owning every allocation,
or a path that must not add allocation latency or failures) use an entry point whose
working memory is a static device array. Two calls in a row must each reproduce the
tables and thresholds that adept_build_tables leaves in a context's arena, within the
1e-12 relative tolerance of the FP64 table tests. This file is collected last so that a
run stopping at the first failure has run everything else before it.
"""
import numpy as np
import pytest

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
        ref = np.zeros((len(mats), 12, A.NNODE))
        ref_cuts = np.zeros((len(mats), 2))
        for m in range(len(mats)):
            r = 0
            for s, nt in NTAB:
                for t in range(nt):
                    rc, v = A.adept_get_table(tr.h, s, t, m, 0)
                    assert rc == 0
                    ref[m, r] = v
                    r += 1
            rc, tc, kc = A.adept_get_cuts(tr.h, m)
            ref_cuts[m] = (tc, kc)
        tr.close()
        stream = torch.cuda.Stream()
        for call in range(2):
            out = torch.full((len(mats), 12, A.NNODE), float("nan"), dtype=torch.float64, device="cuda")
            cuts = torch.full((len(mats), 2), float("nan"), dtype=torch.float64, device="cuda")
            rc = A.adept_build_tables_noalloc(mats, 0.7, out.data_ptr(), cuts.data_ptr(), stream.cuda_stream)
            assert rc == A.OK, call
            stream.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=0)
            np.testing.assert_allclose(cuts.cpu().numpy(), ref_cuts, rtol=1e-12, atol=0)


def test_noalloc_rejects_more_materials_than_its_scratch_holds():
    torch = need_gpu()
    from paper_2209_15445_gb300 import adept as A
    out = torch.zeros(8 * 12 * A.NNODE, dtype=torch.float64, device="cuda")
    cuts = torch.zeros(16, dtype=torch.float64, device="cuda")
    mats = [W.PB] * 5
    assert A.adept_build_tables_noalloc(mats, 0.7, out.data_ptr(), cuts.data_ptr(), 0) == A.EINVAL
    assert A.adept_build_tables_noalloc([], 0.7, out.data_ptr(), cuts.data_ptr(), 0) == A.EINVAL
