"""Compound materials on the GPU (the paper's PbWO4 / lAr calorimeter, Sec. 2.2) against
the FP64 oracle: tables and cuts built on the device from the element list, per-generation
queue sizes and showers in the paper's calorimeter, and bad compounds rejected."""
import numpy as np
import pytest

import oracle
from paper_2209_15445_gb300 import workloads as W

from gpu_common import make, need_gpu
from test_gpu_transport import compare_generations, gpu_run, layer_check, primary_energy

pytestmark = pytest.mark.gpu


def test_tables_and_cuts_of_lead_tungstate():
    need_gpu()
    from paper_2209_15445_gb300 import adept as A
    geom = W.pbwo4_calorimeter()
    tr = make(geom, precision=0)
    o = oracle.Oracle(geom)
    for m in range(2):
        rc, tc, kc = A.adept_get_cuts(tr.h, m)
        otc, okc = o.cuts(m)
        assert rc == 0 and tc == pytest.approx(otc, rel=1e-12, abs=0) and kc == pytest.approx(okc, rel=1e-12, abs=0)
        for s, nt in ((0, 3), (1, 4), (2, 5)):
            for t in range(nt):
                rc, g = A.adept_get_table(tr.h, s, t, m, 0)
                assert rc == 0
                np.testing.assert_allclose(g, o.table(s, t, m), rtol=1e-12, atol=1e-300)
    tr.close()


def test_generation_counts_bit_exact_in_the_papers_calorimeter():
    need_gpu()
    geom = W.pbwo4_calorimeter()
    tr = make(geom, precision=0, graph_generations=16, tuned=False)
    prim = W.electrons(8, 2000.0)
    compare_generations(tr, oracle.Oracle(geom), prim, 0)
    tr.close()


@pytest.mark.parametrize("precision,n,E", [(0, 100, 1000.0), (1, 1000, 1e4)])
def test_showers_in_the_papers_calorimeter(precision, n, E):
    need_gpu()
    geom = W.pbwo4_calorimeter()
    prim = W.electrons(n, E)
    tr = make(geom, precision=precision, arena_bytes=2 << 30)
    edep, meta = gpu_run(tr, prim)
    tr.close()
    E0 = primary_energy(prim)
    assert abs(meta.deposited_MeV + meta.leaked_MeV + meta.killed_MeV - E0.sum()) <= 1e-9 * E0.sum()
    ref = oracle.Oracle(geom).transport(prim)
    worst = layer_check(edep, ref["edep"])
    if precision == 0:
        assert worst < 1e-6


def test_bad_compounds_rejected():
    need_gpu()
    from paper_2209_15445_gb300 import adept as A
    too_many = W.Material("x", 0, 0.0, 1.0, 100.0, elements=tuple((8, 16.0, 1.0) for _ in range(9)))
    bad_z = W.Material("x", 0, 0.0, 1.0, 100.0, elements=((0, 16.0, 1.0),))
    bad_n = W.Material("x", 0, 0.0, 1.0, 100.0, elements=((8, 16.0, 0.0),))
    for mat in (too_many, bad_z, bad_n):
        g = W.Geometry(kind=0, n_layers=2, materials=[mat, W.LAR], sub_materials=[0, 1], sub_thickness=[1.0, 1.0],
                       half_xy=100.0)
        with pytest.raises(A.AdeptError):
            make(g, precision=1)
    # the allocation-free table build takes single elements only: with valid output
    # buffers, only the compound (alone, or after a valid element) makes it refuse
    import torch
    out = torch.zeros(2 * 12 * A.NNODE, dtype=torch.float64, device="cuda")
    cuts = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert A.adept_build_tables_noalloc([W.PB], 0.7, out.data_ptr(), cuts.data_ptr(), None) == A.OK
    assert A.adept_build_tables_noalloc([W.PBWO4], 0.7, out.data_ptr(), cuts.data_ptr(), None) == A.EINVAL
    assert A.adept_build_tables_noalloc([W.PB, W.PBWO4], 0.7, out.data_ptr(), cuts.data_ptr(), None) == A.EINVAL
    torch.cuda.synchronize()
