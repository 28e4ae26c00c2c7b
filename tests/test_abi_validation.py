"""CPU checks of adept_init's argument validation (include/adept.h: invalid arguments return
ADEPT_EINVAL, an arena too small for the layout ADEPT_ENOMEM).

Every case here is rejected on the host before any CUDA call, so the device arena can be a
fake, aligned address that is never dereferenced. The tests skip on a machine with a GPU,
where a case that slipped through validation would hand that address to the driver.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2209_15445_gb300 import workloads as W

FAKE_ARENA = 0x10000000  # 256-byte aligned, never touched


@pytest.fixture(scope="module")
def A():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: these cases use a fake device address")
    from paper_2209_15445_gb300 import adept
    adept.load()
    return adept


def init(A, geom=None, mats=None, cuts=(0.7, 0.0, 1e-3), arena=FAKE_ARENA, arena_bytes=1 << 30, **opts):
    geom = geom or W.slab_calorimeter()
    keep = []
    mats = mats if mats is not None else geom.materials
    marr = (A.adept_material * max(1, len(mats)))(*[A.material_struct(m, keep) for m in mats])
    lm = np.array(geom.sub_materials, np.int32)
    th = np.array(geom.sub_thickness, np.float64)
    lr = np.array(geom.layer_r if geom.layer_r else [0.0], np.float64)
    g = A.adept_geometry(geom.kind, geom.n_layers, len(lm), lm.ctypes.data_as(C.POINTER(C.c_int32)),
                         th.ctypes.data_as(C.POINTER(C.c_double)), geom.half_xy, geom.half_z,
                         lr.ctypes.data_as(C.POINTER(C.c_double)) if geom.layer_r else None)
    o = A.adept_options()
    for k, v in opts.items():
        setattr(o, k, v)
    rc, h = A.adept_init(g, marr, len(mats), A.adept_cuts(*cuts), o, C.c_void_p(arena), arena_bytes, None)
    assert not h.value, "no context may be returned on an error"
    return rc


def test_materials(A):
    assert init(A, mats=[]) == A.EINVAL
    bad_z = W.Material("X", 101, 250.0, 1.0, 100.0)
    assert init(A, mats=[bad_z, W.LAR]) == A.EINVAL
    no_density = W.Material("Pb", 82, 207.2, 0.0, 823.0)
    assert init(A, mats=[no_density, W.LAR]) == A.EINVAL
    bad_element = W.Material("c", 0, 0.0, 8.3, 600.0, elements=((0, 1.0, 1.0),))
    assert init(A, mats=[bad_element, W.LAR]) == A.EINVAL
    nine = W.Material("c", 0, 0.0, 8.3, 600.0, elements=tuple((z, 2.0 * z, 1.0) for z in range(1, 10)))
    assert init(A, mats=[nine, W.LAR]) == A.EINVAL


def test_cuts(A):
    assert init(A, cuts=(0.0, 0.0, 1e-3)) == A.EINVAL
    assert init(A, cuts=(0.7, 0.0, 1e-4)) == A.EINVAL
    assert init(A, cuts=(0.7, 0.0, 2e4)) == A.EINVAL


@pytest.mark.parametrize("opts", [
    dict(precision=2), dict(flags=1 << 8), dict(fused=2), dict(fused=1, flags=2), dict(physics=4),
    dict(msc_range_factor=-1.0), dict(field_max_iterations=-1), dict(fused=1, field_max_iterations=10),
    dict(fused=1, physics=1), dict(delta_chord_mm=-1.0), dict(block_size=48), dict(block_size=512),
    dict(block_size=16), dict(graph_generations=-2), dict(graph_generations=2000),
    dict(max_vacuum_steps=70000), dict(flags=8, fused=1), dict(flags=8, field_max_iterations=10),
])
def test_options(A, opts):
    assert init(A, **opts) == A.EINVAL, opts


def test_geometry(A):
    g = W.slab_calorimeter()
    for bad in (dict(kind=2), dict(n_layers=0), dict(sub_thickness=[2.3, 0.0]), dict(sub_materials=[0, 5]),
                dict(half_xy=0.0)):
        geom = W.Geometry(**{**g.__dict__, **bad})
        assert init(A, geom=geom) == A.EINVAL, bad
    b = W.barrel_calorimeter()
    assert init(A, geom=W.Geometry(**{**b.__dict__, "half_z": 0.0})) == A.EINVAL


def test_arena(A):
    assert init(A, arena=FAKE_ARENA + 16) == A.EINVAL  # not 256-byte aligned
    assert init(A, arena_bytes=1 << 20) == A.ENOMEM  # the fixed parts do not fit
    assert init(A, track_capacity=1 << 40) == A.ENOMEM  # more tracks than the arena holds
