"""ctypes binding of libadept.so (include/adept.h): argument marshalling only.

Every function named ``adept_*`` here forwards to the C entry point of the same name;
``Transport`` bundles one context with a torch-allocated device arena and a torch CUDA
stream (PyTorch provides device memory and streams; all transport work runs in the
library's sm_103a kernels). Loading fails loudly when the library is missing: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libadept.so")

OK, EINVAL, ENOMEM, ESTATE, ECUDA, ETIMEOUT, EBUSY, ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7
_NAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ESTATE: "ESTATE", ECUDA: "ECUDA", ETIMEOUT: "ETIMEOUT",
          EBUSY: "EBUSY", ENOTFOUND: "ENOTFOUND"}
FLAG_TIME_STEPS = 1
FLAG_TIME_SPECIES = 4
FLAG_STEP_HISTOGRAM = 8
# optional continuous physics (adept_options.physics)
PHYS_MSC = 1
PHYS_FLUCT = 2
P_COMPTON, P_CONVERSION, P_PHOTO, P_E_IONI, P_E_BREM, P_POS_IONI, P_POS_BREM, P_ANNIH = (1 << i for i in range(8))
NNODE = 289


class AdeptError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class adept_geometry(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_layers", C.c_int32), ("n_mat_per_layer", C.c_int32),
                ("layer_materials", C.POINTER(C.c_int32)), ("thickness_mm", C.POINTER(C.c_double)),
                ("transverse_half_mm", C.c_double), ("half_length_mm", C.c_double),
                ("layer_inner_r_mm", C.POINTER(C.c_double))]


class adept_material(C.Structure):
    _fields_ = [("Z", C.c_int32), ("A_g_mol", C.c_double), ("density_g_cm3", C.c_double), ("I_eV", C.c_double),
                ("n_elements", C.c_int32), ("element_Z", C.POINTER(C.c_int32)),
                ("element_A", C.POINTER(C.c_double)), ("element_atoms", C.POINTER(C.c_double))]


def material_struct(m, keep):
    """adept_material of a workloads.Material; the element arrays of a compound go to keep"""
    els = getattr(m, "elements", ())
    if not els:
        return adept_material(m.Z, m.A, m.density, m.I_eV, 0, None, None, None)
    z = np.array([e[0] for e in els], np.int32)
    a = np.array([e[1] for e in els], np.float64)
    n = np.array([e[2] for e in els], np.float64)
    keep += [z, a, n]
    return adept_material(0, 0.0, m.density, m.I_eV, len(els), z.ctypes.data_as(C.POINTER(C.c_int32)), _dp(a),
                          _dp(n))


class adept_cuts(C.Structure):
    _fields_ = [("range_cut_mm", C.c_double), ("field_T", C.c_double), ("tracking_cut_MeV", C.c_double)]


class adept_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("block_size", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("graph_generations", C.c_int32), ("seed", C.c_uint32), ("process_mask", C.c_uint32),
                ("max_steps", C.c_uint32), ("max_vacuum_steps", C.c_uint32), ("max_events", C.c_uint32),
                ("max_generation_log", C.c_uint32), ("track_capacity", C.c_uint64),
                ("tracks_per_MeV", C.c_double), ("flags", C.c_int32),
                ("blocks_per_sm_species", C.c_int32 * 3), ("fused", C.c_int32),
                ("physics", C.c_uint32), ("msc_range_factor", C.c_double),
                ("field_max_iterations", C.c_int32), ("delta_chord_mm", C.c_double),
                ("delta_intersection_mm", C.c_double), ("max_outgoing", C.c_uint32),
                ("tail_tracks", C.c_int32)]


TRACK_DTYPE = np.dtype([("pdg", "<i4"), ("pad0", "<i4"), ("E", "<f8"), ("pos", "<f8", 3), ("dir", "<f8", 3),
                        ("event", "<u4"), ("pad1", "<u4")])


class adept_track(C.Structure):
    _fields_ = [("pdg", C.c_int32), ("E_kin_MeV", C.c_double), ("pos_mm", C.c_double * 3),
                ("dir", C.c_double * 3), ("event", C.c_uint32)]


assert C.sizeof(adept_track) == TRACK_DTYPE.itemsize == 72


class adept_result(C.Structure):
    _fields_ = [("request", C.c_uint32), ("n_events", C.c_uint32), ("n_bins", C.c_uint32),
                ("deposited_MeV", C.c_double), ("leaked_MeV", C.c_double), ("killed_MeV", C.c_double),
                ("latency_us", C.c_double)]


class adept_stats(C.Structure):
    _fields_ = [("steps", C.c_uint64 * 3), ("secondaries", C.c_uint64 * 3), ("generations", C.c_uint64),
                ("overflow", C.c_uint64), ("requests_done", C.c_uint64), ("launches", C.c_uint64),
                ("step_launches", C.c_uint64), ("step_kernel_ms", C.c_double), ("species_ms", C.c_double * 3)]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libadept.so (built by paper_2209_15445_gb300.build); raises if it is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run paper_2209_15445_gb300.build.build() "
                              "(the shower transport has no CPU fallback)")
        L = C.CDLL(path)
        vp, sz, i32, u32, u64, dp = C.c_void_p, C.c_size_t, C.c_int32, C.c_uint32, C.c_uint64, C.POINTER(C.c_double)
        u32p, i32p = C.POINTER(C.c_uint32), C.POINTER(C.c_int32)
        sig = {
            "adept_init": [C.POINTER(vp), C.POINTER(adept_geometry), C.POINTER(adept_material), i32,
                           C.POINTER(adept_cuts), C.POINTER(adept_options), vp, sz, vp],
            "adept_build_tables": [vp],
            "adept_submit": [vp, vp, sz, u32p],
            "adept_submit_device": [vp, vp, sz, u32p],
            "adept_transport": [vp, u64],
            "adept_poll": [vp, u32],
            "adept_wait": [vp, u32, u64],
            "adept_get_scoring": [vp, u32, dp, sz, C.POINTER(adept_result)],
            "adept_get_leaked": [vp, u32, C.c_void_p, sz, C.POINTER(C.c_size_t)],
            "adept_get_stats": [vp, C.POINTER(adept_stats)],
            "adept_get_generation_log": [vp, u32p, sz],
            "adept_reset_generation_log": [vp],
            "adept_get_cuts": [vp, i32, dp, dp],
            "adept_get_step_histogram": [vp, C.POINTER(C.c_uint64)],
            "adept_get_table": [vp, i32, i32, i32, i32, dp],
            "adept_probe_philox": [vp, u32p, u32p, sz, u32p],
            "adept_probe_interp": [vp, i32, i32, i32, i32, dp, sz, dp],
            "adept_probe_inverse_range": [vp, i32, i32, i32, dp, sz, dp],
            "adept_probe_distance": [vp, i32, dp, dp, i32p, dp, i32p, sz, dp, i32p],
            "adept_probe_sample": [vp, i32, i32, i32, C.c_double, u32, sz, dp],
            "adept_probe_continuous": [vp, i32, i32, i32, i32, C.c_double, C.c_double, u32, sz, dp],
            "adept_raytrace": [vp, i32, dp, i32, i32, C.c_void_p, i32],
            "adept_probe_chord": [vp, i32, dp, dp, C.POINTER(C.c_int32), dp, C.POINTER(C.c_int32), dp, sz, dp],
            "adept_build_tables_noalloc": [C.POINTER(adept_material), i32, C.c_double, vp, vp, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.adept_last_error.argtypes = [vp]
        L.adept_last_error.restype = C.c_char_p
        L.adept_destroy.argtypes = [vp]
        L.adept_destroy.restype = None
        _lib = L
        return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def _i32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def tracks_array(prim: "W.Primaries") -> np.ndarray:
    """Pack primaries into the adept_track record layout."""
    a = np.zeros(len(prim), TRACK_DTYPE)
    a["pdg"] = prim.pdg
    a["E"] = prim.E
    a["pos"] = prim.pos
    a["dir"] = prim.dir
    a["event"] = prim.event
    return a


# ---- thin forwards with the C names ------------------------------------------------------
def adept_init(geometry, materials, n_materials, cuts, options, dev_arena, arena_bytes, stream):
    h = C.c_void_p()
    rc = load().adept_init(C.byref(h), C.byref(geometry), materials, n_materials, C.byref(cuts),
                           C.byref(options) if options is not None else None, dev_arena, arena_bytes, stream)
    return rc, h


def adept_build_tables(h): return load().adept_build_tables(h)
def adept_transport(h, timeout_us=0): return load().adept_transport(h, timeout_us)
def adept_poll(h, rid): return load().adept_poll(h, rid)
def adept_wait(h, rid, timeout_us=0): return load().adept_wait(h, rid, timeout_us)
def adept_reset_generation_log(h): return load().adept_reset_generation_log(h)
def adept_destroy(h): load().adept_destroy(h)


def adept_last_error(h) -> str:
    s = load().adept_last_error(h)
    return s.decode() if s else ""


def adept_submit(h, tracks: np.ndarray):
    tracks = np.ascontiguousarray(tracks, TRACK_DTYPE)
    rid = C.c_uint32()
    rc = load().adept_submit(h, tracks.ctypes.data if len(tracks) else None, len(tracks), C.byref(rid))
    return rc, rid.value


def adept_submit_device(h, dev_ptr: int, n: int):
    rid = C.c_uint32()
    rc = load().adept_submit_device(h, dev_ptr if n else None, n, C.byref(rid))
    return rc, rid.value


def adept_get_scoring(h, rid, edep_out: np.ndarray):
    meta = adept_result()
    rc = load().adept_get_scoring(h, rid, _dp(edep_out) if edep_out.size else None, edep_out.size, C.byref(meta))
    return rc, meta


def adept_get_stats(h):
    s = adept_stats()
    rc = load().adept_get_stats(h, C.byref(s))
    return rc, s


def adept_get_generation_log(h, n_max=1 << 16):
    out = np.zeros((n_max, 3), np.uint32)
    n = load().adept_get_generation_log(h, _u32p(out), n_max)
    return n, out[: max(n, 0)]


def adept_get_step_histogram(h):
    out = np.zeros((3, 64), np.uint64)
    rc = load().adept_get_step_histogram(h, out.ctypes.data_as(C.POINTER(C.c_uint64)))
    return rc, out


def adept_get_cuts(h, m):
    a, b = C.c_double(), C.c_double()
    rc = load().adept_get_cuts(h, m, C.byref(a), C.byref(b))
    return rc, a.value, b.value


def adept_get_table(h, s, t, m, prec):
    out = np.zeros(NNODE)
    rc = load().adept_get_table(h, s, t, m, prec, _dp(out))
    return rc, out


def adept_probe_philox(h, key, ctr: np.ndarray):
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros_like(ctr)
    rc = load().adept_probe_philox(h, _u32p(k), _u32p(ctr), len(ctr), _u32p(out))
    return rc, out


def adept_probe_interp(h, s, t, m, prec, E):
    E = np.ascontiguousarray(E, np.float64)
    out = np.zeros_like(E)
    rc = load().adept_probe_interp(h, s, t, m, prec, _dp(E), len(E), _dp(out))
    return rc, out


def adept_probe_inverse_range(h, s, m, prec, R):
    R = np.ascontiguousarray(R, np.float64)
    out = np.zeros_like(R)
    rc = load().adept_probe_inverse_range(h, s, m, prec, _dp(R), len(R), _dp(out))
    return rc, out


def adept_probe_distance(h, prec, pos, d, vol, T, q):
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, np.float64).reshape(-1, 3)
    vol = np.ascontiguousarray(vol, np.int32)
    T = np.ascontiguousarray(T, np.float64)
    q = np.ascontiguousarray(q, np.int32)
    n = len(vol)
    s = np.zeros(n)
    nx = np.zeros(n, np.int32)
    rc = load().adept_probe_distance(h, prec, _dp(pos), _dp(d), _i32p(vol), _dp(T), _i32p(q), n, _dp(s), _i32p(nx))
    return rc, s, nx


def adept_build_tables_noalloc(materials, range_cut_mm, dev_tables_ptr, dev_cuts_ptr, stream):
    """Forward to the allocation-free table build; materials is a list of workloads.Material."""
    keep = []
    arr = (adept_material * len(materials))(*[material_struct(m, keep) for m in materials])
    return load().adept_build_tables_noalloc(arr, len(materials), range_cut_mm, dev_tables_ptr, dev_cuts_ptr, stream)


def adept_probe_sample(h, which, m, prec, E, event, n):
    out = np.zeros((n, 12))
    rc = load().adept_probe_sample(h, which, m, prec, E, event, n, _dp(out))
    return rc, out


def adept_raytrace(h, prec, cam, nx, ny):
    """(rc, (ny, nx, 2) image in host memory): mass thickness (g/cm^2), volumes entered"""
    cam = np.ascontiguousarray(cam, np.float64)
    out = np.zeros((ny, nx, 2))
    rc = load().adept_raytrace(h, prec, _dp(cam), nx, ny, out.ctypes.data_as(C.c_void_p), 0)
    return rc, out


def adept_raytrace_device(h, prec, cam, nx, ny, dev_ptr):
    """launch into caller-owned device memory (16 nx ny bytes) on the context's stream"""
    cam = np.ascontiguousarray(cam, np.float64)
    return load().adept_raytrace(h, prec, _dp(cam), nx, ny, C.c_void_p(dev_ptr), 1)


def adept_get_leaked(h, rid):
    """(rc, structured array of adept_track) of a finished request's outgoing particles"""
    n = C.c_size_t()
    L = load()
    rc = L.adept_get_leaked(h, rid, None, 0, C.byref(n))
    if rc != OK:
        return rc, None
    arr = np.zeros(n.value, dtype=TRACK_DTYPE)
    rc = L.adept_get_leaked(h, rid, arr.ctypes.data_as(C.c_void_p), n.value, C.byref(n))
    return rc, arr


def adept_probe_chord(h, prec, pos, d, vol, T, q, s_phys):
    """one chord-propagated step per point: (n, 9) status, path, next, position, direction"""
    pos = np.ascontiguousarray(pos, np.float64); d = np.ascontiguousarray(d, np.float64)
    vol = np.ascontiguousarray(vol, np.int32); T = np.ascontiguousarray(T, np.float64)
    q = np.ascontiguousarray(q, np.int32); s_phys = np.ascontiguousarray(s_phys, np.float64)
    n = len(vol)
    out = np.zeros((n, 9))
    i32p = C.POINTER(C.c_int32)
    rc = load().adept_probe_chord(h, prec, _dp(pos), _dp(d), vol.ctypes.data_as(i32p), _dp(T),
                                  q.ctypes.data_as(i32p), _dp(s_phys), n, _dp(out))
    return rc, out


def adept_probe_continuous(h, which, species, m, prec, T, s, event, n):
    out = np.zeros((n, 3 if which == 0 else 2))
    rc = load().adept_probe_continuous(h, which, species, m, prec, T, s, event, n, _dp(out))
    return rc, out


# ---- convenience wrapper --------------------------------------------------------------
class Transport:
    """One library context on the current CUDA device with a torch-owned arena and stream."""

    def __init__(self, geom: "W.Geometry", *, range_cut_mm=0.7, field_T=0.0, tracking_cut_MeV=1e-3,
                 precision=0, arena_bytes=1 << 30, build_tables=True, **opts):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the shower transport runs on a CUDA GPU; none is available")
        load()
        self.geom = geom
        self.torch = torch
        self.stream = torch.cuda.Stream()
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda")
        self._keep = []
        mats = (adept_material * len(geom.materials))(*[material_struct(m, self._keep) for m in geom.materials])
        lm = np.array(geom.sub_materials, np.int32)
        th = np.array(geom.sub_thickness, np.float64)
        lr = np.array(geom.layer_r if geom.layer_r else [0.0], np.float64)
        self._keep += [mats, lm, th, lr]
        g = adept_geometry(geom.kind, geom.n_layers, len(lm), _i32p(lm), _dp(th), geom.half_xy, geom.half_z,
                           _dp(lr) if geom.layer_r else None)
        cuts = adept_cuts(range_cut_mm, field_T, tracking_cut_MeV)
        o = adept_options()
        o.precision = precision
        if opts.pop("tuned", True):
            # launch settings found by paper_2209_15445_gb300.autotune for this geometry and
            # precision, for the options the caller leaves unset
            from . import autotune
            t = autotune.load().get(autotune.key(geom.kind, precision))
            if t:
                opts.setdefault("graph_generations", t["graph_generations"])
                opts.setdefault("block_size", t["block_size"])
                opts.setdefault("fused", t.get("fused", 0))
                if opts["fused"] and t.get("fused"):
                    opts.setdefault("blocks_per_sm", t["blocks_per_sm"])
                elif "blocks_per_sm" not in opts and "blocks_per_sm_species" in t:
                    opts.setdefault("blocks_per_sm_species", (C.c_int32 * 3)(*t["blocks_per_sm_species"]))
        for k, v in opts.items():
            setattr(o, k, v)
        self.options = o
        self.n_bins = geom.n_bins
        rc, self.h = adept_init(g, mats, len(geom.materials), cuts, o, self.arena.data_ptr(), int(arena_bytes),
                                self.stream.cuda_stream)
        if rc != OK:
            raise AdeptError(rc, "adept_init failed")
        if build_tables:
            self.check(adept_build_tables(self.h))

    def check(self, rc):
        if rc < 0:
            raise AdeptError(rc, adept_last_error(self.h))
        return rc

    def submit(self, prim) -> int:
        arr = prim if isinstance(prim, np.ndarray) else tracks_array(prim)
        rc, rid = adept_submit(self.h, arr)
        self.check(rc)
        return rid

    def submit_device(self, dev_tensor, n) -> int:
        rc, rid = adept_submit_device(self.h, dev_tensor.data_ptr(), n)
        self.check(rc)
        return rid

    def transport(self, timeout_us=0):
        return self.check(adept_transport(self.h, timeout_us))

    def outgoing(self, rid):
        """the outgoing particles of a finished request (before result(), which releases it)"""
        rc, arr = adept_get_leaked(self.h, rid)
        self.check(rc)
        return arr

    def result(self, rid, n_events, out=None):
        """(edep[n_events, n_bins], meta) of a finished request; `out`, if given, is a float64
        array of that shape to fill (reused across requests, it saves the pages of a new one)"""
        if out is None:
            out = np.empty((n_events, self.n_bins))
        elif out.shape != (n_events, self.n_bins) or out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError(f"out must be a C-contiguous float64 array of shape {(n_events, self.n_bins)}")
        # the library writes the request's rows; only rows past them need zeros
        rc, meta = adept_get_scoring(self.h, rid, out)
        self.check(rc)
        out[meta.n_events:] = 0.0
        return out, meta

    def run(self, prim, timeout_us=0):
        """Submit, transport, return (edep[n_events, n_bins], meta)."""
        rid = self.submit(prim)
        self.transport(timeout_us)
        n_ev = len(np.unique(prim.event)) if len(prim) else 0
        return self.result(rid, n_ev)

    def stats(self):
        rc, s = adept_get_stats(self.h)
        self.check(rc)
        return s

    def close(self):
        if getattr(self, "h", None):
            adept_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
