"""ctypes front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the cpu_baseline /
reference legs of ``bench.py`` may use it; the product path never does. The oracle is
plain C built with gcc (``-O2 -ffp-contract=off``) so that x86 and Arm hosts give the
same bits.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NNODE = 289
P_COMPT, P_CONV, P_PHOTO, P_EIONI, P_EBREM, P_PIONI, P_PBREM, P_ANNIH = (1 << i for i in range(8))
# optional continuous physics of or_run_opts.physics
PHYS_MSC, PHYS_FLUCT = 1, 2

# sampler ids of or_sample
S_COMPTON, S_PAIR, S_MOLLER, S_BHABHA, S_BREM, S_ANNIH, S_ANNIH_REST = range(7)


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (only when the source is newer)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-D_GNU_SOURCE", "-o", tmp, src, "-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _RunOpts(C.Structure):
    _fields_ = [("seed", C.c_uint32), ("process_mask", C.c_uint32), ("max_steps", C.c_uint32),
                ("max_vacuum_steps", C.c_uint32), ("n_threads", C.c_int), ("max_gen", C.c_int),
                ("physics", C.c_uint32), ("msc_range_factor", C.c_double),
                ("field_max_iter", C.c_int), ("delta_chord", C.c_double), ("delta_int", C.c_double)]


class _Result(C.Structure):
    _fields_ = [("edep", C.POINTER(C.c_double)), ("leaked", C.POINTER(C.c_double)),
                ("killed", C.POINTER(C.c_double)), ("steps", C.c_uint64 * 3),
                ("created", C.c_uint64 * 3), ("gen_hist", C.POINTER(C.c_uint64)),
                ("steplen_hist", C.POINTER(C.c_uint64)), ("leak_out", C.POINTER(C.c_double)),
                ("leak_cap", C.c_uint64), ("leak_n", C.c_uint64), ("boundary_steps", C.c_uint64 * 3)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i, u32, u64, p = C.c_double, C.c_int, C.c_uint32, C.c_uint64, C.c_void_p
            dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
            L.or_philox.argtypes = [C.POINTER(u32), C.POINTER(u32), C.POINTER(u32)]
            L.or_u01_f64.argtypes = [u32, u32]; L.or_u01_f64.restype = d
            L.or_u01_f32.argtypes = [u32]; L.or_u01_f32.restype = C.c_float
            L.or_child_id.argtypes = [u32, u32, u64, u32, u32]; L.or_child_id.restype = u64
            L.or_create.argtypes = [i, ip, dp, dp, dp, ip, ip, dp, dp, i, i, i, ip, dp, d, d, dp, d, d, d]
            L.or_create.restype = p
            L.or_destroy.argtypes = [p]
            for name in ("or_mu_compton", "or_mu_pair", "or_mu_photo", "or_lambda_annih",
                         "or_density_delta"):
                getattr(L, name).argtypes = [p, i, d]
                getattr(L, name).restype = d
            L.or_inv_X0.argtypes = [p, i]; L.or_inv_X0.restype = d
            L.or_dedx_col.argtypes = [p, i, d, d, i]; L.or_dedx_col.restype = d
            L.or_dedx_rad.argtypes = [p, i, d, d]; L.or_dedx_rad.restype = d
            L.or_lambda_ioni.argtypes = [p, i, d, d, i]; L.or_lambda_ioni.restype = d
            L.or_lambda_brem.argtypes = [p, i, d, d]; L.or_lambda_brem.restype = d
            L.or_sigma_kn.argtypes = [d]; L.or_sigma_kn.restype = d
            L.or_sigma_kn_direct.argtypes = [d]; L.or_sigma_kn_direct.restype = d
            L.or_cuts.argtypes = [p, i, dp, dp]
            L.or_table.argtypes = [p, i, i, i, dp]; L.or_table.restype = i
            L.or_interp.argtypes = [p, i, i, i, d]; L.or_interp.restype = d
            L.or_inverse_range.argtypes = [p, i, i, d]; L.or_inverse_range.restype = d
            L.or_node_energy.argtypes = [i]; L.or_node_energy.restype = d
            L.or_sample.argtypes = [p, i, i, d, u32, u32, i, dp]
            L.or_sample_continuous.argtypes = [p, i, i, i, d, d, u32, u32, i, dp]
            L.or_msc_theta0.argtypes = [p, i, d, d]; L.or_msc_theta0.restype = d
            L.or_chord_step.argtypes = [p, d, i, d, i, d, d, dp, dp, i, ip, dp, ip]
            L.or_chord_step.restype = i
            L.or_raytrace.argtypes = [p, dp, i, i, dp]
            L.or_fluct_sigma2.argtypes = [p, i, d, d, i]; L.or_fluct_sigma2.restype = d
            L.or_n_volumes.argtypes = [p]; L.or_n_volumes.restype = i
            L.or_n_bins.argtypes = [p]; L.or_n_bins.restype = i
            L.or_locate.argtypes = [p, dp, dp]; L.or_locate.restype = i
            L.or_distance.argtypes = [p, dp, dp, i, ip]; L.or_distance.restype = d
            L.or_helix_move.argtypes = [d, d, i, d, dp, dp]
            L.or_helix_distance.argtypes = [p, d, i, dp, dp, i, ip]; L.or_helix_distance.restype = d
            L.or_transport.argtypes = [p, i, ip, dp, dp, dp, C.POINTER(u32), ip, i,
                                       C.POINTER(_RunOpts), C.POINTER(_Result)]
            L.or_transport.restype = i
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def u01_f64(w0, w1) -> float:
    return lib().or_u01_f64(int(w0), int(w1))


def u01_f32(w) -> float:
    return lib().or_u01_f32(int(w))


def child_id(seed, event, parent_id, parent_step, k) -> int:
    return lib().or_child_id(seed, event, parent_id, parent_step, k)


def node_energies() -> np.ndarray:
    return np.array([lib().or_node_energy(i) for i in range(NNODE)])


class Oracle:
    """One material/geometry/cut setup of the oracle."""

    def __init__(self, geom, range_cut_mm=0.7, field_T=0.0, tracking_cut_MeV=1e-3):
        L = lib()
        self.geom = geom
        mats = geom.materials
        self.n_mat = len(mats)
        Z = np.array([m.Z for m in mats], np.int32)
        A = np.array([m.A for m in mats], np.float64)
        rho = np.array([m.density for m in mats], np.float64)
        I = np.array([m.I_eV for m in mats], np.float64)
        # compounds: their elements (Z, A, atoms per formula unit), material after material
        ne = np.array([len(getattr(m, "elements", ())) for m in mats], np.int32)
        els = [e for m in mats for e in getattr(m, "elements", ())] or [(0, 0.0, 0.0)]
        eZ = np.array([e[0] for e in els], np.int32)
        eA = np.array([e[1] for e in els], np.float64)
        en = np.array([e[2] for e in els], np.float64)
        sm = np.array(geom.sub_materials, np.int32)
        st = np.array(geom.sub_thickness, np.float64)
        lr = np.array(geom.layer_r if geom.layer_r else [0.0], np.float64)
        self._keep = (Z, A, rho, I, ne, eZ, eA, en, sm, st, lr)
        self.h = L.or_create(self.n_mat, _ip(Z), _dp(A), _dp(rho), _dp(I), _ip(ne), _ip(eZ), _dp(eA), _dp(en),
                             geom.kind, geom.n_layers,
                             len(sm), _ip(sm), _dp(st), geom.half_xy, geom.half_z, _dp(lr),
                             range_cut_mm, field_T, tracking_cut_MeV)
        if not self.h:
            raise ValueError("oracle setup rejected the geometry")
        self.field_T = field_T
        self.tcut = tracking_cut_MeV
        self.n_bins = L.or_n_bins(self.h)
        self.n_vol = L.or_n_volumes(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().or_destroy(h)
            self.h = None

    # closed forms
    def mu_compton(self, m, E): return lib().or_mu_compton(self.h, m, E)
    def mu_pair(self, m, E): return lib().or_mu_pair(self.h, m, E)
    def mu_photo(self, m, E): return lib().or_mu_photo(self.h, m, E)
    def inv_X0(self, m): return lib().or_inv_X0(self.h, m)
    def dedx_col(self, m, T, cut, positron=0): return lib().or_dedx_col(self.h, m, T, cut, positron)
    def dedx_rad(self, m, T, kcut): return lib().or_dedx_rad(self.h, m, T, kcut)
    def delta(self, m, T): return lib().or_density_delta(self.h, m, T)
    def lambda_ioni(self, m, T, cut, positron=0): return lib().or_lambda_ioni(self.h, m, T, cut, positron)
    def lambda_brem(self, m, T, kcut): return lib().or_lambda_brem(self.h, m, T, kcut)
    def lambda_annih(self, m, T): return lib().or_lambda_annih(self.h, m, T)

    def cuts(self, m):
        a, b = C.c_double(), C.c_double()
        lib().or_cuts(self.h, m, C.byref(a), C.byref(b))
        return a.value, b.value

    def table(self, species, table, m) -> np.ndarray:
        out = np.zeros(NNODE)
        if lib().or_table(self.h, species, table, m, _dp(out)) != 0:
            raise ValueError("no such table")
        return out

    def interp(self, species, table, m, E): return lib().or_interp(self.h, species, table, m, E)
    def inverse_range(self, species, m, R): return lib().or_inverse_range(self.h, species, m, R)

    def sample(self, which, m, E, n, seed=1, event=0) -> np.ndarray:
        out = np.zeros((n, 12))
        lib().or_sample(self.h, which, m, E, seed, event, n, _dp(out))
        return out

    def msc_theta0(self, m, T, s): return lib().or_msc_theta0(self.h, m, T, s)

    def raytrace(self, cam, nx, ny):
        """(ny, nx, 2) image: mass thickness (g/cm^2) and volumes entered per pixel"""
        cam = np.ascontiguousarray(cam, np.float64)
        out = np.zeros((ny, nx, 2))
        lib().or_raytrace(self.h, _dp(cam), nx, ny, _dp(out))
        return out

    def chord_step(self, T, q, s_phys, max_iter, pos, d, vol, delta_chord=0.25, delta_int=0.001):
        """(status, position, direction, next, path, iterations) of one chord-propagated step"""
        pos = np.array(pos, np.float64); d = np.array(d, np.float64)
        nx, sd, it = C.c_int(vol), C.c_double(), C.c_int()
        rc = lib().or_chord_step(self.h, T, q, s_phys, max_iter, delta_chord, delta_int, _dp(pos), _dp(d), vol,
                                 C.byref(nx), C.byref(sd), C.byref(it))
        return rc, pos, d, nx.value, sd.value, it.value
    def fluct_sigma2(self, m, T, s, positron=False): return lib().or_fluct_sigma2(self.h, m, T, s, int(positron))

    def sample_continuous(self, which, species, m, T, s, n, seed=1, event=0) -> np.ndarray:
        """which 0: (n, 3) deflected directions of (0,0,1); which 1: (n, 2) loss and mean loss"""
        out = np.zeros((n, 3 if which == 0 else 2))
        lib().or_sample_continuous(self.h, which, species, m, T, s, seed, event, n, _dp(out))
        return out

    def locate(self, pos, d):
        pos = np.ascontiguousarray(pos, np.float64); d = np.ascontiguousarray(d, np.float64)
        return lib().or_locate(self.h, _dp(pos), _dp(d))

    def distance(self, pos, d, vol):
        pos = np.ascontiguousarray(pos, np.float64); d = np.ascontiguousarray(d, np.float64)
        nx = C.c_int()
        s = lib().or_distance(self.h, _dp(pos), _dp(d), vol, C.byref(nx))
        return s, nx.value

    def helix_distance(self, T, q, pos, d, vol):
        pos = np.ascontiguousarray(pos, np.float64); d = np.ascontiguousarray(d, np.float64)
        nx = C.c_int()
        s = lib().or_helix_distance(self.h, T, q, _dp(pos), _dp(d), vol, C.byref(nx))
        return s, nx.value

    def transport(self, prim, seed=1, process_mask=0, max_steps=100000, max_vacuum_steps=1000,
                  n_threads=None, max_gen=0, steplen=False, event_slot=None, n_events=None,
                  physics=0, msc_range_factor=0.0, field_max_iter=0, delta_chord=0.0, delta_int=0.0,
                  outgoing=0):
        """Transport primaries; tracks with the same event number form one event (slot
        order = first appearance) unless event_slot is given."""
        n = len(prim)
        if event_slot is None:
            _, first, inv = np.unique(prim.event, return_index=True, return_inverse=True)
            order = np.argsort(first)
            rank = np.empty_like(order); rank[order] = np.arange(len(order))
            event_slot = rank[inv].astype(np.int32)
            n_events = len(first)
        event_slot = np.ascontiguousarray(event_slot, np.int32)
        n_bins = self.n_bins
        edep = np.zeros((n_events, n_bins))
        leaked = np.zeros(n_events)
        killed = np.zeros(n_events)
        gen = np.zeros((max(max_gen, 1), 3), np.uint64)
        sl = np.zeros((3, 64), np.uint64)
        res = _Result()
        res.edep = _dp(edep); res.leaked = _dp(leaked); res.killed = _dp(killed)
        res.gen_hist = gen.ctypes.data_as(C.POINTER(C.c_uint64)) if max_gen > 0 else None
        res.steplen_hist = sl.ctypes.data_as(C.POINTER(C.c_uint64)) if steplen else None
        leak = np.zeros((max(outgoing, 1), 9))
        res.leak_out = _dp(leak) if outgoing else None
        res.leak_cap = outgoing
        o = _RunOpts(seed, process_mask, max_steps, max_vacuum_steps,
                     n_threads or os.cpu_count() or 1, max_gen, physics, msc_range_factor, field_max_iter,
                     delta_chord, delta_int)
        pdg = np.ascontiguousarray(prim.pdg, np.int32)
        E = np.ascontiguousarray(prim.E, np.float64)
        pos = np.ascontiguousarray(prim.pos, np.float64)
        d = np.ascontiguousarray(prim.dir, np.float64)
        key = np.ascontiguousarray(prim.event, np.uint32)
        rc = lib().or_transport(self.h, n, _ip(pdg), _dp(E), _dp(pos), _dp(d),
                                key.ctypes.data_as(C.POINTER(C.c_uint32)), _ip(event_slot),
                                n_events, C.byref(o), C.byref(res))
        if rc != 0:
            raise ValueError("oracle transport rejected its input")
        out = dict(edep=edep, leaked=leaked, killed=killed, steps=np.array(list(res.steps), np.uint64),
                   created=np.array(list(res.created), np.uint64),
                   boundary_steps=np.array(list(res.boundary_steps), np.uint64))
        if max_gen > 0:
            out["gen_hist"] = gen
        if steplen:
            out["steplen"] = sl
        if outgoing:
            if res.leak_n > outgoing:
                raise ValueError(f"{res.leak_n} outgoing particles, room for {outgoing}")
            out["outgoing"] = leak[: res.leak_n]
        return out


def helix_move(field_T, T, q, s, pos, d):
    pos = np.array(pos, np.float64); d = np.array(d, np.float64)
    lib().or_helix_move(field_T, T, q, s, _dp(pos), _dp(d))
    return pos, d
