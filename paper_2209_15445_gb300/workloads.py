"""Seeded synthetic inputs for the shower-transport workloads.

This module is the one place that both the CUDA path and the FP64 oracle take their
inputs from. It holds no physics arithmetic: only material constants (PDG values),
the layer layouts of the two calorimeters, and seeded draws of primary particles.

Workloads (the paper validates on a 50-layer sampling calorimeter, Sec. 2.2, and
studies batching of primaries, Sec. 5; the concrete sizes below are this project's):

* ``slab``: 50 layers of 2.3 mm Pb + 5.7 mm liquid argon, 40 x 40 cm transverse,
  starting at z = 0, beam along +z. (The paper uses PbWO4; Pb is used here.)
* ``barrel``: 20 concentric tube layers from r = 300 mm to 1800 mm, |z| <= 3000 mm,
  each Si 0.3 / Fe 20 / Pb 3 / lAr 5 mm from the inside out, vacuum gaps between.

Primary recipes (numpy PCG64 seeded with ``seed``):

* ``electrons(n, E)``: n e- of kinetic energy E at the origin along +z.
* ``mixed(n)``: T log-uniform in [100 MeV, 100 GeV]; species 50 % gamma, 40 % e-,
  10 % e+; at the origin along +z.
* ``barrel_primaries(n)``: T log-uniform in [1, 50] GeV; e-/gamma 50/50; from the
  origin, cos(theta) uniform in [-tanh 1.5, tanh 1.5] (|eta| < 1.5), phi uniform.
* ``serving_batch(n)``: species one third each; 1/E uniform between 1/10 MeV and
  1/20 GeV (an E^-2 spectrum); directions as barrel_primaries; position on the
  inner barrel face r = 300 mm along the direction.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PDG_GAMMA, PDG_ELECTRON, PDG_POSITRON = 22, 11, -11


@dataclass(frozen=True)
class Material:
    name: str
    Z: int
    A: float  # g/mol
    density: float  # g/cm^3
    I_eV: float  # mean excitation energy
    # a compound: ((Z, A g/mol, atoms per formula unit), ...); Z and A above are then unused
    elements: tuple = ()


# PDG "Atomic and nuclear properties of materials" values
PB = Material("Pb", 82, 207.2, 11.35, 823.0)
LAR = Material("lAr", 18, 39.948, 1.396, 188.0)
SI = Material("Si", 14, 28.0855, 2.329, 173.0)
FE = Material("Fe", 26, 55.845, 7.874, 286.0)
# lead tungstate, the paper's compound (PDG: density 8.30 g/cm^3, I = 600.7 eV)
PBWO4 = Material("PbWO4", 0, 0.0, 8.30, 600.7, elements=((82, 207.2, 1.0), (74, 183.84, 1.0), (8, 15.999, 4.0)))


@dataclass
class Geometry:
    kind: int  # 0 = slab stack along z, 1 = concentric tubes around z
    n_layers: int
    materials: list  # list[Material], indexed by sub_materials
    sub_materials: list  # material index of each sublayer of one layer
    sub_thickness: list  # mm
    half_xy: float = 0.0  # slab transverse half width
    half_z: float = 0.0  # tube half length
    layer_r: list = field(default_factory=list)  # tube layer inner radii

    @property
    def n_sub(self) -> int:
        return len(self.sub_materials)

    @property
    def n_bins(self) -> int:
        return self.n_layers * self.n_sub


def slab_calorimeter(n_layers: int = 50) -> Geometry:
    return Geometry(kind=0, n_layers=n_layers, materials=[PB, LAR], sub_materials=[0, 1],
                    sub_thickness=[2.3, 5.7], half_xy=200.0)


def pbwo4_calorimeter(n_layers: int = 50) -> Geometry:
    """the paper's validation calorimeter (Sec. 2.2): 50 layers of PbWO4 2.3 mm + lAr 5.7 mm"""
    return Geometry(kind=0, n_layers=n_layers, materials=[PBWO4, LAR], sub_materials=[0, 1],
                    sub_thickness=[2.3, 5.7], half_xy=200.0)


def barrel_calorimeter() -> Geometry:
    n = 20
    sub = [0.3, 20.0, 3.0, 5.0]
    pitch = (1500.0 - sum(sub)) / (n - 1)
    radii = [300.0 + i * pitch for i in range(n)]
    return Geometry(kind=1, n_layers=n, materials=[SI, FE, PB, LAR], sub_materials=[0, 1, 2, 3],
                    sub_thickness=sub, half_z=3000.0, layer_r=radii)


@dataclass
class Primaries:
    pdg: np.ndarray  # int32
    E: np.ndarray  # float64 kinetic energy, MeV
    pos: np.ndarray  # float64 [n, 3] mm
    dir: np.ndarray  # float64 [n, 3] unit
    event: np.ndarray  # uint32 event number (RNG key)

    def __len__(self) -> int:
        return len(self.E)

    def take(self, idx) -> "Primaries":
        return Primaries(self.pdg[idx], self.E[idx], self.pos[idx], self.dir[idx], self.event[idx])


def _beam(n: int) -> tuple[np.ndarray, np.ndarray]:
    pos = np.zeros((n, 3))
    d = np.zeros((n, 3))
    d[:, 2] = 1.0
    return pos, d


def electrons(n: int, E_MeV: float, first_event: int = 0) -> Primaries:
    pos, d = _beam(n)
    return Primaries(np.full(n, PDG_ELECTRON, np.int32), np.full(n, float(E_MeV)), pos, d,
                     np.arange(first_event, first_event + n, dtype=np.uint32))


def _loguniform(rng, n, lo, hi):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def mixed(n: int, seed: int = 3, first_event: int = 0) -> Primaries:
    rng = np.random.default_rng(seed)
    E = _loguniform(rng, n, 100.0, 1e5)
    u = rng.uniform(size=n)
    pdg = np.where(u < 0.5, PDG_GAMMA, np.where(u < 0.9, PDG_ELECTRON, PDG_POSITRON)).astype(np.int32)
    pos, d = _beam(n)
    return Primaries(pdg, E, pos, d, np.arange(first_event, first_event + n, dtype=np.uint32))


def _eta_directions(rng, n, eta_max=1.5):
    c = rng.uniform(-np.tanh(eta_max), np.tanh(eta_max), n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    s = np.sqrt(1.0 - c * c)
    return np.stack([s * np.cos(phi), s * np.sin(phi), c], axis=1)


def barrel_primaries(n: int, seed: int = 4, first_event: int = 0) -> Primaries:
    rng = np.random.default_rng(seed)
    E = _loguniform(rng, n, 1e3, 5e4)
    pdg = np.where(rng.uniform(size=n) < 0.5, PDG_ELECTRON, PDG_GAMMA).astype(np.int32)
    d = _eta_directions(rng, n)
    return Primaries(pdg, E, np.zeros((n, 3)), d,
                     np.arange(first_event, first_event + n, dtype=np.uint32))


def serving_batch(n: int, seed: int, event: int, r_face: float = 300.0) -> Primaries:
    """One request of the serving workload: n tracks of one event."""
    rng = np.random.default_rng(seed)
    emin, emax = 10.0, 2e4
    E = 1.0 / (1.0 / emin - rng.uniform(size=n) * (1.0 / emin - 1.0 / emax))
    u = rng.uniform(size=n)
    pdg = np.where(u < 1 / 3, PDG_ELECTRON, np.where(u < 2 / 3, PDG_POSITRON, PDG_GAMMA)).astype(np.int32)
    d = _eta_directions(rng, n)
    sT = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
    pos = d * (r_face / sT)[:, None]
    return Primaries(pdg, E, pos, d, np.full(n, event, np.uint32))


def serving_batch_size(rng) -> int:
    """Batch size log-uniform in [10, 10000] tracks."""
    return int(np.exp(rng.uniform(np.log(10.0), np.log(1e4))))


def concat(parts: list) -> Primaries:
    return Primaries(np.concatenate([p.pdg for p in parts]), np.concatenate([p.E for p in parts]),
                     np.concatenate([p.pos for p in parts]), np.concatenate([p.dir for p in parts]),
                     np.concatenate([p.event for p in parts]))
