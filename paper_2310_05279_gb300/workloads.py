"""Seeded synthetic workloads and D3-shaped reference tables.

This module only draws numbers: atomic positions, types, cells and the
per-element reference tables (reference coordination numbers, the C6
reference grid, sqrt(Q) and covalent radii).  It contains none of the D3
arithmetic.  It is the one module that both the CUDA path (tests, bench) and
the CPU oracle's callers use to obtain identical inputs.

The real Grimme tables are not available, so every table is synthetic but has
the shape the method expects (Sec. II A: per-element reference CNs, a C6
reference grid per element pair, a per-element radius parameter for R0 and a
covalent radius for the CN of Eq. 4).  All generators use
``numpy.random.Generator(PCG64(seed))``.

Workloads (sizes as used throughout the package):

* ``bilayer_ab_64``      -- AB bilayer graphene, 64 C atoms, 8.52 x 9.84 x 23.4 A.
* ``bilayer_scan``       -- 128 bilayers of 1440 C atoms: 16 interlayer
  distances in [2.8, 8.0] A x 8 armchair slides in [0, 4.26) A from AA.
* ``mof_like_box``       -- FCC-derived jittered lattice of H/C/N/O/Zn at
  1.0 g/cm^3 in a cubic periodic box (1,048,576 atoms at full size).
* ``uneven_batch``       -- 512 triclinic periodic structures, 50-4000 atoms
  (log-uniform), H/C/N/O/Cu/Zn mixes, 0.8-2.2 g/cm^3.
* ``fit_batch``          -- 256 structures of 200-2000 atoms from the
  ``uneven_batch`` generator, for damping-parameter refits.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Atomic masses (u) of the elements the synthetic workloads use.
MASS = {"H": 1.008, "C": 12.011, "N": 14.007, "O": 15.999, "Cu": 63.546, "Zn": 65.38}
AMU_G = 1.66053906660e-24  # grams per u

# PBE-BJ damping and the CN/weight constants of Eqs. 2-4 used by every workload.
PBE_BJ = dict(s6=1.0, s8=0.7875, a1=0.4289, a2=4.4407, k1=16.0, k2=4.0 / 3.0, k3=4.0,
              rc_disp=12.0, rc_cn=6.0)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclasses.dataclass
class Tables:
    """Per-element reference data, padded to ``max_ref`` references.

    cn_ref[t, a]            reference coordination numbers (entries a >= nref[t] unused)
    c6_ref[ti, tj, a, b]    C6 reference grid, Ha*bohr^6, with c6_ref[ti,tj,a,b] == c6_ref[tj,ti,b,a]
    sqrtq[t]                sqrt(Q) of element t (R0^2 = 3 sqrtq_i sqrtq_j), bohr
    rcov[t]                 covalent radius of element t, bohr (scaled by k2 in Eq. 4)
    """
    names: List[str]
    nref: np.ndarray      # int32 [T]
    cn_ref: np.ndarray    # f64 [T, R]
    c6_ref: np.ndarray    # f64 [T, T, R, R]
    sqrtq: np.ndarray     # f64 [T]
    rcov: np.ndarray      # f64 [T]

    @property
    def ntypes(self) -> int:
        return int(self.nref.shape[0])

    @property
    def max_ref(self) -> int:
        return int(self.cn_ref.shape[1])


@dataclasses.dataclass
class Batch:
    """A batch of periodic structures, concatenated.

    pos      f64 [N, 3] Cartesian positions, Angstrom
    types    int32 [N]  element index into the tables
    offsets  int64 [B+1] atom ranges of the structures
    cells    f64 [B, 3, 3] rows are the lattice vectors, Angstrom
    pbc      int32 [B, 3]
    """
    pos: np.ndarray
    types: np.ndarray
    offsets: np.ndarray
    cells: np.ndarray
    pbc: np.ndarray
    tables: Tables
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def nstruct(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def natoms(self) -> int:
        return int(self.offsets[-1])

    def structure(self, s: int):
        a, b = int(self.offsets[s]), int(self.offsets[s + 1])
        return self.pos[a:b], self.types[a:b], self.cells[s], self.pbc[s]

    def subset(self, idx: Sequence[int]) -> "Batch":
        idx = list(idx)
        pos, typ, offs = [], [], [0]
        for s in idx:
            p, t, _, _ = self.structure(s)
            pos.append(p)
            typ.append(t)
            offs.append(offs[-1] + len(p))
        return Batch(np.concatenate(pos) if pos else np.zeros((0, 3)),
                     np.concatenate(typ).astype(np.int32) if typ else np.zeros(0, np.int32),
                     np.asarray(offs, np.int64), self.cells[idx].copy(), self.pbc[idx].copy(),
                     self.tables, dict(self.info, subset=idx))


def batch_of(structs, tables: Tables, info: Optional[dict] = None) -> Batch:
    """Concatenate ``[(pos, types, cell, pbc), ...]`` into a Batch."""
    pos = [np.asarray(p, np.float64).reshape(-1, 3) for p, _, _, _ in structs]
    typ = [np.asarray(t, np.int32).reshape(-1) for _, t, _, _ in structs]
    offs = np.zeros(len(structs) + 1, np.int64)
    offs[1:] = np.cumsum([len(p) for p in pos])
    cells = np.asarray([np.asarray(c, np.float64).reshape(3, 3) for _, _, c, _ in structs]).reshape(-1, 3, 3)
    pbc = np.asarray([np.asarray(b, np.int32).reshape(3) for _, _, _, b in structs], np.int32).reshape(-1, 3)
    return Batch(np.concatenate(pos) if pos else np.zeros((0, 3)),
                 np.concatenate(typ) if typ else np.zeros(0, np.int32), offs, cells, pbc, tables, info or {})


# --------------------------------------------------------------------------- tables

def carbon_table(seed: int = 1000) -> Tables:
    """One element (C): 5 reference CNs {0,1,2,3,4} +- 0.02, C6ref log-uniform in
    [10, 60] Ha*bohr^6 (symmetric 5x5), sqrt(Q) = 3.1, Rcov = 1.44 bohr."""
    g = _rng(seed)
    R = 5
    cn = np.arange(R, dtype=np.float64) + g.uniform(-0.02, 0.02, R)
    m = np.exp(g.uniform(math.log(10.0), math.log(60.0), (R, R)))
    c6 = np.triu(m) + np.triu(m, 1).T
    return Tables(["C"], np.array([R], np.int32), cn[None, :], c6[None, None, :, :],
                  np.array([3.1]), np.array([1.44]))


def random_tables(names: Sequence[str], seed: int, max_ref: int = 5, nref_max: int = 5,
                  cn_max: float = 4.5, c6_range=(2.0, 400.0), sqrtq_range=(1.5, 8.0),
                  rcov_range=(0.6, 2.6)) -> Tables:
    """D3-shaped tables per element: nref ~ U{1..nref_max}, sorted reference CNs
    ~ U(0, cn_max), C6ref log-uniform in c6_range with the pair symmetry
    C6ref[ti,tj,a,b] == C6ref[tj,ti,b,a], sqrt(Q) ~ U(sqrtq_range), Rcov ~ U(rcov_range) bohr."""
    g = _rng(seed)
    T = len(names)
    nref = g.integers(1, nref_max + 1, T).astype(np.int32)
    cn = np.zeros((T, max_ref))
    for t in range(T):
        cn[t, :nref[t]] = np.sort(g.uniform(0.0, cn_max, nref[t]))
    c6 = np.zeros((T, T, max_ref, max_ref))
    lo, hi = math.log(c6_range[0]), math.log(c6_range[1])
    for ti in range(T):
        for tj in range(ti, T):
            for a in range(nref[ti]):
                for b in range(nref[tj]):
                    if ti == tj and b < a:
                        continue
                    v = math.exp(g.uniform(lo, hi))
                    c6[ti, tj, a, b] = v
                    c6[tj, ti, b, a] = v
    sqrtq = g.uniform(*sqrtq_range, T)
    rcov = g.uniform(*rcov_range, T)
    return Tables(list(names), nref, cn, c6, sqrtq, rcov)


# --------------------------------------------------------------------------- graphene

BOND = 1.42
RECT_X = 3.0 * BOND               # 4.26 A, armchair direction
RECT_Y = math.sqrt(3.0) * BOND    # 2.4595 A


def graphene_layer(nx: int, ny: int) -> np.ndarray:
    """Rectangular graphene sheet of nx x ny 4-atom cells (armchair along x), z = 0."""
    base = np.array([[0.0, 0.0], [BOND, 0.0], [1.5 * BOND, 0.5 * RECT_Y], [2.5 * BOND, 0.5 * RECT_Y]])
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    shifts = np.stack([ix.ravel() * RECT_X, iy.ravel() * RECT_Y], 1)
    xy = (shifts[:, None, :] + base[None, :, :]).reshape(-1, 2)
    return np.concatenate([xy, np.zeros((len(xy), 1))], 1)


def bilayer(nx: int, ny: int, d: float, slide: float, vacuum: float, jitter: float,
            g: np.random.Generator, z0: Optional[float] = None):
    """Two graphene layers, interlayer distance d, top layer slid by ``slide`` along x.
    Cell: nx*4.26 x ny*2.4595 x (d + vacuum), periodic in all three directions."""
    bottom = graphene_layer(nx, ny)
    top = bottom.copy()
    top[:, 0] += slide
    c = d + vacuum
    if z0 is None:
        z0 = 0.5 * (c - d)
    bottom[:, 2] = z0
    top[:, 2] = z0 + d
    pos = np.concatenate([bottom, top])
    if jitter > 0:
        pos = pos + g.uniform(-jitter, jitter, pos.shape)
    cell = np.diag([nx * RECT_X, ny * RECT_Y, c])
    return pos, np.zeros(len(pos), np.int32), cell, np.ones(3, np.int32)


def bilayer_ab_64(seed: int = 0) -> Batch:
    """AB bilayer graphene, 64 C atoms (2 layers x 32), 8.52 x 9.84 A, interlayer
    3.4 A, 20 A vacuum, +-0.02 A jitter.  AB stacking: top layer shifted one bond
    length along the armchair direction."""
    g = _rng(seed)
    s = bilayer(2, 4, 3.4, BOND, 20.0, 0.02, g)
    return batch_of([s], carbon_table(1000), dict(workload="bilayer_ab_64", seed=seed))


def bilayer_scan(seed: int = 1, n_dist: int = 16, n_slide: int = 8, nx: int = 10, ny: int = 18,
                 d_range=(2.8, 8.0)) -> Batch:
    """Binding/sliding scan: n_dist interlayer distances x n_slide slides k*4.26/n_slide
    along the armchair direction from AA; bilayers of nx*ny*8 C atoms (1440 at
    10 x 18), 20 A vacuum, +-0.02 A jitter, the carbon table of ``bilayer_ab_64``."""
    g = _rng(seed)
    structs, grid = [], []
    for d in np.linspace(d_range[0], d_range[1], n_dist):
        for k in range(n_slide):
            slide = k * RECT_X / n_slide
            structs.append(bilayer(nx, ny, float(d), slide, 20.0, 0.02, g))
            grid.append((float(d), slide))
    return batch_of(structs, carbon_table(1000),
                    dict(workload="bilayer_scan", seed=seed, grid=grid, n_dist=n_dist, n_slide=n_slide))


# --------------------------------------------------------------------------- MOF-like box

MOF_ELEMENTS = ["H", "C", "N", "O", "Zn"]
MOF_RATIO = [40, 36, 8, 12, 4]


def mof_like_box(seed: int = 2, ncell: int = 64, a: float = 262.45 / 64.0, jitter: float = 0.5,
                 min_sep: float = 0.95) -> Batch:
    """FCC lattice ncell^3 x 4 sites (lattice constant a), jitter U(-0.5, 0.5) A per
    coordinate, element types in the exact ratio H:C:N:O:Zn = 40:36:8:12:4 by a
    seeded shuffle (floor counts, remainder to H).  At ncell = 64 this is 1,048,576
    atoms in a 262.45 A cube at 1.000 g/cm^3.  The FCC nearest-neighbour distance
    a/sqrt(2) minus the largest jitter displacement sqrt(3) keeps every pair at
    least 1.17 A apart (> min_sep), which is checked here."""
    g = _rng(seed)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    i = np.arange(ncell)
    grid = np.stack(np.meshgrid(i, i, i, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    pos = ((grid[:, None, :] + basis[None]) * a).reshape(-1, 3)
    pos += g.uniform(-jitter, jitter, pos.shape)
    n = len(pos)
    counts = [n * r // sum(MOF_RATIO) for r in MOF_RATIO]
    counts[0] += n - sum(counts)
    types = np.concatenate([np.full(c, t, np.int32) for t, c in enumerate(counts)])
    g.shuffle(types)
    assert a / math.sqrt(2.0) - 2.0 * jitter * math.sqrt(3.0) >= min_sep
    L = ncell * a
    tables = random_tables(MOF_ELEMENTS, 1000 + 2)
    return batch_of([(pos, types, np.eye(3) * L, np.ones(3, np.int32))], tables,
                    dict(workload="mof_like_box", seed=seed, ncell=ncell, L=L))


def density_g_cm3(types: np.ndarray, names: Sequence[str], volume_A3: float) -> float:
    m = sum(MASS[names[t]] for t in types) * AMU_G
    return m / (volume_A3 * 1e-24)


# --------------------------------------------------------------------------- uneven batch

UNEVEN_ELEMENTS = ["H", "C", "N", "O", "Cu", "Zn"]


def _triclinic_cell(g: np.random.Generator) -> np.ndarray:
    """Unit-scale triclinic cell: angles U(70, 110) deg, edge ratios U(0.8, 1.25).
    Rows are lattice vectors in the usual lower-triangular orientation."""
    while True:
        al, be, ga = np.radians(g.uniform(70.0, 110.0, 3))
        la, lb, lc = 1.0, g.uniform(0.8, 1.25), g.uniform(0.8, 1.25)
        ax = np.array([la, 0.0, 0.0])
        bx = np.array([lb * math.cos(ga), lb * math.sin(ga), 0.0])
        cx_ = lc * math.cos(be)
        cy_ = lc * (math.cos(al) - math.cos(be) * math.cos(ga)) / math.sin(ga)
        cz2 = lc * lc - cx_ * cx_ - cy_ * cy_
        if cz2 > 1e-3 * lc * lc:
            return np.array([ax, bx, [cx_, cy_, math.sqrt(cz2)]])


def _perp_widths(cell: np.ndarray) -> np.ndarray:
    V = abs(np.linalg.det(cell))
    a, b, c = cell
    return np.array([V / np.linalg.norm(np.cross(b, c)), V / np.linalg.norm(np.cross(c, a)),
                     V / np.linalg.norm(np.cross(a, b))])


def random_structure(g: np.random.Generator, n: int, names: Sequence[str], dens_range=(0.8, 2.2),
                     min_sep: float = 0.95):
    """One periodic triclinic structure of n atoms.  Element fractions ~ Dirichlet(1),
    density ~ U(dens_range) g/cm^3.  Positions: n distinct points of a fractional
    grid (n1 x n2 x n3 >= n, n_k proportional to the perpendicular widths), each
    displaced by a random vector of length <= (h_min - min_sep)/2, where h_min
    (the smallest perpendicular grid spacing) lower-bounds the grid's shortest
    distance, so every pair stays >= min_sep apart.  If the drawn density would
    make h_min < min_sep / 0.9 the cell is enlarged until it does not (only
    possible for nearly pure-H mixes)."""
    T = len(names)
    frac = g.dirichlet(np.ones(T))
    types = g.choice(T, size=n, p=frac).astype(np.int32)
    rho = g.uniform(*dens_range)
    shape = _triclinic_cell(g)
    mass = sum(MASS[names[t]] for t in types) * AMU_G
    V = mass / rho * 1e24
    cell = shape * (V / abs(np.linalg.det(shape))) ** (1.0 / 3.0)
    for _ in range(60):
        w = _perp_widths(cell)
        nk = np.maximum(1, np.round(w / (np.prod(w) / n) ** (1.0 / 3.0))).astype(int)
        while np.prod(nk) < n:
            k = int(np.argmax(w / nk))
            nk[k] += 1
        h_min = float(np.min(w / nk))
        if h_min >= min_sep / 0.9:
            break
        cell = cell * 1.03
    ijk = np.stack(np.meshgrid(*[np.arange(m) for m in nk], indexing="ij"), -1).reshape(-1, 3)
    pick = g.choice(len(ijk), size=n, replace=False)
    f = (ijk[pick] + 0.5) / nk
    pos = f @ cell
    rad = 0.5 * (h_min - min_sep) * 0.999
    v = g.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pos = pos + v * (rad * g.uniform(0.0, 1.0, (n, 1)) ** (1.0 / 3.0))
    return pos, types, cell, np.ones(3, np.int32)


def uneven_batch(seed: int = 3, nstruct: int = 512, n_range=(50, 4000), names=UNEVEN_ELEMENTS,
                 table_seed: int = 1003) -> Batch:
    """nstruct periodic triclinic structures with log-uniform sizes in n_range."""
    g = _rng(seed)
    sizes = np.rint(np.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1]), nstruct))).astype(int)
    structs = [random_structure(g, int(n), names) for n in sizes]
    return batch_of(structs, random_tables(names, table_seed),
                    dict(workload="uneven_batch", seed=seed, sizes=sizes.tolist()))


def fit_batch(seed: int = 4, nstruct: int = 256, n_range=(200, 2000)) -> Batch:
    """Damping-refit workload: the uneven-batch generator at 200-2000 atoms."""
    b = uneven_batch(seed=seed, nstruct=nstruct, n_range=n_range, table_seed=1004)
    b.info["workload"] = "fit_batch"
    return b


def perturbed_damping(seed: int = 4, base: Optional[dict] = None) -> dict:
    """Damping parameters for the refit targets: s8, a1, a2 each scaled by U(0.9, 1.1)."""
    base = dict(base or PBE_BJ)
    g = _rng(10_000 + seed)
    f = g.uniform(0.9, 1.1, 3)
    base["s8"] *= f[0]
    base["a1"] *= f[1]
    base["a2"] *= f[2]
    return base


KB_EV = 8.617333262e-5          # Boltzmann constant, eV/K
EV_PER_AMU_A2_FS2 = 103.6427      # 1 amu A^2 / fs^2 in eV (so 1 eV/amu = 9.6485e-3 A^2/fs^2)


def atom_masses(batch: "Batch") -> np.ndarray:
    """Mass (u) of every atom, from the element names of the batch's tables."""
    return np.array([MASS[batch.tables.names[t]] for t in batch.types], np.float64)


def maxwell_velocities(masses: np.ndarray, T_K: float, seed: int) -> np.ndarray:
    """Velocities (A/fs) drawn from the Maxwell-Boltzmann distribution at T_K
    (each component normal with variance kB T / m), centre-of-mass motion removed."""
    g = _rng(seed)
    sigma = np.sqrt(KB_EV * T_K / masses / EV_PER_AMU_A2_FS2)
    v = g.normal(size=(len(masses), 3)) * sigma[:, None]
    v -= (masses[:, None] * v).sum(0) / masses.sum()
    return v


def displacement_direction(n: int, seed: int) -> np.ndarray:
    """Unit-scale random direction field (N x 3), e.g. for tangent checks."""
    return _rng(seed).normal(size=(n, 3))


WORKLOADS = {
    "bilayer_ab_64": bilayer_ab_64,
    "bilayer_scan": bilayer_scan,
    "mof_like_box": mof_like_box,
    "uneven_batch": uneven_batch,
    "fit_batch": fit_batch,
}
