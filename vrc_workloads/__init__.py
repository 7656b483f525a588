"""Seeded synthetic inputs for the volumetric-ray-casting (VRC) estimator.

This module is shared by the FP64 CPU oracle and the CUDA path, so it holds
input generation only: mesh layouts, cross-section tables, ray batches and
group edges.  It contains none of the estimator's arithmetic (no cross-section
interpolation, no traversal, no scoring).  Every array is produced by
``numpy.random.default_rng(seed)``.

The paper's workloads (a PWR assembly, a criticality-accident room and
reflected Godiva, all with ACE nuclear data; Sec. 5, Tests 1-3) cannot be
reproduced without that data, so these generators stand in for them and take
their shapes: an optically thin 3-D mesh (accident room, 400x400x50), a fine
pin-lattice mesh (PWR, 0.6 mm cells) and a range of cubic meshes (Godiva's
100^3).  Cross sections are synthetic continuous-energy total cross sections:
a smooth ``0.1 + 2/sqrt(E)`` part plus Lorentzian resonances, tabulated on a
log-spaced energy grid (Sec. 3 describes tabulated continuous-energy data
interpolated linearly between table points).

Rays carry ``x, y, z, u, v, w, E, wt`` as float32 arrays (structure of
arrays); ``wt`` already includes the 1/N of Eq. 4.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

E_MIN_EV = 1.0e-5
E_MAX_EV = 2.0e7
RAY_FIELDS = ("x", "y", "z", "u", "v", "w", "E", "wt")


@dataclasses.dataclass
class Mesh:
    """A uniform 3-D Cartesian mesh; ``material`` is uint8 [nz][ny][nx]."""

    nx: int
    ny: int
    nz: int
    x0: float
    y0: float
    z0: float
    dx: float
    dy: float
    dz: float
    material: np.ndarray

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def lo(self):
        return (self.x0, self.y0, self.z0)

    @property
    def hi(self):
        return (self.x0 + self.nx * self.dx, self.y0 + self.ny * self.dy,
                self.z0 + self.nz * self.dz)


@dataclasses.dataclass
class RectMesh:
    """A rectilinear (non-uniform Cartesian) mesh: cell (ix, iy, iz) spans
    [xe[ix], xe[ix+1]) x [ye[iy], ye[iy+1]) x [ze[iz], ze[iz+1]); each edge
    array is strictly ascending float64 of n+1 values; ``material`` is uint8
    [nz][ny][nx]."""

    xe: np.ndarray
    ye: np.ndarray
    ze: np.ndarray
    material: np.ndarray

    @property
    def nx(self) -> int:
        return len(self.xe) - 1

    @property
    def ny(self) -> int:
        return len(self.ye) - 1

    @property
    def nz(self) -> int:
        return len(self.ze) - 1

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    # first plane and mean spacing per axis (the box; not cell sizes)
    x0 = property(lambda self: float(self.xe[0]))
    y0 = property(lambda self: float(self.ye[0]))
    z0 = property(lambda self: float(self.ze[0]))
    dx = property(lambda self: float(self.xe[-1] - self.xe[0]) / self.nx)
    dy = property(lambda self: float(self.ye[-1] - self.ye[0]) / self.ny)
    dz = property(lambda self: float(self.ze[-1] - self.ze[0]) / self.nz)

    @property
    def lo(self):
        return (self.x0, self.y0, self.z0)

    @property
    def hi(self):
        return (float(self.xe[-1]), float(self.ye[-1]), float(self.ze[-1]))


@dataclasses.dataclass
class Problem:
    """One tally problem: mesh, per-material tables, group edges, rays."""

    name: str
    mesh: Mesh
    tables: List[Optional[tuple]]  # per material: (E_eV float64, sigma float64) or None = void
    group_edges: Optional[np.ndarray]  # float64, ascending, n_groups+1; None = one group
    rays: dict  # field -> float32 array

    @property
    def n_materials(self) -> int:
        return len(self.tables)

    @property
    def n_groups(self) -> int:
        return 1 if self.group_edges is None else len(self.group_edges) - 1

    @property
    def n_rays(self) -> int:
        return int(self.rays["x"].shape[0])

    @property
    def tally_size(self) -> int:
        return self.n_groups * self.mesh.ncells


# --------------------------------------------------------------------------
# cross-section tables
# --------------------------------------------------------------------------

def xs_table(rng: np.random.Generator, n_points: int, n_resonances: int,
             peak_lo: float = 1.0, peak_hi: float = 1.0e3,
             e_min: float = E_MIN_EV, e_max: float = E_MAX_EV):
    """A synthetic total cross-section table (energies in eV, sigma in 1/cm).

    ``n_points`` log-spaced energies over [e_min, e_max]; sigma is
    ``0.1 + 2/sqrt(E)`` plus ``n_resonances`` Lorentzians
    ``A / (1 + ((E - E_r)/G)^2)`` with E_r log-uniform in [1, 1e5] eV,
    A log-uniform in [peak_lo, peak_hi] 1/cm and G = E_r * 10^U(-3, -1.5).
    The tabulated points define the cross section; the formula only fills
    the table.
    """
    E = np.logspace(math.log10(e_min), math.log10(e_max), n_points)
    E[0], E[-1] = e_min, e_max
    sig = 0.1 + 2.0 / np.sqrt(E)
    er = 10.0 ** rng.uniform(0.0, 5.0, n_resonances)
    amp = 10.0 ** rng.uniform(math.log10(peak_lo), math.log10(peak_hi), n_resonances)
    gam = er * 10.0 ** rng.uniform(-3.0, -1.5, n_resonances)
    for r in range(n_resonances):
        sig += amp[r] / (1.0 + ((E - er[r]) / gam[r]) ** 2)
    return E.astype(np.float64), sig.astype(np.float64)


def log_group_edges(n_groups: int, e_min: float = E_MIN_EV, e_max: float = E_MAX_EV):
    edges = np.logspace(math.log10(e_min), math.log10(e_max), n_groups + 1)
    edges[0], edges[-1] = e_min, e_max
    return edges.astype(np.float64)


# --------------------------------------------------------------------------
# rays
# --------------------------------------------------------------------------

def isotropic_dirs(rng: np.random.Generator, n: int):
    """Isotropic unit directions: mu = 2 xi - 1, phi = 2 pi xi (float32)."""
    mu = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    return ((s * np.cos(phi)).astype(np.float32), (s * np.sin(phi)).astype(np.float32),
            mu.astype(np.float32))


def log_uniform(rng: np.random.Generator, n: int, lo: float = E_MIN_EV, hi: float = E_MAX_EV):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n)).astype(np.float32)


def uniform_positions(rng: np.random.Generator, mesh: Mesh, n: int):
    lo, hi = mesh.lo, mesh.hi
    out = []
    for k in range(3):
        p = (lo[k] + (hi[k] - lo[k]) * rng.random(n)).astype(np.float32)
        # float32 rounding may land exactly on the upper face; keep inside
        p = np.minimum(p, np.nextafter(np.float32(hi[k]), np.float32(-np.inf)))
        out.append(p)
    return out


def make_rays(x, y, z, u, v, w, E, wt) -> dict:
    r = dict(x=x, y=y, z=z, u=u, v=v, w=w, E=E, wt=wt)
    return {k: np.ascontiguousarray(r[k], dtype=np.float32) for k in RAY_FIELDS}


# --------------------------------------------------------------------------
# the five workloads (scaled-down variants keep the same recipe)
# --------------------------------------------------------------------------

def uniform_small(seed: int = 0, n: int = 32, n_rays: int = 1 << 17,
                  n_points: int = 1000, n_resonances: int = 5) -> Problem:
    """n^3 mesh of 1 cm cells, void + one material, uniform-random layout.

    The plain-VRC parity workload: 32^3, 2 materials (0 = void), a
    1,000-point table with 5 resonances, 2^17 isotropic rays of weight 1,
    one total-fluence group, seed 0.
    """
    rng = np.random.default_rng(seed)
    mat = rng.integers(0, 2, size=(n, n, n), dtype=np.uint8)
    mesh = Mesh(n, n, n, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, mat)
    tables = [None, xs_table(rng, n_points, n_resonances)]
    x, y, z = uniform_positions(rng, mesh, n_rays)
    u, v, w = isotropic_dirs(rng, n_rays)
    E = log_uniform(rng, n_rays)
    wt = np.ones(n_rays, np.float32)
    return Problem(f"uniform{n}", mesh, tables, None, make_rays(x, y, z, u, v, w, E, wt))


def slab_room(seed: int = 1, n: int = 256, n_rays: int = 1 << 24, n_materials: int = 8,
              n_points: int = 20000, n_resonances: int = 200, n_slabs: int = 16,
              n_groups: int = 16) -> Problem:
    """n^3 mesh of 1 cm cells painted with random axis-aligned slabs.

    The throughput workload: 256^3, 8 materials with 20,000-point tables of
    200 resonances (peaks log-uniform 1-1e3 /cm), background material 0 then
    16 slabs (random axis, random index interval, random material) painted in
    order, 2^24 rays with lognormal(0, 0.5) weights, 16 log-uniform groups,
    seed 1.
    """
    rng = np.random.default_rng(seed)
    tables = [xs_table(rng, n_points, n_resonances) for _ in range(n_materials)]
    mat = np.zeros((n, n, n), np.uint8)
    for _ in range(n_slabs):
        axis = int(rng.integers(0, 3))
        a, b = sorted(int(t) for t in rng.integers(0, n + 1, size=2))
        if a == b:
            b = min(n, a + 1)
        m = int(rng.integers(0, n_materials))
        sl = [slice(None)] * 3
        sl[2 - axis] = slice(a, b)  # array axes are [z][y][x]
        mat[tuple(sl)] = m
    mesh = Mesh(n, n, n, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, mat)
    x, y, z = uniform_positions(rng, mesh, n_rays)
    u, v, w = isotropic_dirs(rng, n_rays)
    E = log_uniform(rng, n_rays)
    wt = rng.lognormal(0.0, 0.5, n_rays).astype(np.float32)
    return Problem(f"slab{n}", mesh, tables, log_group_edges(n_groups),
                   make_rays(x, y, z, u, v, w, E, wt))


def pin_lattice(seed: int = 2, pins: int = 17, cells_per_pin: int = 32, nz: int = 64,
                n_rays: int = 1 << 24, n_points: int = 20000, n_resonances: int = 200,
                inside_frac: float = 0.7) -> Problem:
    """A 17x17 lattice of cylinders (pitch 1.26 cm, radius 0.45 cm).

    Voxelised by cell centre on a 544x544x64 mesh of 0.039375 x 0.039375 x
    5 cm cells.  Materials: 0 moderator, 1 fuel core (r < 0.36),
    2 void gap (0.36 <= r < 0.40; no table, sigma = 0), 3 cladding
    (0.40 <= r < 0.45).  70% of start points are uniform in the r < 0.45
    discs times z, the rest uniform over the mesh; energies 1/E; seed 2.
    """
    rng = np.random.default_rng(seed)
    pitch = 1.26
    n = pins * cells_per_pin
    dx = pitch / cells_per_pin
    dz = 5.0
    c = (np.arange(n) + 0.5) * dx
    xc = np.mod(c, pitch) - 0.5 * pitch
    r = np.sqrt(xc[None, :] ** 2 + xc[:, None] ** 2)  # [iy][ix]
    layer = np.zeros((n, n), np.uint8)
    layer[r < 0.45] = 3
    layer[r < 0.40] = 2
    layer[r < 0.36] = 1
    mat = np.ascontiguousarray(np.broadcast_to(layer, (nz, n, n)))
    mesh = Mesh(n, n, nz, 0.0, 0.0, 0.0, dx, dx, dz, mat)
    tables = [xs_table(rng, n_points, n_resonances), xs_table(rng, n_points, n_resonances),
              None, xs_table(rng, n_points, n_resonances)]
    n_in = int(round(inside_frac * n_rays))
    n_out = n_rays - n_in
    pin = rng.integers(0, pins * pins, n_in)
    rr = 0.45 * np.sqrt(rng.random(n_in))
    th = 2.0 * math.pi * rng.random(n_in)
    xi = ((pin % pins) + 0.5) * pitch + rr * np.cos(th)
    yi = ((pin // pins) + 0.5) * pitch + rr * np.sin(th)
    zi = nz * dz * rng.random(n_in)
    xo, yo, zo = uniform_positions(rng, mesh, n_out)
    hi = mesh.hi
    x = np.concatenate([xi.astype(np.float32), xo])
    y = np.concatenate([yi.astype(np.float32), yo])
    z = np.concatenate([zi.astype(np.float32), zo])
    for arr, h in ((x, hi[0]), (y, hi[1]), (z, hi[2])):
        np.minimum(arr, np.nextafter(np.float32(h), np.float32(-np.inf)), out=arr)
    u, v, w = isotropic_dirs(rng, n_rays)
    E = log_uniform(rng, n_rays)
    wt = np.ones(n_rays, np.float32)
    return Problem("pinlattice", mesh, tables, None, make_rays(x, y, z, u, v, w, E, wt))


def graded_edges(fine_cells: int, fine_width: float, grow: float, coarse_width: float,
                 half_width: float) -> np.ndarray:
    """Symmetric graded edges: fine_cells cells of fine_width centred on 0,
    then cells growing by the factor grow up to coarse_width on each side
    until |x| reaches half_width (the last cell is cut at half_width)."""
    core = fine_cells * fine_width / 2.0
    right = list(np.linspace(0.0, core, fine_cells // 2 + 1)) if fine_cells % 2 == 0 else None
    if right is None:
        raise ValueError("fine_cells must be even")
    w = fine_width
    x = core
    while x < half_width - 1e-12:
        w = min(w * grow, coarse_width)
        x = min(x + w, half_width)
        right.append(x)
    right = np.asarray(right)
    return np.concatenate([-right[:0:-1], right])


def graded_assembly(seed: int = 5, pins: int = 16, cells_per_pin: int = 21, reflector: float = 30.0,
                    nz: int = 5, height: float = 100.0, n_rays: int = 1 << 24,
                    n_points: int = 20000, n_resonances: int = 200,
                    inside_frac: float = 0.7) -> Problem:
    """A 16x16 pin assembly on a graded (rectilinear) mesh.

    The PWR test put a 0.6 mm mesh over the whole 340 x 340 x 5 problem,
    reflector included; a non-uniform Cartesian mesh (Sec. 6 outlook) keeps
    0.6 mm cells (1.26 cm pitch / 21) over the assembly and grows them by
    1.1x per cell up to 2 cm through a 30 cm solution-and-graphite
    reflector.  Materials: 0 moderator, 1 fuel (r < 0.36), 2 void gap
    (0.36 <= r < 0.40), 3 cladding (0.40 <= r < 0.45), 4 uranyl-nitrate-like
    solution (first 10 cm outside the assembly), 5 graphite beyond; nz
    uniform layers over the height.  70% of starts uniform in the fuel
    discs, the rest uniform over the box; energies 1/E; seed 5.
    """
    rng = np.random.default_rng(seed)
    pitch = 1.26
    half_core = pins * pitch / 2.0
    xe = graded_edges(pins * cells_per_pin, pitch / cells_per_pin, 1.1, 2.0, half_core + reflector)
    ze = np.linspace(0.0, height, nz + 1)
    c = 0.5 * (xe[:-1] + xe[1:])
    inside = np.abs(c) < half_core
    local = np.mod(c + half_core, pitch) - 0.5 * pitch
    r = np.sqrt(local[None, :] ** 2 + local[:, None] ** 2)  # [iy][ix]
    core = inside[None, :] & inside[:, None]
    layer = np.zeros(r.shape, np.uint8)
    layer[core & (r < 0.45)] = 3
    layer[core & (r < 0.40)] = 2
    layer[core & (r < 0.36)] = 1
    dist = np.maximum(np.abs(c)[None, :], np.abs(c)[:, None]) - half_core
    layer[(~core) & (dist < 10.0)] = 4
    layer[(~core) & (dist >= 10.0)] = 5
    mat = np.ascontiguousarray(np.broadcast_to(layer, (nz, len(c), len(c))))
    mesh = RectMesh(xe, xe.copy(), ze, mat)
    tables = [xs_table(rng, n_points, n_resonances), xs_table(rng, n_points, n_resonances), None,
              xs_table(rng, n_points, n_resonances), xs_table(rng, n_points, n_resonances),
              xs_table(rng, n_points, n_resonances)]
    n_in = int(round(inside_frac * n_rays))
    n_out = n_rays - n_in
    pin = rng.integers(0, pins * pins, n_in)
    rr = 0.36 * np.sqrt(rng.random(n_in))
    th = 2.0 * math.pi * rng.random(n_in)
    xi = -half_core + ((pin % pins) + 0.5) * pitch + rr * np.cos(th)
    yi = -half_core + ((pin // pins) + 0.5) * pitch + rr * np.sin(th)
    zi = height * rng.random(n_in)
    xo, yo, zo = uniform_positions(rng, mesh, n_out)
    hi = mesh.hi
    x = np.concatenate([xi.astype(np.float32), xo])
    y = np.concatenate([yi.astype(np.float32), yo])
    z = np.concatenate([zi.astype(np.float32), zo])
    for arr, h in ((x, hi[0]), (y, hi[1]), (z, hi[2])):
        np.minimum(arr, np.nextafter(np.float32(h), np.float32(-np.inf)), out=arr)
    u, v, w = isotropic_dirs(rng, n_rays)
    E = log_uniform(rng, n_rays)
    wt = np.ones(n_rays, np.float32)
    return Problem("graded", mesh, tables, None, make_rays(x, y, z, u, v, w, E, wt))


def batched_problems(seed: int = 3, n_problems: int = 1024, side_lo: int = 16,
                     side_hi: int = 128, rays_lo: float = 1e3, rays_hi: float = 1e6,
                     n_points: int = 1000, n_resonances: int = 5) -> List[Problem]:
    """Many independent problems of uneven size for the batched form.

    Cubic meshes of 1 cm cells with side log-uniform in [16, 128], 2-8
    materials per problem (every one a 1,000-point, 5-resonance table, no
    void), uniform-random layout, ray counts log-uniform in [1e3, 1e6],
    one group per problem; seed 3.
    """
    rng = np.random.default_rng(seed)
    out = []
    for p in range(n_problems):
        side = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        nr = int(round(math.exp(rng.uniform(math.log(rays_lo), math.log(rays_hi)))))
        nm = int(rng.integers(2, 9))
        tables = [xs_table(rng, n_points, n_resonances) for _ in range(nm)]
        mat = rng.integers(0, nm, size=(side, side, side), dtype=np.uint8)
        mesh = Mesh(side, side, side, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, mat)
        x, y, z = uniform_positions(rng, mesh, nr)
        u, v, w = isotropic_dirs(rng, nr)
        E = log_uniform(rng, nr)
        wt = np.ones(nr, np.float32)
        out.append(Problem(f"batch{p}", mesh, tables, None, make_rays(x, y, z, u, v, w, E, wt)))
    return out


def surrogate_mesh(seed: int = 4, n: int = 32, n_rays: int = 1 << 24, n_materials: int = 16,
                   n_points: int = 20000, n_resonances: int = 200) -> Problem:
    """n^3 mesh of 1 cm cells with 16 materials (uniform-random layout).

    Tables come from the 20,000-point, 200-resonance generator; 2^24 rays;
    one group; seed 4.  Used for the learned cross-section surrogate.
    """
    rng = np.random.default_rng(seed)
    tables = [xs_table(rng, n_points, n_resonances) for _ in range(n_materials)]
    mat = rng.integers(0, n_materials, size=(n, n, n), dtype=np.uint8)
    mesh = Mesh(n, n, n, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, mat)
    x, y, z = uniform_positions(rng, mesh, n_rays)
    u, v, w = isotropic_dirs(rng, n_rays)
    E = log_uniform(rng, n_rays)
    wt = np.ones(n_rays, np.float32)
    return Problem("surrogate32", mesh, tables, None, make_rays(x, y, z, u, v, w, E, wt))


def take_rays(p: Problem, idx) -> Problem:
    """The same problem restricted to a subset (slice or index array) of its rays."""
    return dataclasses.replace(p, rays={k: np.ascontiguousarray(v[idx]) for k, v in p.rays.items()})


def ray_batches(p: Problem, n_batches: int) -> Sequence[dict]:
    n = p.n_rays
    bounds = [n * i // n_batches for i in range(n_batches + 1)]
    return [{k: v[bounds[i]:bounds[i + 1]] for k, v in p.rays.items()} for i in range(n_batches)]
