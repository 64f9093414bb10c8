"""Seeded synthetic cavity geometries: the inputs of the Dey--Mittra eigensolver.

This module only produces inputs -- a Yee grid description and the level set
phi sampled at the grid nodes (phi < 0 is vacuum, phi >= 0 is conductor) plus
the shift, mode count and seeds of each workload.  It holds none of the
method's arithmetic (no fractions, no operators), so that both the CPU oracle
and the CUDA path can take their inputs from it without sharing method code.

Workloads (the paper's test problems, Sec. 6, rebuilt synthetically):

* ``sphere``       spherical PEC cavity of radius R (Sec. 6.1 and 6.2, the
                   TM/TE modes of Eq. waveb with analytic frequencies),
* ``box``          grid-aligned PEC box (every fraction is 0 or 1: plain Yee,
                   Eq. discWaveB, with closed-form discrete eigenvalues),
* ``ellipsoid``    axis-aligned ellipsoid with seeded semi-axes,
* ``nine_cell``    a synthetic 9-cell elliptical accelerating cavity standing
                   in for the TESLA cavity of Sec. 6.3 (whose exact shape is
                   not given in the paper).

Node (i, j, k) sits at ``origin + (i*dx, j*dy, k*dz)``; phi arrays have shape
``(nz+1, ny+1, nx+1)`` (i fastest, C order).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Grid", "Workload", "node_coords", "sphere_phi", "box_phi", "ellipsoid_phi",
    "nine_cell_profile", "nine_cell_phi", "sphere_workload", "octant_sphere_workload", "box_workload",
    "ellipsoid_workload", "nine_cell_workload", "batch_workloads", "SEED_BASE",
]

SEED_BASE = 1301
# (kR)^2 of the lowest (TM_1) mode of a unit PEC sphere, kR = 2.743707: only
# used to place the batch recipe's shifts below each cavity's lowest mode
TM1_SPHERE_K2 = 2.743707 ** 2


@dataclasses.dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def shape_nodes(self):
        return (self.nz + 1, self.ny + 1, self.nx + 1)

    @property
    def n_cells(self):
        return self.nx * self.ny * self.nz

    @property
    def n_faces(self):
        nx, ny, nz = self.nx, self.ny, self.nz
        return (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1)

    @property
    def n_edges(self):
        nx, ny, nz = self.nx, self.ny, self.nz
        return nx * (ny + 1) * (nz + 1) + (nx + 1) * ny * (nz + 1) + (nx + 1) * (ny + 1) * nz


@dataclasses.dataclass
class Workload:
    """One eigenproblem: grid, nodal level set, shift sigma and mode count."""
    name: str
    grid: Grid
    phi: np.ndarray          # (nz+1, ny+1, nx+1) float64
    sigma: float
    nev: int
    seed: int
    meta: dict = dataclasses.field(default_factory=dict)
    # outer-wall kinds (x-low, x-high, y-low, y-high, z-low, z-high): "pec" is
    # a perfect conductor on the wall's node plane, "pmc" a magnetic symmetry
    # plane half a cell outside it
    walls: tuple = ("pec",) * 6


def node_coords(g: Grid):
    """Coordinates of all nodes, each array of shape (nz+1, ny+1, nx+1)."""
    x = g.origin[0] + g.dx * np.arange(g.nx + 1, dtype=np.float64)
    y = g.origin[1] + g.dy * np.arange(g.ny + 1, dtype=np.float64)
    z = g.origin[2] + g.dz * np.arange(g.nz + 1, dtype=np.float64)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def sphere_phi(g: Grid, center=(0.0, 0.0, 0.0), radius=1.0):
    """Signed distance |x - c| - R (negative inside the cavity)."""
    X, Y, Z = node_coords(g)
    return np.sqrt((X - center[0]) ** 2 + (Y - center[1]) ** 2 + (Z - center[2]) ** 2) - radius


def box_phi(g: Grid, lo, hi):
    """Signed box function: negative strictly inside [lo, hi], zero on its walls."""
    X, Y, Z = node_coords(g)
    parts = []
    for c, a, b in ((X, lo[0], hi[0]), (Y, lo[1], hi[1]), (Z, lo[2], hi[2])):
        parts.append(np.maximum(a - c, c - b))
    return np.maximum(np.maximum(parts[0], parts[1]), parts[2])


def ellipsoid_phi(g: Grid, center, semi_axes):
    """Level set of an axis-aligned ellipsoid; its zero set is the exact surface."""
    X, Y, Z = node_coords(g)
    a, b, c = semi_axes
    q = np.sqrt(((X - center[0]) / a) ** 2 + ((Y - center[1]) / b) ** 2 + ((Z - center[2]) / c) ** 2)
    return (q - 1.0) * min(a, b, c)


# ---------------------------------------------------------------------------
# synthetic 9-cell elliptical cavity (stand-in for the TESLA cavity, Sec. 6.3)
# ---------------------------------------------------------------------------

def _tangent_slope(a, b, zi, ri, A, B, ze, re):
    """Slope of the line tangent to the iris ellipse (centre (zi, ri), half-axes
    a along z, b along r; touched on its lower-right quarter) and the equator
    ellipse (centre (ze, re), half-axes A, B; touched on its upper-left quarter)."""
    def gap(m):
        c1 = ri - m * zi - math.sqrt(a * a * m * m + b * b)
        c2 = re - m * ze + math.sqrt(A * A * m * m + B * B)
        return c1 - c2
    lo, hi = 1e-6, 1e6
    if gap(lo) * gap(hi) > 0:
        raise ValueError("no common tangent for these cell parameters")
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if gap(lo) * gap(mid) <= 0:
            hi = mid
        else:
            lo = mid
    return math.sqrt(lo * hi)


def nine_cell_profile(z, cell_length, r_equator, r_iris, n_cells=9,
                      eq_axes=None, iris_axes=None, equator_scale=None):
    """Wall radius r(z) of the synthetic multi-cell cavity.

    Irises sit at z = n*cell_length (n = 0..n_cells), equators half-way between.
    Each half-cell is an iris ellipse arc, a common tangent line and an equator
    ellipse arc.  Outside [0, n_cells*cell_length] the beam pipe has radius
    ``r_iris``.  ``equator_scale[n]`` scales the equator radius of cell n.
    """
    Lc = cell_length
    A, B = eq_axes if eq_axes is not None else (0.35 * Lc, 0.35 * Lc)
    a, b = iris_axes if iris_axes is not None else (0.10 * Lc, 0.15 * Lc)
    z = np.asarray(z, dtype=np.float64)
    r = np.full(z.shape, float(r_iris))
    scales = np.ones(n_cells) if equator_scale is None else np.asarray(equator_scale, dtype=np.float64)
    for n in range(n_cells):
        req = r_equator * scales[n]
        half = 0.5 * Lc
        zi, ri = 0.0, r_iris + b
        ze, re = half, req - B
        m = _tangent_slope(a, b, zi, ri, A, B, ze, re)
        u1 = math.atan(-b / (a * m))
        zt1 = zi + a * math.cos(u1)
        u2 = math.pi - math.atan(B / (A * m))
        zt2 = ze + A * math.cos(u2)
        c = ri - m * zi - math.sqrt(a * a * m * m + b * b)
        # local coordinate s in [0, Lc], mirrored about the equator
        s = z - n * Lc
        inside = (s >= 0.0) & (s <= Lc)
        t = np.where(s <= half, s, Lc - s)
        t = np.clip(t, 0.0, half)
        ri_arc = ri - b * np.sqrt(np.clip(1.0 - (t / a) ** 2, 0.0, None))
        line = m * t + c
        eq_arc = re + B * np.sqrt(np.clip(1.0 - ((t - ze) / A) ** 2, 0.0, None))
        prof = np.where(t <= zt1, ri_arc, np.where(t <= zt2, line, eq_arc))
        r = np.where(inside, prof, r)
    return r


def nine_cell_phi(g: Grid, cell_length, r_equator, r_iris, n_cells=9, equator_scale=None):
    X, Y, Z = node_coords(g)
    r = nine_cell_profile(Z, cell_length, r_equator, r_iris, n_cells=n_cells, equator_scale=equator_scale)
    return np.sqrt(X ** 2 + Y ** 2) - r


# ---------------------------------------------------------------------------
# the paper's workloads as seeded synthetic recipes
# ---------------------------------------------------------------------------

def sphere_workload(n=16, radius=1.0, half_width=1.1, sigma=7.0, nev=4, offset_seed=None):
    """Sphere of radius ``radius`` in [-half_width, half_width]^3 on an n^3 grid.

    With ``offset_seed`` the centre moves by a seeded uniform shift in [0, dx)^3
    so that the cut fractions span (0, 1)."""
    h = 2.0 * half_width / n
    g = Grid(n, n, n, h, h, h, (-half_width, -half_width, -half_width))
    center = np.zeros(3)
    seed = -1
    if offset_seed is not None:
        seed = int(offset_seed)
        center = np.random.default_rng(seed).uniform(0.0, h, size=3)
    return Workload(f"sphere{n}", g, sphere_phi(g, center, radius), sigma, nev, seed,
                    {"center": tuple(center), "radius": radius})


def octant_sphere_workload(n=16, radius=1.0, extent=1.1, sigma=20.0, nev=1):
    """The positive octant of a sphere centred at the origin on [0, extent]^3
    (Sec. 6.2's convergence study): the grid's walls at x, y, z = 0 are the
    perfectly conducting symmetry planes."""
    h = extent / n
    g = Grid(n, n, n, h, h, h, (0.0, 0.0, 0.0))
    return Workload(f"octant{n}", g, sphere_phi(g, (0.0, 0.0, 0.0), radius), sigma, nev, -1,
                    {"center": (0.0, 0.0, 0.0), "radius": radius})


def quarter_nine_cell_workload(nq=48, nz=1152, seed=None, sigma=None, nev=9, n_cavities=1, gap_cells=4,
                               cell_length=0.1154, r_equator=0.1033, r_iris=0.035):
    """The quarter x >= 0, y >= 0 of the synthetic 9-cell cavity with magnetic
    symmetry planes x = 0 and y = 0 (Sec. 6.3: the TM010-like accelerating
    modes are then the lowest ones).  The grid has nq cells of the full
    cavity's 2 nq-cell spacing across x and y, its first node planes half a
    cell from the symmetry planes (origin (h/2, h/2, z0)).  ``n_cavities`` > 1
    strings that many cavities end to end along z, beam pipes of
    ``gap_cells`` cell lengths between them (the cryomodule of Sec. 6.3);
    nz is then the cell count of the whole string."""
    hw = 1.065 * r_equator
    h = 2 * hw / (2 * nq)
    period = (9 + gap_cells) * cell_length
    z0 = -2.0 * cell_length
    z1 = (n_cavities - 1) * period + 11.0 * cell_length
    g = Grid(nq, nq, nz, h, h, (z1 - z0) / nz, (0.5 * h, 0.5 * h, z0))
    scale = None
    if seed is not None:
        scale = 1.0 + 0.01 * np.random.default_rng(seed).standard_normal(9)
    X, Y, Z = node_coords(g)
    r = np.full(Z.shape, float(r_iris))
    for c in range(n_cavities):
        rc = nine_cell_profile(Z - c * period, cell_length, r_equator, r_iris, equator_scale=scale)
        r = np.maximum(r, rc)
    phi = np.sqrt(X ** 2 + Y ** 2) - r
    if sigma is None:
        sigma = 0.25 * (math.pi / (z1 - z0)) ** 2
    name = f"quarter_ninecell{nq}x{nq}x{nz}" + (f"_string{n_cavities}" if n_cavities > 1 else "")
    return Workload(name, g, phi, sigma, nev, -1 if seed is None else seed,
                    {"cell_length": cell_length, "r_equator": r_equator, "r_iris": r_iris,
                     "n_cavities": n_cavities, "symmetry_planes": "x = 0 and y = 0, magnetic"},
                    walls=("pmc", "pec", "pmc", "pec", "pec", "pec"))


def box_workload(nx=12, ny=10, nz=8, lx=1.0, ly=0.8, lz=0.6, sigma=7.0, nev=4):
    """Grid-aligned PEC box filling the whole grid: every fraction is 0 or 1."""
    g = Grid(nx, ny, nz, lx / nx, ly / ny, lz / nz, (0.0, 0.0, 0.0))
    # The level set is negative on every node (a box half a cell larger than
    # the grid); the perfectly conducting outer walls of the grid then form the
    # cavity.  Putting phi = 0 on the wall nodes instead would let the
    # piecewise-linear surface close triangles whose three corners all lie on
    # walls.
    pad = 0.5 * min(g.dx, g.dy, g.dz)
    phi = box_phi(g, (-pad, -pad, -pad), (lx + pad, ly + pad, lz + pad))
    return Workload(f"box{nx}x{ny}x{nz}", g, phi, sigma, nev, -1, {"lengths": (lx, ly, lz)})


def ellipsoid_workload(n=192, seed=SEED_BASE + 3, sigma=5.0, nev=16):
    """Seeded axis-aligned ellipsoid, semi-axes U[0.6, 1.0], domain half-width
    1.1 * max semi-axis, cubic cells, seeded sub-cell centre offset."""
    rng = np.random.default_rng(seed)
    axes = rng.uniform(0.6, 1.0, size=3)
    hw = 1.1 * float(axes.max())
    h = 2.0 * hw / n
    g = Grid(n, n, n, h, h, h, (-hw, -hw, -hw))
    center = rng.uniform(0.0, h, size=3)
    return Workload(f"ellipsoid{n}", g, ellipsoid_phi(g, center, axes), sigma, nev, seed,
                    {"center": tuple(center), "semi_axes": tuple(axes)})


def nine_cell_workload(nxy=96, nz=1152, seed=None, sigma=None, nev=20,
                       cell_length=0.1154, r_equator=0.1033, r_iris=0.035):
    """Synthetic 9-cell cavity in metres: beam pipes of 2 cell lengths on each
    side, square cross-section of half-width 1.065 * r_equator.  ``seed`` draws
    per-cell equator radius scales 1 + 0.01 N(0, 1) (a perturbed variant)."""
    hw = 1.065 * r_equator
    z0 = -2.0 * cell_length
    z1 = 11.0 * cell_length
    g = Grid(nxy, nxy, nz, 2 * hw / nxy, 2 * hw / nxy, (z1 - z0) / nz, (-hw, -hw, z0))
    scale = None
    if seed is not None:
        scale = 1.0 + 0.01 * np.random.default_rng(seed).standard_normal(9)
    phi = nine_cell_phi(g, cell_length, r_equator, r_iris, equator_scale=scale)
    if sigma is None:
        # A shift of the order of the operator's smallest nonzero eigenvalue
        # (Sec. 4.1), kept below it: a quarter of (pi / L)^2, L the length of
        # the structure, the estimate of its lowest longitudinal grad-div mode.
        # K - sigma A is then positive definite.  A shift just below the
        # accelerating passband lies deep inside the spectrum, where the
        # multigrid-preconditioned inner solve stalls.
        sigma = 0.25 * (math.pi / (z1 - z0)) ** 2
    return Workload(f"ninecell{nxy}x{nxy}x{nz}", g, phi, sigma, nev, -1 if seed is None else seed,
                    {"cell_length": cell_length, "r_equator": r_equator, "r_iris": r_iris,
                     "equator_scale": None if scale is None else tuple(scale)})


def batch_workloads(count=48, seed=SEED_BASE + 4, sizes=(32, 48, 64, 80, 96)):
    """Uneven batch of cavities: spheres and ellipsoids with p = 1/2, grid size
    drawn from ``sizes``, 1-4 sorted shifts and 4-8 modes each.

    The shifts sit in the low end of each cavity's spectrum, as the paper's
    shift-and-invert discussion (Sec. 4.1) asks: sigma = u * 7.5279 / r^2 with
    u ~ U[0.3, 0.9] and r the largest semi-axis (the radius of a sphere), i.e.
    below the estimated lowest electromagnetic mode (7.5279 = (kR)^2 of the
    TM_1 sphere mode).  Shifts deep inside the spectrum make K - sigma A too
    indefinite for a multigrid-preconditioned inner solve.
    Returns a list of (Workload, shifts, nev)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(count):
        n = int(rng.choice(sizes))
        kind = "sphere" if rng.random() < 0.5 else "ellipsoid"
        nshift = int(rng.integers(1, 5))
        u = np.sort(rng.uniform(0.3, 0.9, size=nshift))
        nev = int(rng.integers(4, 9))
        sub = int(rng.integers(0, 2 ** 31 - 1))
        if kind == "sphere":
            shifts = u * TM1_SPHERE_K2
            w = sphere_workload(n=n, sigma=float(shifts[0]), nev=nev, offset_seed=sub)
        else:
            w = ellipsoid_workload(n=n, seed=sub, sigma=5.0, nev=nev)
            shifts = u * TM1_SPHERE_K2 / max(w.meta["semi_axes"]) ** 2
            w.sigma = float(shifts[0])
        w.name = f"{kind}{n}_{c}"
        out.append((w, [float(s) for s in shifts], nev))
    return out
