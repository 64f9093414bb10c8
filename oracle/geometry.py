"""Oracle: Dey--Mittra cut fractions from a nodal level set (plain FP64, numpy).

Definitions (Bauer, Werner & Cary, arXiv:1301.3794):

* Sec. 2 (Eq. farInt, Fig. dmFace): l and a are the parts of an edge length and
  a face area lying *outside* the conductor; the fractions are L = l / Delta and
  A = a / (Delta Delta').
* Sec. 5.1 (Eq. divBInt, Fig. dmVol): v is the part of the cell volume outside
  the conductor; V = v / (dx dy dz).
* Sec. 6.1: cut-cell volumes are built from tetrahedral subvolumes conforming to
  the embedded surface, exact in the limit of smooth boundaries.

Reading used here (the paper does not say how the surface is represented): the
surface is the zero set of the piecewise-linear interpolant of the nodal level
set phi on the Kuhn split of each cell into 6 tetrahedra (all sharing the
(0,0,0)-(1,1,1) diagonal).  That split is conforming across cells and induces,
on every face, the diagonal from its lowest to its highest corner; the same
interpolant then defines l on edges, a on face triangles and v in tetrahedra,
so the three measures are mutually consistent.  phi < 0 is vacuum, phi >= 0 is
conductor (a node exactly on the surface counts as conductor).

Domain walls are perfect conductors (Sec. 6): normal faces and tangential edges
on the outer walls get fraction 0.  A wall may instead be a symmetry plane of
the perfect-magnetic-conductor kind (Sec. 6.3, the quarter TESLA cavity); the
reading used here puts that plane half a cell outside the wall's node plane
(through the centres of the mirrored cells), where the Yee unknowns of fields
that are even under the mirror map pair up exactly with their images: the
wall's normal faces and tangential edges then keep their fractions, and every
entity beyond the wall is zero.  A perfect-electric symmetry plane (Sec. 6.2,
the octant sphere) lies on the wall's node plane and is the ordinary wall.

Pins (tests/test_oracle_geometry.py): simplex fractions against brute-force
lattice sampling and the divided-difference closed form; half-space and corner
cuts of a cube against exact volumes; sphere volume convergence to 4 pi / 3 at
second order; the paper's magnetic-component counts of Tab. invPerf.
"""
from __future__ import annotations

import itertools

import numpy as np


def _root_frac(u, v):
    """Fraction of the way from a vertex with value u to the zero of the linear
    interpolant between u and v (u and v of opposite sign).  Entries where the
    signs agree are never selected by the callers; they may hold inf/nan."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return u / (u - v)


def segment_fraction(p0, p1):
    """Length fraction of {phi < 0} on a segment with endpoint values p0, p1."""
    p0 = np.asarray(p0, dtype=np.float64)
    p1 = np.asarray(p1, dtype=np.float64)
    n0 = p0 < 0
    n1 = p1 < 0
    out = np.where(n0 & n1, 1.0, 0.0)
    out = np.where(n0 & ~n1, _root_frac(p0, p1), out)
    out = np.where(~n0 & n1, _root_frac(p1, p0), out)
    return out


def triangle_fraction(p0, p1, p2):
    """Area fraction of {phi < 0} on a triangle with linear phi.

    Vertex values are sorted, q0 <= q1 <= q2, so the negative vertices come
    first.  One negative vertex: a similar corner triangle with edge ratios
    t01, t02.  Two: the whole minus the positive corner triangle."""
    q = np.sort(np.stack(np.broadcast_arrays(p0, p1, p2)).astype(np.float64), axis=0)
    q0, q1, q2 = q
    nneg = (q < 0).sum(axis=0)
    with np.errstate(invalid="ignore"):
        one = _root_frac(q0, q1) * _root_frac(q0, q2)
        two = 1.0 - _root_frac(q2, q0) * _root_frac(q2, q1)
    out = np.zeros_like(q0)
    out = np.where(nneg == 1, one, out)
    out = np.where(nneg == 2, two, out)
    out = np.where(nneg == 3, 1.0, out)
    return out


def tet_fraction(p0, p1, p2, p3):
    """Volume fraction of {phi < 0} in a tetrahedron with linear phi.

    Sorted values q0 <= ... <= q3.  One negative vertex: corner tetrahedron,
    fraction t01 t02 t03.  Three: the whole minus the positive corner.  Two
    (q0, q1 negative): the negative part is a triangular prism with vertices
    q0, q1 and the zero points on the four mixed edges; split into three
    tetrahedra (vertex q0 with the face (p02, p03, p13), vertex q0 with
    (p02, p12, p13), vertex q0 with (q1, p12, p13)), whose volumes relative to
    the whole are alpha beta (1 - delta), alpha delta (1 - gamma) and
    gamma delta with alpha = t02, beta = t03, gamma = t12, delta = t13."""
    q = np.sort(np.stack(np.broadcast_arrays(p0, p1, p2, p3)).astype(np.float64), axis=0)
    q0, q1, q2, q3 = q
    nneg = (q < 0).sum(axis=0)
    with np.errstate(invalid="ignore"):
        one = _root_frac(q0, q1) * _root_frac(q0, q2) * _root_frac(q0, q3)
        three = 1.0 - _root_frac(q3, q0) * _root_frac(q3, q1) * _root_frac(q3, q2)
    al = _root_frac(q0, q2)
    be = _root_frac(q0, q3)
    ga = _root_frac(q1, q2)
    de = _root_frac(q1, q3)
    with np.errstate(invalid="ignore"):
        two = al * be * (1.0 - de) + al * de * (1.0 - ga) + ga * de
    out = np.zeros_like(q0)
    out = np.where(nneg == 1, one, out)
    out = np.where(nneg == 2, two, out)
    out = np.where(nneg == 3, three, out)
    out = np.where(nneg == 4, 1.0, out)
    return out


def _quad_fraction(c00, c10, c01, c11):
    """Face fraction: the face (local corners c_ab, a along the first in-plane
    axis, b along the second) is split by its c00-c11 diagonal into two
    triangles of equal area."""
    return 0.5 * (triangle_fraction(c00, c10, c11) + triangle_fraction(c00, c01, c11))


WALLS_PEC = ("pec",) * 6


def fractions(phi, a_min=0.0, walls=WALLS_PEC):
    """Cut fractions of every edge, face and cell.

    ``phi`` has shape (nz+1, ny+1, nx+1).  Returns a dict of arrays in natural
    shapes: Lx (nz+1, ny+1, nx), Ly (nz+1, ny, nx+1), Lz (nz, ny+1, nx+1),
    Ax (nz, ny, nx+1), Ay (nz, ny+1, nx), Az (nz+1, ny, nx), V (nz, ny, nx).

    ``a_min`` > 0 neglects faces with 0 < A < a_min (Sec. 3): the face and the
    edges bounding it get fraction 0.

    ``walls``: the kind of each outer wall, in the order x-low, x-high, y-low,
    y-high, z-low, z-high: "pec" (closed) or "pmc" (symmetry plane half a cell
    outside, its faces and edges open).
    """
    p = np.asarray(phi, dtype=np.float64)
    nz, ny, nx = (s - 1 for s in p.shape)
    f = {}
    # edges (Sec. 2: length outside the conductor)
    f["Lx"] = segment_fraction(p[:, :, :-1], p[:, :, 1:])
    f["Ly"] = segment_fraction(p[:, :-1, :], p[:, 1:, :])
    f["Lz"] = segment_fraction(p[:-1, :, :], p[1:, :, :])
    # faces: x-face corners in (y, z); y-face in (x, z); z-face in (x, y)
    f["Ax"] = _quad_fraction(p[:-1, :-1, :], p[:-1, 1:, :], p[1:, :-1, :], p[1:, 1:, :])
    f["Ay"] = _quad_fraction(p[:-1, :, :-1], p[:-1, :, 1:], p[1:, :, :-1], p[1:, :, 1:])
    f["Az"] = _quad_fraction(p[:, :-1, :-1], p[:, :-1, 1:], p[:, 1:, :-1], p[:, 1:, 1:])
    # cells: 6 Kuhn tetrahedra, vertex path (0,0,0) -> +e_a -> +e_b -> (1,1,1)
    def corner(off):
        ox, oy, oz = off
        return p[oz:oz + nz, oy:oy + ny, ox:ox + nx]
    vol = np.zeros((nz, ny, nx))
    for perm in itertools.permutations(range(3)):
        path = [(0, 0, 0)]
        cur = [0, 0, 0]
        for ax in perm:
            cur[ax] = 1
            path.append(tuple(cur))
        vol += tet_fraction(*(corner(v) for v in path))
    f["V"] = vol / 6.0
    # perfect-conductor walls: their normal faces and tangential edges are closed
    walls = tuple(walls)
    if len(walls) != 6 or any(w not in ("pec", "pmc") for w in walls):
        raise ValueError("walls: six entries, each 'pec' or 'pmc'")
    for axis in range(3):                      # 0 = x, 1 = y, 2 = z
        ax_arr = 2 - axis                      # array axis of that direction (arrays are (z, y, x))
        for side, idx in ((0, 0), (1, -1)):
            if walls[2 * axis + side] != "pec":
                continue
            sl = [slice(None)] * 3
            sl[ax_arr] = idx
            sl = tuple(sl)
            f["A" + "xyz"[axis]][sl] = 0.0     # normal faces
            for e in range(3):                 # tangential edges
                if e != axis:
                    f["L" + "xyz"[e]][sl] = 0.0
    if a_min > 0.0:
        _neglect_faces(f, a_min)
    return f


def _neglect_faces(f, a_min):
    """Sec. 3: faces with area fraction below a_min are dropped, together with
    the electric-field edges bounding them."""
    Lx, Ly, Lz = f["Lx"], f["Ly"], f["Lz"]
    small = (f["Ax"] > 0) & (f["Ax"] < a_min)          # x-face (k, j, i): y-edges k, k+1; z-edges j, j+1
    kk, jj, ii = np.nonzero(small)
    Ly[kk, jj, ii] = 0; Ly[kk + 1, jj, ii] = 0; Lz[kk, jj, ii] = 0; Lz[kk, jj + 1, ii] = 0
    f["Ax"][small] = 0.0
    small = (f["Ay"] > 0) & (f["Ay"] < a_min)          # y-face: x-edges k, k+1; z-edges i, i+1
    kk, jj, ii = np.nonzero(small)
    Lx[kk, jj, ii] = 0; Lx[kk + 1, jj, ii] = 0; Lz[kk, jj, ii] = 0; Lz[kk, jj, ii + 1] = 0
    f["Ay"][small] = 0.0
    small = (f["Az"] > 0) & (f["Az"] < a_min)          # z-face: x-edges j, j+1; y-edges i, i+1
    kk, jj, ii = np.nonzero(small)
    Lx[kk, jj, ii] = 0; Lx[kk, jj + 1, ii] = 0; Ly[kk, jj, ii] = 0; Ly[kk, jj, ii + 1] = 0
    f["Az"][small] = 0.0


def coarsen_phi(phi):
    """Level set of the next-coarser grid: the nodes of every second fine node."""
    return np.ascontiguousarray(np.asarray(phi)[::2, ::2, ::2])
