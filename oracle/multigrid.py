"""Oracle: the geometric multigrid V-cycles the library uses inside the inner solves.

The paper inverts K - sigma A (Eq. discLaplDM) and D A D^T (Eq. proj) with GMRES
preconditioned by algebraic multigrid: a V-cycle with one order-1 polynomial
smoother step per level on the way down and one on the way up (Sec. 6, opening
paragraphs).  The library replaces the algebraic hierarchy by a geometric one.
The V-cycles are written out here as plain sparse-matrix steps, in the order the
cycle takes them, so that each stage of the CUDA cycle can be compared element
by element.  Everything below is the library's design, not the paper's:

Vector cycle (faces, operator K - sigma A):
* coarse grid: every second node; cut fractions of the coarse grid are the
  averages of the fine fractions they cover (a coarse face = 4 fine faces, a
  coarse edge = 2 fine edges, a coarse cell = 8 fine cells), so every level sees
  the areas and volumes of the same fine surface; K_c - sigma A_c is the same
  formula at the coarse spacing;
* prolongation P: per face component, linear across the face plane (a fine face
  on a coarse plane copies it, a fine face half-way takes the mean of the two
  neighbours) and bilinear within the plane (weights 3/4, 1/4 towards the nearer
  and farther coarse face centre; at a domain wall the missing neighbour's
  weight goes to the nearer face), then masked by the open fine faces;
* restriction R = P^T / 8 (full weighting);
* smoother: damped Jacobi x <- x + omega D^-1 (f - (K - sigma A) x), D the
  diagonal, followed by a restricted additive Schwarz step on the *band*: the
  open faces adjacent to a cell within one cell (26-neighbourhood) of a cut
  cell (0 < V < 1).  The band is covered by bricks of b^3 nodes (a face
  belongs to the node at its lower corner); the subdomain of a brick is every
  band face whose node lies within one node of the brick (overlap 1).  From
  the residual r0 = f - (K - sigma A) x, each subdomain runs ``band_sweeps``
  damped Jacobi sweeps on its own rows, d <- d + omega D^-1 (r0 - K_SS d) from
  d = 0 (couplings to faces outside the subdomain stay at their start
  values), and x takes d on the faces the brick owns.  Without this step the
  cut-cell faces slow the cycle to ~0.6-0.7 per iteration at 32^3-64^3; with
  it (b = 8, 16 sweeps) it contracts at ~0.22 at 64^3 and ~0.30 at 128^3, in
  line with the paper's AMG (~0.25, Tab. invPerf).  With one brick covering
  the grid the step is plain band-restricted Jacobi;
* coarsest level: exact solve on its open faces.

Scalar cycle (cells, operator S = D A D^T):
* the same coarse fractions; prolongation P: a fine cell copies its parent
  (constant), masked by the active fine cells (cells with an open face);
  R = P^T / 8; damped Jacobi; coarsest: exact solve with, in each connected
  component of active cells, the lowest-index cell pinned to 0 (S is singular
  with one constant null vector per component), except in components that
  reach an open outer-wall face (a magnetic symmetry plane), which are regular.

Pins (tests/test_oracle_multigrid.py): P's partition of unity and exactness for
affine fields away from walls; restriction as the explicit transpose; the
coarsened fractions of a box stay 0/1 and average exactly; V-cycle contraction
on a box.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph

from . import geometry, operators
from .operators import shapes, _index_blocks


def can_coarsen(nx, ny, nz, max_coarse=4):
    """Halve the grid while every dimension is even, the coarse grid keeps at
    least 2 cells per dimension and the grid is larger than ``max_coarse``."""
    return (nx % 2 == 0 and ny % 2 == 0 and nz % 2 == 0 and max(nx, ny, nz) > max_coarse
            and min(nx, ny, nz) >= 4)


def coarsen_fractions(fr):
    """Coarse fractions as averages of the fine fractions they cover."""
    c = {}
    Ax, Ay, Az = fr["Ax"], fr["Ay"], fr["Az"]
    # x-face (k, j, i) of the coarse grid = fine x-faces (2k+b, 2j+a, 2i)
    c["Ax"] = 0.25 * (Ax[0::2, 0::2, 0::2] + Ax[0::2, 1::2, 0::2] + Ax[1::2, 0::2, 0::2] + Ax[1::2, 1::2, 0::2])
    c["Ay"] = 0.25 * (Ay[0::2, 0::2, 0::2] + Ay[0::2, 0::2, 1::2] + Ay[1::2, 0::2, 0::2] + Ay[1::2, 0::2, 1::2])
    c["Az"] = 0.25 * (Az[0::2, 0::2, 0::2] + Az[0::2, 0::2, 1::2] + Az[0::2, 1::2, 0::2] + Az[0::2, 1::2, 1::2])
    Lx, Ly, Lz = fr["Lx"], fr["Ly"], fr["Lz"]
    c["Lx"] = 0.5 * (Lx[0::2, 0::2, 0::2] + Lx[0::2, 0::2, 1::2])
    c["Ly"] = 0.5 * (Ly[0::2, 0::2, 0::2] + Ly[0::2, 1::2, 0::2])
    c["Lz"] = 0.5 * (Lz[0::2, 0::2, 0::2] + Lz[1::2, 0::2, 0::2])
    V = fr["V"]
    c["V"] = 0.125 * sum(V[a::2, b::2, d::2] for a in (0, 1) for b in (0, 1) for d in (0, 1))
    return c


def _axis_weights(idx, n_coarse, normal):
    """Per-axis interpolation stencil: list of (coarse index, weight) pairs."""
    if normal:
        even = idx % 2 == 0
        return [(idx // 2, np.where(even, 1.0, 0.5)),
                (np.where(even, idx // 2, idx // 2 + 1), np.where(even, 0.0, 0.5))]
    c = idx // 2
    nb = np.where(idx % 2 == 0, c - 1, c + 1)
    inside = (nb >= 0) & (nb < n_coarse)
    return [(c, np.where(inside, 0.75, 1.0)),
            (np.clip(nb, 0, n_coarse - 1), np.where(inside, 0.25, 0.0))]


def face_prolongation(nxc, nyc, nzc):
    """P: coarse faces -> fine faces (fine grid = 2x coarse), not masked."""
    nx, ny, nz = 2 * nxc, 2 * nyc, 2 * nzc
    shf, shc = shapes(nx, ny, nz), shapes(nxc, nyc, nzc)
    Ff, nff = _index_blocks(shf, ("fx", "fy", "fz"))
    Fc, nfc = _index_blocks(shc, ("fx", "fy", "fz"))
    rows, cols, vals = [], [], []
    for comp, normal_axis in (("fx", 2), ("fy", 1), ("fz", 0)):
        fine, coarse = Ff[comp], Fc[comp]
        idx = np.meshgrid(*(np.arange(s) for s in fine.shape), indexing="ij")
        per_axis = [_axis_weights(idx[ax], coarse.shape[ax], ax == normal_axis) for ax in range(3)]
        for ck, wk in per_axis[0]:
            for cj, wj in per_axis[1]:
                for ci, wi in per_axis[2]:
                    w = wk * wj * wi
                    m = w != 0
                    rows.append(fine[m]); cols.append(coarse[ck[m], cj[m], ci[m]]); vals.append(w[m])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nff, nfc))


def cell_prolongation(nxc, nyc, nzc):
    """P: coarse cells -> fine cells, each fine cell copies its parent."""
    nx, ny, nz = 2 * nxc, 2 * nyc, 2 * nzc
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    fine = (I + nx * (J + ny * K)).ravel()
    parent = (I // 2 + nxc * (J // 2 + nyc * (K // 2))).ravel()
    return sp.csr_matrix((np.ones(fine.size), (fine, parent)), shape=(nx * ny * nz, nxc * nyc * nzc))


def band_faces(fr, open_mask):
    """Open faces adjacent to a cell within one cell of a cut cell (0 < V < 1)."""
    V = fr["V"]
    cut = (V > 0) & (V < 1)
    nz, ny, nx = V.shape
    pad = np.pad(cut, 1)
    dil = np.zeros_like(cut)
    for a in range(3):
        for b in range(3):
            for c in range(3):
                dil |= pad[a:a + nz, b:b + ny, c:c + nx]
    bx = np.zeros((nz, ny, nx + 1), bool); bx[:, :, :-1] |= dil; bx[:, :, 1:] |= dil
    by = np.zeros((nz, ny + 1, nx), bool); by[:, :-1, :] |= dil; by[:, 1:, :] |= dil
    bz = np.zeros((nz + 1, ny, nx), bool); bz[:-1] |= dil; bz[1:] |= dil
    return np.concatenate([bx.ravel(), by.ravel(), bz.ravel()]) & open_mask


class VectorLevel:
    def __init__(self, grid, fr, sigma):
        self.grid = grid
        self.fr = fr
        self.ops = operators.DMOperators(grid, fr)
        self.sigma = sigma
        self.K = self.ops.K(sigma)
        d = self.K.diagonal()
        self.inv_d = np.where(self.ops.open & (d != 0), 1.0 / np.where(d != 0, d, 1.0), 0.0)
        self.mask = self.ops.open.astype(np.float64)
        self.band = band_faces(fr, self.ops.open).astype(np.float64)


class ScalarLevel:
    def __init__(self, grid, fr):
        self.grid = grid
        self.fr = fr
        self.ops = operators.DMOperators(grid, fr)
        S = self.ops.scalar_laplacian()
        self.active = np.asarray(abs(S).sum(axis=1)).ravel() > 0
        self.mask = self.active.astype(np.float64)
        self.S = S
        d = S.diagonal()
        self.inv_d = np.where(self.active, 1.0 / np.where(self.active, d, 1.0), 0.0)


def open_face_count(fr):
    return int((fr["Ax"] > 0).sum() + (fr["Ay"] > 0).sum() + (fr["Az"] > 0).sum())


# a level with at most this many open faces is the coarsest (solved exactly)
DENSE_COARSE = 2048


def level_fractions(grid, phi, max_coarse=4, fine=None, dense_coarse=DENSE_COARSE, walls=geometry.WALLS_PEC):
    """Grids and fractions of every level; ``fine`` replaces the fine-level
    fractions computed from phi (for perturbation studies).  Coarsening stops
    when the grid cannot be halved (``can_coarsen``) or when the current level
    has at most ``dense_coarse`` open faces (0: no such limit).  ``walls``: the
    outer-wall kinds of oracle.geometry.fractions (the coarse levels average
    the fine fractions, walls included)."""
    from workloads import Grid
    grids = [grid]
    frs = [geometry.fractions(phi, walls=walls) if fine is None else fine]
    g = grid
    while can_coarsen(g.nx, g.ny, g.nz, max_coarse) and (dense_coarse <= 0 or open_face_count(frs[-1]) > dense_coarse):
        g = Grid(g.nx // 2, g.ny // 2, g.nz // 2, 2 * g.dx, 2 * g.dy, 2 * g.dz, g.origin)
        grids.append(g)
        frs.append(coarsen_fractions(frs[-1]))
    return grids, frs


def build_vector_hierarchy(grid, phi, sigma, max_coarse=4, fine=None, dense_coarse=DENSE_COARSE,
                           walls=geometry.WALLS_PEC):
    grids, frs = level_fractions(grid, phi, max_coarse, fine, dense_coarse, walls)
    levels = [VectorLevel(g, f, sigma) for g, f in zip(grids, frs)]
    for l in range(len(levels) - 1):
        c = levels[l + 1].grid
        levels[l].P = face_prolongation(c.nx, c.ny, c.nz)
    return levels


def build_scalar_hierarchy(grid, phi, max_coarse=4, dense_coarse=DENSE_COARSE, walls=geometry.WALLS_PEC):
    grids, frs = level_fractions(grid, phi, max_coarse, dense_coarse=dense_coarse, walls=walls)
    levels = [ScalarLevel(g, f) for g, f in zip(grids, frs)]
    for l in range(len(levels) - 1):
        c = levels[l + 1].grid
        levels[l].P = cell_prolongation(c.nx, c.ny, c.nz)
    return levels


# -- vector V-cycle -----------------------------------------------------------

def jacobi(level, f, x, omega):
    return x + omega * level.inv_d * (f - level.K @ x)


def face_nodes(grid):
    """(i, j, k) of the lower-corner node of every face, natural [x | y | z] order."""
    out = []
    sh = shapes(grid.nx, grid.ny, grid.nz)
    for key in ("fx", "fy", "fz"):
        k, j, i = np.meshgrid(*[np.arange(n) for n in sh[key]], indexing="ij")
        out.append(np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1))
    return np.concatenate(out)


def band_subdomains(level, brick):
    """Subdomains of the band smoother: for every brick of brick^3 nodes that
    owns a band face, (rows of the subdomain, which of them the brick owns).
    A band face with lower node P is owned by brick floor(P / brick) and
    belongs to the subdomain of every brick B with B*brick - 1 <= P <= B*brick + brick
    on each axis (overlap of one node)."""
    key = (id(level), brick)
    cache = level.__dict__.setdefault("_subdomains", {})
    if key in cache:
        return cache[key]
    rows = np.nonzero(level.band > 0)[0]
    P = face_nodes(level.grid)[rows]
    own = P // brick
    out = []
    for B in np.unique(own, axis=0):
        inside = np.all((P >= B * brick - 1) & (P <= B * brick + brick), axis=1)
        r = rows[inside]
        owned = np.all(own[inside] == B, axis=1)
        out.append((r, owned))
    cache[key] = out
    return out


def band_schwarz(level, f, x, omega, sweeps, brick):
    """Restricted additive Schwarz step on the band (see the module header)."""
    if sweeps <= 0 or not level.band.any():
        return x
    r0 = f - level.K @ x
    Kc = level.K.tocsr()
    x = x.copy()
    for rows, owned in band_subdomains(level, brick):
        Kss = Kc[rows][:, rows]
        dinv = level.inv_d[rows]
        d = np.zeros(rows.size)
        for _ in range(sweeps):
            d = d + omega * dinv * (r0[rows] - Kss @ d)
        x[rows[owned]] += d[owned]
    return x


def smooth(level, f, x, omega, band_sweeps, from_zero=False, brick=8, jacobi_sweeps=1):
    """``jacobi_sweeps`` damped Jacobi sweeps (the first from x = 0 when
    ``from_zero``), then the band smoother."""
    x = omega * level.inv_d * f if from_zero else jacobi(level, f, x, omega)
    for _ in range(jacobi_sweeps - 1):
        x = jacobi(level, f, x, omega)
    return band_schwarz(level, f, x, omega, band_sweeps, brick)


def restrict(levels, l, r):
    """f_c = R r = P^T r / 8, masked by the open coarse faces."""
    return levels[l + 1].mask * (levels[l].P.T @ r) / 8.0


def prolong_add(levels, l, x, ec):
    return x + levels[l].mask * (levels[l].P @ ec)


def coarsest_solve(level, f):
    o = level.ops.open_idx
    Kd = level.K.tocsr()[o][:, o].toarray()
    x = np.zeros_like(f)
    x[o] = np.linalg.solve(Kd, f[o])
    return x


def vcycle(levels, f, omegas, band_sweeps=16, l=0, brick=8, band_sweeps_coarse=None, jacobi_sweeps=1):
    """e ~= (K_l - sigma A_l)^-1 f: one V(nu,nu) cycle from a zero guess, nu =
    ``jacobi_sweeps`` damped Jacobi sweeps per smoothing step.  The band
    smoother runs ``band_sweeps`` sweeps on the fine level and
    ``band_sweeps_coarse`` (default: the same) on the coarser ones."""
    lev = levels[l]
    if l == len(levels) - 1:
        return coarsest_solve(lev, f)
    coarse = band_sweeps if band_sweeps_coarse is None else band_sweeps_coarse
    sweeps = band_sweeps if l == 0 else coarse
    e = smooth(lev, f, None, omegas[l], sweeps, from_zero=True, brick=brick, jacobi_sweeps=jacobi_sweeps)
    r = f - lev.K @ e
    ec = vcycle(levels, restrict(levels, l, r), omegas, band_sweeps, l + 1, brick, coarse, jacobi_sweeps)
    e = prolong_add(levels, l, e, ec)
    return smooth(lev, f, e, omegas[l], sweeps, brick=brick, jacobi_sweeps=jacobi_sweeps)


# -- scalar V-cycle -----------------------------------------------------------

def scalar_coarsest_solve(level, f):
    """Exact solve with the lowest-index cell of every connected component of
    active cells pinned to 0 (components with an open wall face: none)."""
    act = np.nonzero(level.active)[0]
    Sa = level.S[act][:, act].tocsr()
    ncomp, labels = csgraph.connected_components(Sa, directed=False)
    grounded = level.ops.grounded_cells()[act]
    keep = np.ones(act.size, dtype=bool)
    for c in range(ncomp):
        members = np.nonzero(labels == c)[0]
        if not grounded[members].any():
            keep[members[0]] = False
    kk = np.nonzero(keep)[0]
    x = np.zeros_like(f)
    if kk.size:
        x[act[kk]] = np.linalg.solve(Sa[kk][:, kk].toarray(), f[act[kk]])
    return x


def scalar_vcycle(levels, f, omegas, l=0):
    lev = levels[l]
    if l == len(levels) - 1:
        return scalar_coarsest_solve(lev, f)
    e = omegas[l] * lev.inv_d * f
    r = f - lev.S @ e
    fc = levels[l + 1].mask * (lev.P.T @ r) / 8.0
    ec = scalar_vcycle(levels, fc, omegas, l + 1)
    e = e + lev.mask * (lev.P @ ec)
    return e + omegas[l] * lev.inv_d * (f - lev.S @ e)


def complexity(levels):
    """Sum over levels of open unknowns / fine open unknowns (cf. Tab. invPerf)."""
    n = [int(lev.mask.sum()) for lev in levels]
    return sum(n) / n[0]


def fgmres(apply, b, precond, tol=1e-10, restart=40, maxiter=400):
    """Right-preconditioned flexible GMRES (Saad 1993) with classical
    Gram-Schmidt applied twice; a plain reference for iteration counts."""
    n = b.size
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    hist = []
    total = 0
    while total < maxiter:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
        Vs = [r / beta]
        Zs = []
        H = np.zeros((restart + 1, restart))
        for j in range(restart):
            z = precond(Vs[j]); Zs.append(z)
            w = apply(z)
            for _ in range(2):
                h = np.array([v @ w for v in Vs])
                H[:j + 1, j] += h
                w = w - sum(hh * v for hh, v in zip(h, Vs))
            H[j + 1, j] = np.linalg.norm(w)
            Vs.append(w / H[j + 1, j])
            e1 = np.zeros(j + 2); e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
            res = np.linalg.norm(H[:j + 2, :j + 1] @ y - e1) / bnorm
            hist.append(res)
            total += 1
            if res <= tol or total >= maxiter:
                break
        x = x + np.array(Zs).T @ y
        if hist[-1] <= tol:
            break
    return x, hist
