"""Oracle: assembled sparse Yee / Dey--Mittra operators (plain FP64, scipy).

Orderings (natural, i fastest within each block):

* faces  = [x-faces (nz, ny, nx+1) | y-faces (nz, ny+1, nx) | z-faces (nz+1, ny, nx)]
* edges  = [x-edges (nz+1, ny+1, nx) | y-edges (nz+1, ny, nx+1) | z-edges (nz, ny+1, nx+1)]
* cells  = (nz, ny, nx)

x-face (i, j, k) sits at x = x_i and spans [y_j, y_j+1] x [z_k, z_k+1]; the
y-edge (i, j, k) runs from node (i, j, k) to (i, j+1, k); and so on.

Passages:
* C (edges -> faces), Eq. farInt with unit fractions: the x-row is
  (e_z(i,j+1,k) - e_z(i,j,k))/dy - (e_y(i,j,k+1) - e_y(i,j,k))/dz; C C^T is the
  vacuum curl-curl of Eq. discWaveB.
* D (faces -> cells), Eq. divB; -D^T is the gradient of Eq. gradPhi.
* Dey--Mittra: A = diag(face fractions), L = diag(edge fractions),
  V = diag(cell fractions) (Sec. 2, Eq. discWaveBDM; Sec. 5.1, Eq. divBDM).
* K(sigma) = C L C^T + A D^T V^-1 D A - sigma A, the A-scaled shifted vector
  Laplacian of Eq. discLaplDM (V^-1 taken as 0 on cells with V = 0).
* P_DM = I - D^T (D A D^T)^-1 D A, Eq. proj.

The unknowns are the open faces (A > 0); closed faces carry b = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph
import scipy.sparse.linalg as spla


def shapes(nx, ny, nz):
    return {
        "fx": (nz, ny, nx + 1), "fy": (nz, ny + 1, nx), "fz": (nz + 1, ny, nx),
        "ex": (nz + 1, ny + 1, nx), "ey": (nz + 1, ny, nx + 1), "ez": (nz, ny + 1, nx + 1),
        "c": (nz, ny, nx),
    }


def _index_blocks(sh, keys):
    out, off = {}, 0
    for k in keys:
        n = int(np.prod(sh[k]))
        out[k] = off + np.arange(n).reshape(sh[k])
        off += n
    return out, off


def curl(nx, ny, nz, dx, dy, dz):
    """C: edges -> faces (Eq. farInt with unit fractions)."""
    sh = shapes(nx, ny, nz)
    F, nf = _index_blocks(sh, ("fx", "fy", "fz"))
    E, ne = _index_blocks(sh, ("ex", "ey", "ez"))
    rows, cols, vals = [], [], []

    def add(r, c, v):
        rows.append(r.ravel()); cols.append(c.ravel()); vals.append(np.full(r.size, v))
    fx, fy, fz = F["fx"], F["fy"], F["fz"]
    ex, ey, ez = E["ex"], E["ey"], E["ez"]
    # x-face: d_y e_z - d_z e_y
    add(fx, ez[:, 1:, :], 1 / dy); add(fx, ez[:, :-1, :], -1 / dy)
    add(fx, ey[1:, :, :], -1 / dz); add(fx, ey[:-1, :, :], 1 / dz)
    # y-face: d_z e_x - d_x e_z
    add(fy, ex[1:, :, :], 1 / dz); add(fy, ex[:-1, :, :], -1 / dz)
    add(fy, ez[:, :, 1:], -1 / dx); add(fy, ez[:, :, :-1], 1 / dx)
    # z-face: d_x e_y - d_y e_x
    add(fz, ey[:, :, 1:], 1 / dx); add(fz, ey[:, :, :-1], -1 / dx)
    add(fz, ex[:, 1:, :], -1 / dy); add(fz, ex[:, :-1, :], 1 / dy)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nf, ne))


def divergence(nx, ny, nz, dx, dy, dz):
    """D: faces -> cells (Eq. divB)."""
    sh = shapes(nx, ny, nz)
    F, nf = _index_blocks(sh, ("fx", "fy", "fz"))
    cells = np.arange(nx * ny * nz).reshape(sh["c"])
    rows, cols, vals = [], [], []

    def add(c, v):
        rows.append(cells.ravel()); cols.append(c.ravel()); vals.append(np.full(cells.size, v))
    add(F["fx"][:, :, 1:], 1 / dx); add(F["fx"][:, :, :-1], -1 / dx)
    add(F["fy"][:, 1:, :], 1 / dy); add(F["fy"][:, :-1, :], -1 / dy)
    add(F["fz"][1:, :, :], 1 / dz); add(F["fz"][:-1, :, :], -1 / dz)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nx * ny * nz, nf))


def face_vector(fr):
    return np.concatenate([fr["Ax"].ravel(), fr["Ay"].ravel(), fr["Az"].ravel()])


def edge_vector(fr):
    return np.concatenate([fr["Lx"].ravel(), fr["Ly"].ravel(), fr["Lz"].ravel()])


class DMOperators:
    """All assembled matrices of one grid and geometry (full face/edge/cell
    index spaces; ``open`` selects the unknowns)."""

    def __init__(self, grid, fr):
        g = grid
        self.grid = g
        self.nx, self.ny, self.nz = g.nx, g.ny, g.nz
        self.h = (g.dx, g.dy, g.dz)
        self.fr = fr
        self.C = curl(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)
        self.D = divergence(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)
        self.a = face_vector(fr)
        self.l = edge_vector(fr)
        self.v = fr["V"].ravel().copy()
        with np.errstate(divide="ignore"):
            self.inv_v = np.where(self.v > 0, 1.0 / np.where(self.v > 0, self.v, 1.0), 0.0)
        self.open = self.a > 0
        self.open_idx = np.nonzero(self.open)[0]
        A = sp.diags(self.a)
        # curl-curl with edge fractions (Eq. discWaveBDM times A)
        self.CLCt = (self.C @ sp.diags(self.l) @ self.C.T).tocsr()
        # A-scaled Dey--Mittra grad-div (Eq. discLaplDM)
        self.GD = (A @ self.D.T @ sp.diags(self.inv_v) @ self.D @ A).tocsr()
        self.A = A.tocsr()

    # -- full-space operators -------------------------------------------------
    def K(self, sigma=0.0):
        """K - sigma A of Eq. discLaplDM on the full face space."""
        return (self.CLCt + self.GD - sigma * self.A).tocsr()

    def apply_K(self, x, sigma=0.0):
        return self.K(sigma) @ x

    def diag_K(self, sigma=0.0):
        return self.K(sigma).diagonal()

    # -- restriction to the open faces ---------------------------------------
    def restrict(self, M):
        o = self.open_idx
        return M.tocsr()[o][:, o].tocsc()

    def scalar_laplacian(self):
        """D A D^T on cells (the matrix inverted inside P_DM, Eq. proj)."""
        S = (self.D @ self.A @ self.D.T).tocsr()
        S.eliminate_zeros()
        return S

    def project(self, x):
        """P_DM x = x - D^T (D A D^T)^-1 D A x (Eq. proj) on the full face space.

        D A D^T is singular with one constant null vector per connected vacuum
        component enclosed by closed faces; D A x has zero sum on each such
        component, so pinning one cell of each gives an exact solution (the
        constant is irrelevant to D^T restricted to open faces).  A component
        that reaches an open face on the outer wall (a magnetic symmetry
        plane, see oracle.geometry) sees the zero potential beyond it and is
        regular: it is not pinned.  Closed faces of the result are 0."""
        S = self.scalar_laplacian()
        active = np.nonzero(self.v > 0)[0]
        Sa = S[active][:, active].tocsr()
        ncomp, labels = csgraph.connected_components(Sa, directed=False)
        grounded = self.grounded_cells()[active]
        keep = np.ones(active.size, dtype=bool)
        for c in range(ncomp):
            members = np.nonzero(labels == c)[0]
            if not grounded[members].any():
                keep[members[0]] = False
        s = (self.D @ (self.a * x))[active]
        psi_a = np.zeros(active.size)
        kk = np.nonzero(keep)[0]
        if kk.size:
            psi_a[kk] = spla.spsolve(Sa[kk][:, kk].tocsc(), s[kk])
        psi = np.zeros(self.v.size)
        psi[active] = psi_a
        y = x - self.D.T @ psi
        y[~self.open] = 0.0
        return y

    def grounded_cells(self):
        """Cells with an open face on the outer wall (a face of D with one cell)."""
        cells_per_face = np.asarray((self.D != 0).sum(axis=0)).ravel()
        wall_open = (cells_per_face == 1) & self.open
        return np.asarray(abs(self.D) @ wall_open.astype(float)).ravel() > 0

    def vacuum_components(self):
        S = self.scalar_laplacian()
        active = np.nonzero(self.v > 0)[0]
        ncomp, _ = csgraph.connected_components(S[active][:, active], directed=False)
        return ncomp
