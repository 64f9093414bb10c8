"""Surface fields of the octant's lowest mode (Sec. 6.2, Eq. errorNorm), shared
by the oracle pin and the GPU test: the computed electric field interpolated
to a shell and compared with the analytic TM field."""
import numpy as np

from oracle import analytic, geometry, operators


def edge_field_at(e, g, pts):
    """Trilinear interpolation of an edge field (natural edge layout) to pts:
    e_x sits at (x_i + dx/2, y_j, z_k), e_y at (x_i, y_j + dy/2, z_k), e_z at
    (x_i, y_j, z_k + dz/2); half a cell beyond the outermost edges it
    extrapolates linearly."""
    from scipy.interpolate import RegularGridInterpolator
    nx, ny, nz = g.nx, g.ny, g.nz
    shapes = [(nz + 1, ny + 1, nx), (nz + 1, ny, nx + 1), (nz, ny + 1, nx + 1)]
    parts = np.split(e, np.cumsum([int(np.prod(s)) for s in shapes])[:-1])
    out = np.zeros((pts.shape[0], 3))
    for c in range(3):
        arr = parts[c].reshape(shapes[c])
        ax = [g.origin[0] + g.dx * (np.arange(shapes[c][2]) + (0.5 if c == 0 else 0.0)),
              g.origin[1] + g.dy * (np.arange(shapes[c][1]) + (0.5 if c == 1 else 0.0)),
              g.origin[2] + g.dz * (np.arange(shapes[c][0]) + (0.5 if c == 2 else 0.0))]
        f = RegularGridInterpolator((ax[2], ax[1], ax[0]), arr, method="linear", bounds_error=False, fill_value=None)
        out[:, c] = f(pts[:, ::-1])
    return out


def _points(seed=3):
    rng = np.random.default_rng(seed)
    dirs = np.abs(rng.standard_normal((400, 3)))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    dirs = dirs[np.min(dirs, axis=1) > 0.05]          # off the symmetry planes
    vol = np.abs(rng.standard_normal((2000, 3)))
    vol /= np.linalg.norm(vol, axis=1)[:, None]
    vol *= rng.uniform(0.1, 0.8, len(vol))[:, None] ** (1.0 / 3.0)
    return dirs, vol


def surface_field_error(w, a_min, b):
    """Eq. errorNorm for the octant's lowest mode (TM, l = 3): the electric
    field e = C^T b on the open edges (Ampere's law up to a constant; closed
    edges such as the walls' tangential ones carry none), trilinearly
    interpolated to a shell 3 dx inside the unit sphere, against the analytic
    field, after both are scaled to the same l2 norm over points filling the
    cavity (the sign by their correlation)."""
    k3 = [r for r, kind, l, _ in analytic.sphere_modes(xmax=6.0) if kind == "TM" and l == 3][0]
    g = w.grid
    dirs, vol = _points()
    ops = operators.DMOperators(g, geometry.fractions(w.phi, a_min=a_min))
    e = (ops.l > 0) * (ops.C.T @ b)
    shell = dirs * (1.0 - 3.0 * g.dx)
    Evol = analytic.tm_xyz_e(k3, vol)
    ev, es = edge_field_at(e, g, vol), edge_field_at(e, g, shell)
    alpha = np.linalg.norm(Evol) / np.linalg.norm(ev) * np.sign(np.sum(ev * Evol))
    Es = analytic.tm_xyz_e(k3, shell)
    return float(np.sqrt(np.sum((alpha * es - Es) ** 2) / np.sum(Es ** 2)))
