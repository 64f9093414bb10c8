"""Oracle pins with closed forms: the discrete Yee box and the spherical cavity.

* Grid-aligned PEC box (every fraction 0 or 1): the Dey--Mittra operator is the
  vacuum Yee curl-curl C C^T of Eq. discWaveB on the interior faces.  Its
  nonzero eigenvalues are those of the discrete vector Laplacian (Eq. discLaplB)
  restricted to divergence-free fields:
      k^2 = (2/dx sin(pi p / 2 nx))^2 + (2/dy sin(pi q / 2 ny))^2 + (2/dz sin(pi r / 2 nz))^2
  for 0 <= p < nx, 0 <= q < ny, 0 <= r < nz with at most one index zero;
  multiplicity 2 when all three are nonzero (two polarisations), 1 when one is
  zero.  The divergent modes of K (Eq. discLaplB) carry the Neumann scalar
  Laplacian eigenvalues, the same formula with any indices, (p, q, r) != 0.
* Spherical PEC cavity of radius R (Sec. 6.2, ref. Jackson): TE_lm modes at the
  zeros of j_l(kR), TM_lm modes at the zeros of d/dx [x j_l(x)] at x = kR, each
  (2l + 1)-fold degenerate.  The Neumann (divergent, spurious) modes sit at the
  zeros of j_l'(x).
"""
from __future__ import annotations

import math

import numpy as np


def box_eigenvalues(nx, ny, nz, dx, dy, dz):
    """Sorted electromagnetic eigenvalues of the PEC box, with multiplicity."""
    sx = (2.0 / dx * np.sin(np.pi * np.arange(nx) / (2 * nx))) ** 2
    sy = (2.0 / dy * np.sin(np.pi * np.arange(ny) / (2 * ny))) ** 2
    sz = (2.0 / dz * np.sin(np.pi * np.arange(nz) / (2 * nz))) ** 2
    out = []
    for p in range(nx):
        for q in range(ny):
            for r in range(nz):
                zeros = (p == 0) + (q == 0) + (r == 0)
                if zeros >= 2:
                    continue
                mult = 2 if zeros == 0 else 1
                out += [sx[p] + sy[q] + sz[r]] * mult
    return np.sort(np.array(out))


def box_eigenvalues_magnetic_x(m, ny, nz, dx, dy, dz):
    """Sorted electromagnetic eigenvalues of the box of m cells along x whose
    x-low wall is a magnetic symmetry plane half a cell outside it (and whose
    other walls are conductors): the modes of the conductor box of 2m + 1
    cells that are even under x -> -x about its middle.  There B_x ~ sin(p pi
    x' / L) (x' from the conductor wall) is even exactly for odd p, so the
    spectrum is the box rule above restricted to odd p (p never zero)."""
    nx = 2 * m + 1
    sx = (2.0 / dx * np.sin(np.pi * np.arange(nx) / (2 * nx))) ** 2
    sy = (2.0 / dy * np.sin(np.pi * np.arange(ny) / (2 * ny))) ** 2
    sz = (2.0 / dz * np.sin(np.pi * np.arange(nz) / (2 * nz))) ** 2
    out = []
    for p in range(1, nx, 2):
        for q in range(ny):
            for r in range(nz):
                zeros = (q == 0) + (r == 0)
                if zeros >= 2:
                    continue
                out += [sx[p] + sy[q] + sz[r]] * (2 if zeros == 0 else 1)
    return np.sort(np.array(out))


def box_scalar_eigenvalues(nx, ny, nz, dx, dy, dz):
    """Nonzero Neumann eigenvalues of the cell Laplacian D D^T on the box."""
    sx = (2.0 / dx * np.sin(np.pi * np.arange(nx) / (2 * nx))) ** 2
    sy = (2.0 / dy * np.sin(np.pi * np.arange(ny) / (2 * ny))) ** 2
    sz = (2.0 / dz * np.sin(np.pi * np.arange(nz) / (2 * nz))) ** 2
    tot = (sx[None, None, :] + sy[None, :, None] + sz[:, None, None]).ravel()
    return np.sort(tot)[1:]


def box_mode_count(nx, ny, nz):
    a, b, c = nx - 1, ny - 1, nz - 1
    return 2 * a * b * c + a * b + b * c + c * a


# ---------------------------------------------------------------------------
# spherical Bessel functions (power series, Abramowitz & Stegun 10.1.2)
# ---------------------------------------------------------------------------

def sph_jn(l, x):
    """j_l(x) = x^l sum_m (-x^2/2)^m / (m! (2l + 2m + 1)!!), summed until the
    terms fall below 1e-18 of the running maximum (fine for x <~ 15)."""
    x = float(x)
    df = 1.0
    for t in range(1, 2 * l + 2, 2):
        df *= t
    term = x ** l / df
    s = term
    m = 0
    big = abs(term)
    while True:
        m += 1
        term *= -(x * x / 2.0) / (m * (2 * l + 2 * m + 1))
        s += term
        big = max(big, abs(term))
        if abs(term) < 1e-18 * big and m > 4:
            break
        if m > 400:
            break
    return s


def sph_jn_prime(l, x):
    """j_l'(x) = j_{l-1}(x) - (l+1)/x j_l(x)  (j_0' = -j_1)."""
    if l == 0:
        return -sph_jn(1, x)
    return sph_jn(l - 1, x) - (l + 1) / x * sph_jn(l, x)


def riccati_prime(l, x):
    """d/dx [x j_l(x)] = x j_{l-1}(x) - l j_l(x)  (l >= 1)."""
    return x * sph_jn(l - 1, x) - l * sph_jn(l, x)


def _roots(f, xmax, step=1e-3, xmin=1e-3):
    roots = []
    x0 = xmin
    f0 = f(x0)
    x = x0
    while x < xmax:
        x1 = x + step
        f1 = f(x1)
        if f0 == 0.0:
            roots.append(x)
        elif f0 * f1 < 0:
            a, b, fa = x, x1, f0
            for _ in range(100):
                m = 0.5 * (a + b)
                fm = f(m)
                if fa * fm <= 0:
                    b = m
                else:
                    a, fa = m, fm
            roots.append(0.5 * (a + b))
        x, f0 = x1, f1
    return roots


def sphere_modes(xmax=7.0, lmax=6):
    """Sorted list of (kR, kind, l, degeneracy) for TE and TM modes with kR < xmax."""
    out = []
    for l in range(1, lmax + 1):
        for r in _roots(lambda x: sph_jn(l, x), xmax, xmin=0.5):
            out.append((r, "TE", l, 2 * l + 1))
        for r in _roots(lambda x: riccati_prime(l, x), xmax, xmin=0.5):
            out.append((r, "TM", l, 2 * l + 1))
    out.sort()
    return out


def sphere_k2_list(radius=1.0, count=10, xmax=9.0):
    """The lowest ``count`` eigenvalues k^2 of the spherical cavity, with multiplicity."""
    vals = []
    for r, _, _, deg in sphere_modes(xmax=xmax):
        vals += [(r / radius) ** 2] * deg
    vals.sort()
    return np.array(vals[:count])


def sphere_neumann_modes(xmax=5.0, lmax=4):
    """(kR, l, degeneracy) of the Neumann scalar Laplacian: zeros of j_l'."""
    out = []
    for l in range(0, lmax + 1):
        for r in _roots(lambda x: sph_jn_prime(l, x), xmax, xmin=0.5):
            out.append((r, l, 2 * l + 1))
    out.sort()
    return out


def sphere_volume(radius=1.0):
    return 4.0 / 3.0 * math.pi * radius ** 3


# ---------------------------------------------------------------------------
# the octant's lowest mode: TM, l = 3, angular part x y z / r^3
# ---------------------------------------------------------------------------

def _xyz_harmonic_curl(pts):
    """(x cross grad) u for u = x y z / r^3 (a real l = 3 harmonic), at pts (N x 3)."""
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    r2 = x * x + y * y + z * z
    r3 = r2 * np.sqrt(r2)
    r5 = r3 * r2
    p = x * y * z
    g = np.stack([y * z / r3 - 3.0 * x * p / r5, x * z / r3 - 3.0 * y * p / r5, x * y / r3 - 3.0 * z * p / r5], axis=1)
    return np.cross(pts, g)


def tm_xyz_b(k, pts):
    """Magnetic field of the spherical cavity's TM mode of l = 3 with angular
    part x y z / r^3 (Jackson's TM modes: B = j_l(k r) (r cross grad) Y, E
    from Ampere's law), up to a constant factor: B = j_3(k r) (x cross grad) u."""
    pts = np.asarray(pts, dtype=float)
    r = np.linalg.norm(pts, axis=1)
    j3 = np.array([sph_jn(3, k * v) for v in r])
    return j3[:, None] * _xyz_harmonic_curl(pts)


def curl_numeric(f, pts, h=1e-4):
    """curl f at pts by fourth-order central differences of the vector field f."""
    pts = np.asarray(pts, dtype=float)
    J = np.zeros((pts.shape[0], 3, 3))   # J[:, i, j] = d f_i / d x_j
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        J[:, :, j] = (-f(pts + 2 * e) + 8 * f(pts + e) - 8 * f(pts - e) + f(pts - 2 * e)) / (12 * h)
    return np.stack([J[:, 2, 1] - J[:, 1, 2], J[:, 0, 2] - J[:, 2, 0], J[:, 1, 0] - J[:, 0, 1]], axis=1)


def tm_xyz_e(k, pts):
    """Electric field of the same mode, up to the same constant (and a factor
    i c): E = curl B / k."""
    return curl_numeric(lambda p: tm_xyz_b(k, p), pts) / k
