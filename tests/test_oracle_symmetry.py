"""Pins of the oracle's symmetry-plane walls (Sec. 6.2-6.3).

A magnetic (PMC) symmetry plane is read as the plane half a cell outside the
wall's node plane.  The half-domain problem with that wall must then have, as
its spectrum, exactly the modes of the mirrored full-domain problem that are
even under the mirror map (normal flux even, tangential flux odd), and an
electric (PEC) wall on a node plane exactly the odd ones.  These tests build
the full domain independently (ordinary closed walls, the geometry mirrored
entity by entity) and compare spectra, so that a wrong wall entity, a wrong
ghost value or a wrongly pinned potential in the half domain shows up.
"""
import numpy as np
import pytest

import workloads as W
from oracle import analytic, eigen, geometry, operators

PMC_XLO = ("pmc", "pec", "pec", "pec", "pec", "pec")


def _full_and_half_grids(m, ny, nz, h, y0, z0):
    """Full grid of 2m+1 cells across x centred on x = 0 (a cell centre) and
    the half grid of its m cells with x > h/2 (origin x = h/2)."""
    full = W.Grid(2 * m + 1, ny, nz, h, h, h, (-(m + 0.5) * h, y0, z0))
    half = W.Grid(m, ny, nz, h, h, h, (0.5 * h, y0, z0))
    return full, half


def _mirror_fractions(fr, m):
    """Full-domain fractions made exactly mirror-symmetric about x = 0: every
    entity with x < 0 takes the value of its image with x > 0.  Entities that
    are their own image (the centre cell column, its y/z-faces and x-edges)
    keep their values: they carry no field of either parity class."""
    out = {k: v.copy() for k, v in fr.items()}
    nx = 2 * m + 1
    # x-faces and y/z-edges sit on node planes i = 0 .. nx (image nx - i);
    # y/z-faces, x-edges and cells on cell planes i = 0 .. nx-1 (image nx-1-i)
    for key in ("Ax", "Ly", "Lz"):
        a = out[key]
        for i in range(m + 1):
            a[..., i] = a[..., nx - i]
    for key in ("Ay", "Az", "Lx", "V"):
        a = out[key]
        for i in range(m):
            a[..., i] = a[..., nx - 1 - i]
    return out


def _parity_counts(ops, m, k2, B, rel=1e-9):
    """For each distinct eigenvalue (within rel), how many A-orthonormal
    eigenvectors are even under the mirror map x -> -x with the magnetic
    parity (x-faces +1, y/z-faces -1): trace of the map on the eigenspace."""
    g = ops.grid
    sh = operators.shapes(g.nx, g.ny, g.nz)
    nfx, nfy = int(np.prod(sh["fx"])), int(np.prod(sh["fy"]))

    def mirror(b):
        bx = b[:nfx].reshape(sh["fx"])[..., ::-1]
        by = -b[nfx:nfx + nfy].reshape(sh["fy"])[..., ::-1]
        bz = -b[nfx + nfy:].reshape(sh["fz"])[..., ::-1]
        return np.concatenate([bx.ravel(), by.ravel(), bz.ravel()])

    out = []
    i = 0
    while i < k2.size:
        j = i
        while j + 1 < k2.size and abs(k2[j + 1] - k2[i]) <= rel * abs(k2[i]):
            j += 1
        Q = B[:, i:j + 1]
        tr = sum(float(Q[:, c] @ (ops.a * mirror(Q[:, c]))) for c in range(Q.shape[1]))
        dim = j - i + 1
        n_even = int(round((dim + tr) / 2))
        assert abs((dim + tr) / 2 - n_even) < 1e-6, (k2[i], dim, tr)
        out.append((float(k2[i]), n_even, dim - n_even))
        i = j + 1
    return out


def _even_spectrum(ops, m):
    k2, B = eigen.dense_modes(ops)
    out = []
    for lam, ne, _ in _parity_counts(ops, m, k2, B):
        out += [lam] * ne
    return np.array(sorted(out))


def test_pmc_half_box_is_the_even_part_of_the_full_box():
    m, ny, nz, h = 3, 4, 3, 0.25
    full, half = _full_and_half_grids(m, ny, nz, h, 0.0, 0.0)
    pad = 0.5 * h
    phi_f = W.box_phi(full, (-10, -pad, -pad), (10, ny * h + pad, nz * h + pad))
    phi_h = W.box_phi(half, (-10, -pad, -pad), (10, ny * h + pad, nz * h + pad))
    ops_f = operators.DMOperators(full, geometry.fractions(phi_f))
    ops_h = operators.DMOperators(half, geometry.fractions(phi_h, walls=PMC_XLO))
    even = _even_spectrum(ops_f, m)
    k2h, _ = eigen.dense_modes(ops_h)
    assert k2h.size == even.size, (k2h.size, even.size)
    assert np.max(np.abs(np.sort(k2h) - even) / even) < 1e-10
    # and it is a proper subset: the odd modes exist and are absent
    k2f, _ = eigen.dense_modes(ops_f)
    assert k2f.size > k2h.size


def test_pmc_half_box_matches_the_closed_form():
    """The half box's spectrum against the closed form of the Yee box restricted
    to the modes even under the mirror (oracle.analytic)."""
    m, ny, nz, h = 3, 4, 3, 0.25
    _, half = _full_and_half_grids(m, ny, nz, h, 0.0, 0.0)
    pad = 0.5 * h
    phi_h = W.box_phi(half, (-10, -pad, -pad), (10, ny * h + pad, nz * h + pad))
    ops_h = operators.DMOperators(half, geometry.fractions(phi_h, walls=PMC_XLO))
    k2h = np.sort(eigen.dense_modes(ops_h)[0])
    ref = analytic.box_eigenvalues_magnetic_x(m, ny, nz, h, h, h)
    assert k2h.size == ref.size, (k2h.size, ref.size)
    assert np.max(np.abs(k2h - ref) / ref) < 1e-10


def test_pmc_half_sphere_with_cut_cells_matches_the_mirrored_full_domain():
    m, n, h = 4, 8, 0.3
    full, half = _full_and_half_grids(m, n, n, h, -n * h / 2 + 0.037, -n * h / 2 - 0.021)
    R = 1.05
    phi_f = W.sphere_phi(full, (0.0, 0.0, 0.0), R)
    phi_h = np.ascontiguousarray(phi_f[..., m + 1:])     # the same node values (half-grid nodes)
    fr_f = _mirror_fractions(geometry.fractions(phi_f), m)
    fr_h = geometry.fractions(phi_h, walls=PMC_XLO)
    # the half domain's fractions are the full domain's on x > 0, wall entities included
    # (node-plane entities: full planes m+1 .. 2m+1; cell-plane ones: cells m+1 .. 2m)
    for key in ("Ax", "Ly", "Lz", "Ay", "Az", "Lx", "V"):
        np.testing.assert_array_equal(fr_h[key], fr_f[key][..., m + 1:])
    assert (fr_h["Ax"][..., 0] > 0).any() and (fr_h["Ly"][..., 0] > 0).any()
    ops_f = operators.DMOperators(full, fr_f)
    ops_h = operators.DMOperators(half, fr_h)
    even = _even_spectrum(ops_f, m)
    k2h = np.sort(eigen.dense_modes(ops_h)[0])
    assert k2h.size == even.size, (k2h.size, even.size)
    assert np.max(np.abs(k2h - even) / even) < 1e-9


def test_projection_with_a_magnetic_wall_is_exact():
    """A vacuum component that reaches the magnetic wall is regular (zero
    potential beyond the wall): P_DM must leave D A P x = 0 on every active
    cell and be idempotent, which a pinned cell in that component breaks."""
    m, n, h = 4, 8, 0.3
    _, half = _full_and_half_grids(m, n, n, h, -n * h / 2, -n * h / 2)
    fr = geometry.fractions(W.sphere_phi(half, (0.0, 0.0, 0.0), 1.05), walls=PMC_XLO)
    ops = operators.DMOperators(half, fr)
    assert ops.grounded_cells().any()
    x = np.random.default_rng(3).standard_normal(ops.a.size) * ops.open
    y = ops.project(x)
    div = ops.D @ (ops.a * y)
    assert np.max(np.abs(div)) < 1e-10 * np.max(np.abs(ops.D @ (ops.a * x)))
    np.testing.assert_allclose(ops.project(y), y, atol=1e-12 * np.max(np.abs(y)))


def test_pec_walls_are_unchanged_by_the_wall_option():
    w = W.sphere_workload(10, offset_seed=4)
    a = geometry.fractions(w.phi)
    b = geometry.fractions(w.phi, walls=("pec",) * 6)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    with pytest.raises(ValueError):
        geometry.fractions(w.phi, walls=("pec",) * 5)
