"""Symmetry-plane walls on the GPU path (Sec. 6.2-6.3) against the oracle:
magnetic planes half a cell outside the wall node plane, electric planes on it
(see dm_geometry_create_walls)."""
import numpy as np
import pytest

import workloads as W
from oracle import eigen, geometry, multigrid as MG, operators

pytestmark = pytest.mark.gpu

PMC_XLO = ("pmc", "pec", "pec", "pec", "pec", "pec")


def _half_sphere(m=8, n=16, h=0.14, sigma=12.0, nev=4):
    """Sphere of radius 1.05 cut by the magnetic plane x = 0: the grid holds
    x > 0 (first node plane at h/2), offset slightly in y and z."""
    g = W.Grid(m, n, n, h, h, h, (0.5 * h, -n * h / 2 + 0.013, -n * h / 2 - 0.029))
    phi = W.sphere_phi(g, (0.0, 0.0, 0.0), 1.05)
    return W.Workload(f"halfsphere{m}x{n}x{n}", g, phi, sigma, nev, -1, walls=PMC_XLO)


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


@pytest.fixture(scope="module")
def half(dm, ctx):
    w = _half_sphere()
    geom = dm.Geometry.from_workload(ctx, w)
    levels = MG.build_vector_hierarchy(w.grid, w.phi, w.sigma, walls=w.walls)
    op = dm.Operator(ctx, geom, w.sigma)
    return w, geom, levels, op


def test_fractions_with_magnetic_wall(half):
    w, geom, levels, op = half
    assert op.num_levels == len(levels)
    for l, lev in enumerate(levels):
        L, A, V = geom.fractions(l)
        assert _rel(L, operators.edge_vector(lev.fr)) < 1e-14, l
        assert _rel(A, operators.face_vector(lev.fr)) < 1e-14, l
        assert _rel(V, lev.fr["V"].ravel()) < 1e-14, l
        assert np.array_equal(A > 0, operators.face_vector(lev.fr) > 0), l
    # the magnetic wall's normal faces are open on the fine level
    assert (levels[0].fr["Ax"][..., 0] > 0).sum() > 10


def test_apply_with_magnetic_wall(half):
    w, geom, levels, op = half
    rng = np.random.default_rng(5)
    for l, lev in enumerate(levels):
        x = rng.standard_normal(lev.mask.size) * lev.mask
        assert _rel(op.apply(x, level=l), lev.K @ x) < 1e-13, l
    x = rng.standard_normal(levels[0].mask.size) * levels[0].mask
    assert _rel(op.apply_ff(x), levels[0].K @ x) < 1e-12


def test_projection_with_magnetic_wall(half):
    """The vacuum region reaches the magnetic wall, so D A D^T is regular
    there: the projection must match the oracle's unpinned solve."""
    w, geom, levels, op = half
    ops = levels[0].ops
    assert ops.grounded_cells().any()
    x = np.random.default_rng(6).standard_normal(ops.a.size) * ops.open
    y, it = op.project(x, tol=1e-13)
    ref = ops.project(x)
    assert _rel(y, ref) < 1e-9, _rel(y, ref)
    assert it < 100
    assert np.max(np.abs(ops.D @ (ops.a * y))) < 1e-9 * np.max(np.abs(ops.D @ (ops.a * x)))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-9)])
def test_eigensolve_with_magnetic_wall(dm, ctx, half, prec, tol):
    w, geom, levels, _ = half
    ops = levels[0].ops
    kref, Bref, _ = eigen.shift_invert_modes(ops, w.sigma, w.nev)
    k2, B, rep, st = dm.eigensolve(ctx, geom, w.sigma, w.nev, precision=prec)
    print(f"\nhalf sphere ({prec}): k2 {np.round(k2, 6)}, oracle {np.round(kref, 6)}; "
          f"outer {rep['outer_iters']}, inner {rep['inner_iters']}, proj {rep['proj_iters']}")
    assert st == 0, rep
    assert np.max(np.abs(k2 - kref) / kref) < tol, (k2, kref)
    for i in range(w.nev):
        c = eigen.certificate(ops, k2[i], B[i])
        assert c["rho"] < 1e-8 and c["delta"] < 1e-8, c


def test_quarter_nine_cell_with_two_magnetic_planes(dm, ctx):
    """The quarter 9-cell cavity of Sec. 6.3 (magnetic planes x = 0, y = 0) at
    a coarse resolution: the GPU eigenpairs against the oracle's, and the
    lowest mode is the accelerating TM010-like one (its field on the axis is
    longitudinal: B_z small against B_x, B_y)."""
    w = W.quarter_nine_cell_workload(nq=10, nz=120, nev=3)
    ops = operators.DMOperators(w.grid, geometry.fractions(w.phi, walls=w.walls))
    kref, Bref, _ = eigen.shift_invert_modes(ops, w.sigma, w.nev)
    geom = dm.Geometry.from_workload(ctx, w)
    k2, B, rep, st = dm.eigensolve(ctx, geom, w.sigma, w.nev, precision="f32")
    print(f"\nquarter 9-cell: k2 {k2}, oracle {kref}; outer {rep['outer_iters']}, inner {rep['inner_iters']}")
    assert st == 0, rep
    assert np.max(np.abs(k2 - kref) / kref) < 1e-9, (k2, kref)
    sh = operators.shapes(w.grid.nx, w.grid.ny, w.grid.nz)
    nfx, nfy = int(np.prod(sh["fx"])), int(np.prod(sh["fy"]))
    b = B[0]
    transverse = np.linalg.norm(b[:nfx + nfy])
    assert np.linalg.norm(b[nfx + nfy:]) < 0.05 * transverse
    # the accelerating passband of a 9-cell cavity: nine modes closely spaced;
    # its lowest member sits near (2 pi 1.3 GHz / c)^2 = 742 m^-2 for this shape
    f = np.sqrt(k2[0]) * 299792458.0 / (2 * np.pi)
    assert 1.0e9 < f < 1.6e9, f


def test_string_of_cavities_with_magnetic_planes(dm, ctx):
    """Two 9-cell cavities strung along z (the cryomodule of Sec. 6.3, here two
    cavities at a coarse resolution, one cell length of beam pipe between
    them): every mode of one cavity splits into a pair through the pipe
    (relative splitting 5e-7 here), and both members come out.  With longer
    pipes the splitting falls below the inner-solve tolerance (6e-10 at two
    cell lengths); a single-vector Krylov method then sees one eigenvalue of
    multiplicity two, and may return the next mode instead of the twin."""
    w = W.quarter_nine_cell_workload(nq=8, nz=200, nev=4, n_cavities=2, gap_cells=1)
    ops = operators.DMOperators(w.grid, geometry.fractions(w.phi, walls=w.walls))
    kref, _, _ = eigen.shift_invert_modes(ops, w.sigma, w.nev)
    geom = dm.Geometry.from_workload(ctx, w)
    k2, B, rep, st = dm.eigensolve(ctx, geom, w.sigma, w.nev, precision="f32")
    assert st == 0, rep
    assert np.max(np.abs(k2 - kref) / kref) < 1e-9, (k2, kref)
