"""GPU parity of geometry, operator, smoother, transfers and V-cycles against
the oracle (element by element, FP64 unless stated)."""
import numpy as np
import pytest

import workloads as W
from oracle import geometry, multigrid as MG, operators

pytestmark = pytest.mark.gpu

CASES = {
    "sphere16": lambda: W.sphere_workload(16, offset_seed=W.SEED_BASE + 1, sigma=7.0),
    "sphere32": lambda: W.sphere_workload(32, offset_seed=W.SEED_BASE + 2, sigma=5.0),
    "ellipsoid24": lambda: W.ellipsoid_workload(24, seed=W.SEED_BASE + 3, sigma=5.0),
    "box12x10x8": lambda: W.box_workload(),
    "ragged13x11x9": lambda: W.sphere_workload(13, offset_seed=5, sigma=6.0),
    "slab40x8x12": lambda: W.Workload("slab", W.Grid(40, 8, 12, 0.05, 0.11, 0.09, (-1.0, -0.44, -0.54)),
                                      W.ellipsoid_phi(W.Grid(40, 8, 12, 0.05, 0.11, 0.09, (-1.0, -0.44, -0.54)),
                                                      (0.013, 0.02, -0.01), (0.93, 0.41, 0.5)), 5.0, 4, 0),
}


SWEEPS, COARSE_SWEEPS, BRICK = 24, 16, 8    # band smoother defaults of the library (fine, coarser levels, brick)
JACOBI = 2                                  # damped Jacobi sweeps per smoothing step (library default)


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, dm, ctx):
    w = CASES[request.param]()
    geom = dm.Geometry.from_workload(ctx, w)
    levels = MG.build_vector_hierarchy(w.grid, w.phi, w.sigma)
    op = dm.Operator(ctx, geom, w.sigma)
    return w, geom, levels, op


def test_level_count(case):
    w, geom, levels, op = case
    assert geom.num_levels >= op.num_levels == len(levels)


def test_fractions_all_levels(case):
    w, geom, levels, op = case
    for l, lev in enumerate(levels):
        L, A, V = geom.fractions(l)
        fr = lev.fr
        assert _rel(L, operators.edge_vector(fr)) < 1e-14
        assert _rel(A, operators.face_vector(fr)) < 1e-14
        assert _rel(V, fr["V"].ravel()) < 1e-14
        # open/closed decisions and cut-cell flags are exact
        assert np.array_equal(A > 0, operators.face_vector(fr) > 0)
        assert np.array_equal((V > 0) & (V < 1), (fr["V"].ravel() > 0) & (fr["V"].ravel() < 1))


def test_apply_all_levels(case):
    w, geom, levels, op = case
    rng = np.random.default_rng(3)
    for l, lev in enumerate(levels):
        x = rng.standard_normal(lev.mask.size) * lev.mask
        y = op.apply(x, level=l)
        assert _rel(y, lev.K @ x) < 1e-13, l


def test_apply_device_pointers(case):
    import torch
    w, geom, levels, op = case
    lev = levels[0]
    x = np.random.default_rng(4).standard_normal(lev.mask.size) * lev.mask
    y = op.apply(torch.from_numpy(x).cuda())
    assert y.is_cuda
    assert _rel(y.cpu().numpy(), lev.K @ x) < 1e-13


def test_apply_float_float(case):
    """The float-float product of the shifted solves' iterations against the
    oracle's FP64 matrix: about 48 significant bits per operation, and the
    result cancels against terms up to (k h)^-2 times its size on smooth
    fields, so 1e-12 (random) and 1e-11 (smooth) of the largest entry."""
    w, geom, levels, op = case
    lev = levels[0]
    rng = np.random.default_rng(7)
    x = rng.standard_normal(lev.mask.size) * lev.mask
    assert _rel(op.apply_ff(x), lev.K @ x) < 1e-12
    xs = np.cos(np.arange(lev.mask.size) * 1e-3) * lev.mask
    assert _rel(op.apply_ff(xs), lev.K @ xs) < 1e-11
    y = op.apply_ff(x)
    assert np.all(y[lev.mask == 0] == 0.0)


def test_projection_with_float_float_scalar_iterations(dm, ctx, case):
    """P_DM with the float-float scalar apply inside its FGMRES matches the
    FP64 apply's result and the oracle's projection."""
    w, geom, levels, op = case
    ops = levels[0].ops
    x = np.random.default_rng(9).standard_normal(ops.a.size) * ops.open
    y1, it1 = op.project(x, tol=1e-12)
    op0 = dm.Operator(ctx, geom, w.sigma, krylov_ff=0)
    y0, it0 = op0.project(x, tol=1e-12)
    op0.close()
    assert abs(it1 - it0) <= 2, (it0, it1)
    ref = ops.project(x)
    e1 = np.linalg.norm(y1 - ref) / np.linalg.norm(ref)
    e0 = np.linalg.norm(y0 - ref) / np.linalg.norm(ref)
    # the projection's own bar (test_project_matches_oracle), and no worse than the FP64 iterations
    assert e1 < 1e-9 and e1 < max(2.0 * e0, 1e-11), (e1, e0)
    assert np.linalg.norm(y1 - y0) / np.linalg.norm(y0) < 1e-9


def test_krylov_float_float_solve_matches_f64(dm, ctx, case):
    """The shifted solve with float-float iterations reaches the same FP64
    residual, and the same solution, as with FP64 iterations."""
    w, geom, levels, op = case
    lev = levels[0]
    b = np.random.default_rng(8).standard_normal(lev.mask.size) * lev.mask
    x1, it1, rr1 = op.solve(b, tol=1e-10)
    op0 = dm.Operator(ctx, geom, w.sigma, krylov_ff=0)
    x0, it0, rr0 = op0.solve(b, tol=1e-10)
    op0.close()
    assert rr1 < 1e-9 and rr0 < 1e-9
    assert abs(it1 - it0) <= 1, (it0, it1)
    assert np.linalg.norm(x1 - x0) / np.linalg.norm(x0) < 1e-8
    with pytest.raises(Exception):
        op_no = dm.Operator(ctx, geom, w.sigma, krylov_ff=0)
        try:
            op_no.apply_ff(b)
        finally:
            op_no.close()


def test_diagonal(case):
    w, geom, levels, op = case
    for l, lev in enumerate(levels):
        assert _rel(op.diagonal(l), lev.K.diagonal() * lev.mask) < 1e-13


def test_smooth_restrict_prolong(case):
    w, geom, levels, op = case
    rng = np.random.default_rng(5)
    for l in range(len(levels) - 1):
        lev = levels[l]
        om = op.omega(l)
        assert 0.3 < om < 1.5
        f = rng.standard_normal(lev.mask.size) * lev.mask
        x = rng.standard_normal(lev.mask.size) * lev.mask
        got = op.smooth(f, x, level=l)
        ref = MG.smooth(lev, f, x, om, SWEEPS if l == 0 else COARSE_SWEEPS, brick=BRICK, jacobi_sweeps=JACOBI)
        assert _rel(got, ref) < 1e-12, l
        r = rng.standard_normal(lev.mask.size) * lev.mask
        assert _rel(op.restrict(r, level=l), MG.restrict(levels, l, r)) < 1e-13, l
        ec = rng.standard_normal(levels[l + 1].mask.size) * levels[l + 1].mask
        assert _rel(op.prolong(ec, x, level=l), MG.prolong_add(levels, l, x, ec)) < 1e-13, l


@pytest.mark.parametrize("case_name,brick,sweeps", [("sphere16", 2, 5), ("sphere16", 4, 16), ("sphere32", 10, 9),
                                                   ("ragged13x11x9", 16, 7)])
def test_band_smoother_bricks(case_name, brick, sweeps, dm, ctx):
    """Other brick sizes and sweep counts; a 16-node brick covers the 13x11x9
    grid (one subdomain: plain band-restricted Jacobi)."""
    w = CASES[case_name]()
    geom = dm.Geometry.from_workload(ctx, w)
    op = dm.Operator(ctx, geom, w.sigma, band_brick=brick, band_sweeps=sweeps, band_sweeps_coarse=sweeps)
    levels = MG.build_vector_hierarchy(w.grid, w.phi, w.sigma)
    rng = np.random.default_rng(11)
    for l in range(len(levels) - 1):
        lev = levels[l]
        f = rng.standard_normal(lev.mask.size) * lev.mask
        x = rng.standard_normal(lev.mask.size) * lev.mask
        got = op.smooth(f, x, level=l)
        ref = MG.smooth(lev, f, x, op.omega(l), sweeps, brick=brick, jacobi_sweeps=JACOBI)
        assert _rel(got, ref) < 1e-12, (l, _rel(got, ref))


def test_band_brick_too_large_is_rejected(dm, ctx):
    """A subdomain whose local box does not fit in shared memory is an argument error."""
    w = CASES["sphere32"]()
    geom = dm.Geometry.from_workload(ctx, w)
    with pytest.raises(dm.DMError) as err:
        dm.Operator(ctx, geom, w.sigma, band_brick=64)
    assert "brick too large" in str(err.value)


def test_vcycle_fp64(case):
    w, geom, levels, op = case
    om = [op.omega(l) for l in range(len(levels))]
    f = np.random.default_rng(6).standard_normal(levels[0].mask.size) * levels[0].mask
    got = op.vcycle(f)
    ref = MG.vcycle(levels, f, om, band_sweeps=SWEEPS, brick=BRICK, band_sweeps_coarse=COARSE_SWEEPS,
                    jacobi_sweeps=JACOBI)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-9


@pytest.mark.parametrize("nu", [1, 2, 3])
def test_vcycle_and_smoother_jacobi_sweeps(nu, dm, ctx):
    """nu damped Jacobi sweeps per smoothing step (the buffers swap roles at
    every sweep, so odd and even counts take different paths)."""
    w = CASES["sphere16"]()
    geom = dm.Geometry.from_workload(ctx, w)
    op = dm.Operator(ctx, geom, w.sigma, jacobi_sweeps=nu)
    levels = MG.build_vector_hierarchy(w.grid, w.phi, w.sigma)
    om = [op.omega(l) for l in range(len(levels))]
    rng = np.random.default_rng(12)
    f = rng.standard_normal(levels[0].mask.size) * levels[0].mask
    got = op.vcycle(f)
    ref = MG.vcycle(levels, f, om, band_sweeps=SWEEPS, brick=BRICK, band_sweeps_coarse=COARSE_SWEEPS,
                    jacobi_sweeps=nu)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-9
    x = rng.standard_normal(levels[0].mask.size) * levels[0].mask
    got = op.smooth(f, x, level=0)
    ref = MG.smooth(levels[0], f, x, om[0], SWEEPS, brick=BRICK, jacobi_sweeps=nu)
    assert _rel(got, ref) < 1e-12


def test_scalar_vcycle_fp64(case, dm, ctx):
    w, geom, levels, op = case
    sl = MG.build_scalar_hierarchy(w.grid, w.phi)
    om = [op.omega(l, scalar=True) for l in range(len(sl))]
    f = np.random.default_rng(7).standard_normal(sl[0].mask.size) * sl[0].mask
    got = op.scalar_vcycle(f)
    ref = MG.scalar_vcycle(sl, f, om)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-9


@pytest.mark.parametrize("prec,tol", [("f32", 2e-5), ("bf16", 6e-2)])
def test_vcycle_low_precision(prec, tol, dm, ctx):
    w = CASES["sphere16"]()
    geom = dm.Geometry.from_workload(ctx, w)
    op = dm.Operator(ctx, geom, w.sigma, precision=prec)
    levels = MG.build_vector_hierarchy(w.grid, w.phi, w.sigma)
    om = [op.omega(l) for l in range(len(levels))]
    f = np.random.default_rng(8).standard_normal(levels[0].mask.size) * levels[0].mask
    got = op.vcycle(f)
    ref = MG.vcycle(levels, f, om, band_sweeps=SWEEPS, brick=BRICK, band_sweeps_coarse=COARSE_SWEEPS,
                    jacobi_sweeps=JACOBI)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol


def test_solve_matches_direct(case):
    import scipy.sparse.linalg as spla
    w, geom, levels, op = case
    lev = levels[0]
    b = np.random.default_rng(9).standard_normal(lev.mask.size) * lev.mask
    x, it, rr = op.solve(b, tol=1e-10)
    res = np.linalg.norm(b - lev.K @ x) / np.linalg.norm(b)
    assert res < 1e-9 and it <= 60, (res, it, rr)
    o = lev.ops.open_idx
    xd = np.zeros_like(b)
    xd[o] = spla.spsolve(lev.ops.restrict(lev.K), b[o])
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-6


def test_project_matches_oracle(case):
    w, geom, levels, op = case
    lev = levels[0]
    x = np.random.default_rng(10).standard_normal(lev.mask.size) * lev.mask
    y, it = op.project(x, tol=1e-12)
    ref = lev.ops.project(x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-9, it
    assert np.linalg.norm(lev.ops.D @ (lev.ops.a * y)) < 1e-10 * np.linalg.norm(lev.ops.D @ (lev.ops.a * x))
