"""Batched eigensolves over worker streams and the stencil tile-shape autotuner."""
import numpy as np
import pytest

import workloads as W
from oracle import eigen, geometry, operators

pytestmark = pytest.mark.gpu


def _cavities():
    return [W.sphere_workload(16, offset_seed=11, sigma=7.0, nev=4),
            W.ellipsoid_workload(20, seed=21, sigma=6.0, nev=3),
            W.sphere_workload(24, offset_seed=12, sigma=9.0, nev=5),
            W.box_workload(12, 10, 8, 1.0, 0.8, 0.6, sigma=30.0, nev=4)]


def test_batched_matches_single_solves(dm, ctx):
    ws = _cavities()
    geoms = [dm.Geometry.from_workload(ctx, w) for w in ws]
    jobs = []
    for w, g in zip(ws, geoms):
        jobs.append({"geom": g, "sigma": w.sigma, "nev": w.nev, "precision": "f32"})
    jobs.append({"geom": geoms[0], "sigma": 14.0, "nev": 3, "precision": "f32"})   # second shift, same cavity
    out = dm.eigensolve_batched(ctx, jobs, streams=3)
    for job, (k2, rep, st) in zip(jobs, out):
        assert st == 0, rep
        ref, _, _, st1 = dm.eigensolve(ctx, job["geom"], job["sigma"], job["nev"], vectors=None, precision="f32")
        assert st1 == 0
        assert np.max(np.abs(k2 - ref) / np.abs(ref)) < 1e-12
        assert rep["rho_max"] < 1e-8


def test_batched_item_against_oracle(dm, ctx):
    w = W.ellipsoid_workload(20, seed=21, sigma=6.0, nev=3)
    ops = operators.DMOperators(w.grid, geometry.fractions(w.phi))
    kref, _, _ = eigen.shift_invert_modes(ops, w.sigma, w.nev)
    g = dm.Geometry.from_workload(ctx, w)
    (k2, rep, st), = dm.eigensolve_batched(ctx, [{"geom": g, "sigma": w.sigma, "nev": w.nev, "precision": "f32"}])
    assert st == 0
    assert np.max(np.abs(k2 - kref) / kref) < 1e-8


def test_autotuned_shape_does_not_change_results(dm, ctx):
    w = W.sphere_workload(32, offset_seed=5, sigma=5.0)
    g = dm.Geometry.from_workload(ctx, w)
    tuned = dm.Operator(ctx, g, w.sigma, precision="f32", autotune=1)
    plain = dm.Operator(ctx, g, w.sigma, precision="f32", autotune=0)
    for l in range(tuned.num_levels - 1):
        assert tuned.stencil_shape(l) in range(6)
        assert plain.stencil_shape(l) == 0
    _, A, _ = g.fractions(0)
    x = np.random.default_rng(0).standard_normal(A.size) * (A > 0)
    for l in range(tuned.num_levels - 1):
        tuned.set_omega(l, plain.omega(l))
    # the one-node-per-thread and the z-marching kernels evaluate the same
    # expressions; only the compiler's FMA contraction may differ between them
    ya, yb = tuned.apply(x), plain.apply(x)
    assert np.max(np.abs(ya - yb)) <= 1e-13 * np.max(np.abs(yb))
    va, vb = tuned.vcycle(x), plain.vcycle(x)
    assert np.max(np.abs(va - vb)) <= 1e-5 * np.max(np.abs(vb))


@pytest.mark.parametrize("shape", range(6))
def test_every_stencil_shape_matches_oracle(dm, ctx, shape):
    """Each tile shape of the vector stencil, forced on every level, applies
    K - sigma A (Eq. discLaplDM) like the oracle's assembled matrix."""
    from oracle import geometry, operators
    w = W.ellipsoid_workload(40, seed=1307, sigma=5.0)
    g = dm.Geometry.from_workload(ctx, w)
    op = dm.Operator(ctx, g, w.sigma, precision="f64", autotune=0, force_shape=shape)
    assert op.stencil_shape(0) == shape
    ops = operators.DMOperators(w.grid, geometry.fractions(w.phi))
    x = np.random.default_rng(shape).standard_normal(ops.a.size) * (ops.a > 0)
    y = op.apply(x)
    yr = ops.apply_K(x, w.sigma)
    assert np.max(np.abs(y - yr)) <= 1e-12 * np.max(np.abs(yr))


@pytest.mark.parametrize("shape", range(6))
def test_every_stencil_shape_vcycle_two_and_three_sweeps(dm, ctx, shape):
    """Each tile shape forced on every level, with two and three damped Jacobi
    sweeps per smoothing step: the pre-smoothing's first two sweeps run as one
    stencil launch that forms the first iterate omega D^-1 f where it loads x.
    The V-cycle must equal the oracle's, which takes the sweeps one by one."""
    from oracle import multigrid as MG
    w = W.ellipsoid_workload(40, seed=1307, sigma=5.0)
    g = dm.Geometry.from_workload(ctx, w)
    levels = MG.build_vector_hierarchy(w.grid, w.phi, w.sigma)
    f = np.random.default_rng(40 + shape).standard_normal(levels[0].mask.size) * levels[0].mask
    for nu in (2, 3):
        op = dm.Operator(ctx, g, w.sigma, precision="f64", autotune=0, force_shape=shape, jacobi_sweeps=nu)
        assert op.stencil_shape(0) == shape
        om = [op.omega(l) for l in range(len(levels))]
        got = op.vcycle(f)
        ref = MG.vcycle(levels, f, om, band_sweeps=24, brick=8, band_sweeps_coarse=16, jacobi_sweeps=nu)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-9, (nu, shape)
