"""GPU eigensolver parity against the oracle and the closed forms."""
import numpy as np
import pytest

import workloads as W
from oracle import analytic, eigen, geometry, operators

pytestmark = pytest.mark.gpu


def _ops(w):
    return operators.DMOperators(w.grid, geometry.fractions(w.phi))


def test_box_closed_form(dm, ctx):
    w = W.box_workload()
    g = w.grid
    geom = dm.Geometry.from_workload(ctx, w)
    k2, B, rep, st = dm.eigensolve(ctx, geom, w.sigma, w.nev)
    ref = analytic.box_eigenvalues(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)
    want = np.sort(ref[eigen.wanted_order(ref, w.sigma)[:w.nev]])
    assert st == 0
    assert np.max(np.abs(k2 - want) / want) < 1e-10
    assert rep["rho_max"] < 1e-8 and rep["n_converged"] == w.nev


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-8), ("bf16", 1e-8)])
def test_sphere16_against_oracle(dm, ctx, prec, tol):
    w = W.sphere_workload(16, sigma=7.0, nev=4)
    ops = _ops(w)
    kref, Bref, _ = eigen.shift_invert_modes(ops, w.sigma, w.nev)
    geom = dm.Geometry.from_workload(ctx, w)
    k2, B, rep, st = dm.eigensolve(ctx, geom, w.sigma, w.nev, precision=prec)
    assert st == 0, rep
    assert np.max(np.abs(k2 - kref) / kref) < tol, (k2, kref)
    for i in range(w.nev):
        c = eigen.certificate(ops, k2[i], B[i])
        assert c["rho"] < 1e-8 and c["delta"] < 1e-8, c
        assert abs(c["rq"] - k2[i]) / k2[i] < 1e-12
    # degenerate TM_1 triplet: compare subspaces, not vectors
    assert eigen.subspace_angle_max(ops, B[:3].T, Bref[:, :3]) < 1e-6
    # eigenvectors are A-orthonormal
    G = (B * ops.a) @ B.T
    assert np.max(np.abs(G - np.eye(w.nev))) < 1e-9


def test_sphere_offset_10_modes(dm, ctx):
    w = W.sphere_workload(24, sigma=5.0, nev=10, offset_seed=W.SEED_BASE + 2)
    ops = _ops(w)
    kref, Bref, _ = eigen.shift_invert_modes(ops, w.sigma, w.nev)
    geom = dm.Geometry.from_workload(ctx, w)
    k2, B, rep, st = dm.eigensolve(ctx, geom, w.sigma, w.nev)
    assert st == 0, rep
    assert np.max(np.abs(k2 - kref) / kref) < 1e-10, (k2, kref)
    assert rep["rho_max"] < 1e-8


def test_certify_matches_oracle(dm, ctx):
    w = W.sphere_workload(16, sigma=7.0, nev=2)
    ops = _ops(w)
    kref, Bref, _ = eigen.shift_invert_modes(ops, w.sigma, 2)
    geom = dm.Geometry.from_workload(ctx, w)
    rho, delta, rq = dm.certify(ctx, geom, kref, Bref.T.copy())
    for i in range(2):
        c = eigen.certificate(ops, kref[i], Bref[:, i])
        assert abs(rho[i] - c["rho"]) < 1e-13 + 1e-6 * c["rho"]
        assert abs(rq[i] - c["rq"]) / c["rq"] < 1e-13


def test_device_vectors(dm, ctx):
    import torch
    w = W.box_workload(8, 6, 4, 0.8, 0.6, 0.4, sigma=20.0, nev=3)
    geom = dm.Geometry.from_workload(ctx, w)
    k2h, Bh, _, _ = dm.eigensolve(ctx, geom, w.sigma, w.nev, vectors="host")
    k2d, Bd, _, _ = dm.eigensolve(ctx, geom, w.sigma, w.nev, vectors="device")
    assert isinstance(Bd, torch.Tensor) and Bd.is_cuda
    assert np.allclose(k2h, k2d, rtol=1e-12)


def test_empty_geometry_is_an_error(dm, ctx):
    w = W.sphere_workload(8, radius=0.0)
    geom = dm.Geometry.from_workload(ctx, w, phi=np.abs(w.phi.ravel()) + 1.0)
    with pytest.raises(dm.DMError):
        dm.eigensolve(ctx, geom, 1.0, 2)


def test_invalid_arguments(dm, ctx):
    w = W.box_workload(4, 4, 4, 1, 1, 1)
    geom = dm.Geometry.from_workload(ctx, w)
    with pytest.raises(dm.DMError):
        dm.eigensolve(ctx, geom, 1.0, 0)
    with pytest.raises(dm.DMError):
        dm.Geometry(ctx, 1, 4, 4, 1, 1, 1, np.zeros(2 * 5 * 5))
