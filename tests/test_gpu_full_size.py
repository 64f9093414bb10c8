"""Parity at full size: the 128^3 sphere and the 192^3 ellipsoid of the
headline configuration.

At these sizes (2.5 M and 5.6 M open faces) the oracle does not run its own eigensolve;
instead its assembled K and A re-certify every pair the GPU returns (the
residual of the original problem, the Dey--Mittra divergence and the Rayleigh
quotient, Sec. 5.1-5.2), and the eigenvalues are compared with the analytic
modes of the unit sphere (Sec. 6.2) within the discretisation error."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import analytic, eigen, geometry, operators

pytestmark = pytest.mark.gpu


def test_sphere128_bench_configuration_certified_by_oracle(dm, ctx):
    w = W.sphere_workload(128, radius=1.0, half_width=1.1, sigma=5.0, nev=10, offset_seed=W.SEED_BASE + 2)
    geom = dm.Geometry.from_workload(ctx, w)
    k2, B, rep, st = dm.eigensolve(ctx, geom, w.sigma, w.nev, vectors="host", precision="f32")
    geom.close()
    assert st == 0 and rep["n_converged"] == w.nev, rep
    ops = operators.DMOperators(w.grid, geometry.fractions(w.phi))
    for i in range(w.nev):
        c = eigen.certificate(ops, k2[i], B[i])
        assert c["rho"] < 1e-8 and c["delta"] < 1e-8, (i, c)
        assert abs(c["rq"] - k2[i]) / k2[i] < 1e-12, (i, c["rq"], k2[i])
    # closed faces hold zero; the pairs are A-orthonormal
    assert np.all(B[:, ~ops.open] == 0.0)
    G = (B * ops.a) @ B.T
    assert np.max(np.abs(G - np.eye(w.nev))) < 1e-8
    # TM_1 triplet, TM_2 quintuplet and two of the TE_1 triplet of the unit
    # sphere; the discretisation error at h = 2.2/128 is a few 1e-4
    ref = analytic.sphere_k2_list(1.0, w.nev)
    assert np.max(np.abs(k2 - ref) / ref) < 2e-3, (k2, ref)


def test_ellipsoid192_headline_configuration_certified_by_oracle(dm, ctx):
    """The headline configuration of bench.py (192^3 seeded ellipsoid, 16 modes
    nearest sigma = 5, FP32 V-cycle, library defaults): the oracle's assembled K
    and A re-certify every pair, and the eigenvalues agree with the oracle's own
    sparse eigensolve of the same ellipsoid at 48^3 within the discretisation
    error (second order: a few 1e-3 at 48^3), which pins which modes came out."""
    w = W.ellipsoid_workload(192)
    geom = dm.Geometry.from_workload(ctx, w)
    k2, B, rep, st = dm.eigensolve(ctx, geom, w.sigma, w.nev, vectors="host", precision="f32")
    geom.close()
    assert st == 0 and rep["n_converged"] == w.nev, rep
    ops = operators.DMOperators(w.grid, geometry.fractions(w.phi))
    for i in range(w.nev):
        c = eigen.certificate(ops, k2[i], B[i])
        assert c["rho"] < 1e-8 and c["delta"] < 1e-8, (i, c)
        assert abs(c["rq"] - k2[i]) / k2[i] < 1e-12, (i, c["rq"], k2[i])
    assert np.all(B[:, ~ops.open] == 0.0)
    G = (B * ops.a) @ B.T
    assert np.max(np.abs(G - np.eye(w.nev))) < 1e-8
    # the oracle's 48^3 modes of the same ellipsoid (tests/golden/make_ellipsoid48_modes.py)
    with open(os.path.join(os.path.dirname(__file__), "golden", "ellipsoid48_modes.json")) as f:
        ref = json.load(f)
    assert np.allclose(ref["semi_axes"], w.meta["semi_axes"], rtol=0, atol=1e-15)
    kc = np.asarray(ref["k2"])
    for v in k2:
        assert np.min(np.abs(kc - v)) / v < 5e-3, (v, kc)
