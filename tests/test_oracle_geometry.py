"""Pins of the oracle's cut-fraction geometry (Sec. 2, Sec. 5.1, Sec. 6.1)."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import analytic, geometry

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lattice_fraction(vals, dim, m):
    """Brute force: share of a barycentric lattice (m steps) where the linear
    interpolant is negative."""
    vals = np.asarray(vals, dtype=np.float64)
    cnt = tot = 0
    for c in itertools.product(range(m + 1), repeat=dim):
        if sum(c) > m:
            continue
        w = np.array(list(c) + [m - sum(c)], dtype=np.float64) / m
        tot += 1
        cnt += (w @ vals) < 0
    return cnt / tot


def _divided_difference(vals):
    """P(phi < 0) of a uniform point of a d-simplex with linear phi and distinct
    vertex values: sum_i (-phi_i)_+^d / prod_{j != i} (phi_j - phi_i)."""
    d = len(vals) - 1
    s = 0.0
    for i, p in enumerate(vals):
        if p < 0:
            s += (-p) ** d / np.prod([vals[j] - p for j in range(len(vals)) if j != i])
    return s


def test_simplex_fractions_vs_divided_difference():
    rng = np.random.default_rng(1)
    for _ in range(300):
        v = rng.standard_normal(4)
        assert abs(geometry.tet_fraction(*v) - _divided_difference(v)) < 1e-10
        assert abs(geometry.triangle_fraction(*v[:3]) - _divided_difference(v[:3])) < 1e-10
        assert abs(geometry.segment_fraction(*v[:2]) - _divided_difference(v[:2])) < 1e-12


def test_simplex_fractions_vs_lattice_sampling():
    rng = np.random.default_rng(2)
    for _ in range(6):
        v = rng.standard_normal(4)
        assert abs(geometry.tet_fraction(*v) - _lattice_fraction(v, 3, 40)) < 0.04
        assert abs(geometry.triangle_fraction(*v[:3]) - _lattice_fraction(v[:3], 2, 200)) < 0.01


def test_complement_and_degenerate_values():
    rng = np.random.default_rng(3)
    v = rng.standard_normal((4, 1000))
    assert np.allclose(geometry.tet_fraction(*v) + geometry.tet_fraction(*(-v)), 1.0, atol=1e-12)
    assert np.allclose(geometry.triangle_fraction(*v[:3]) + geometry.triangle_fraction(*(-v[:3])), 1.0, atol=1e-12)
    # equal values (the divided-difference form breaks down; the oracle must not)
    assert geometry.tet_fraction(-1.0, -1.0, 1.0, 1.0) == pytest.approx(0.5, abs=1e-15)
    assert geometry.tet_fraction(-1.0, -1.0, -1.0, -1.0) == 1.0
    assert geometry.tet_fraction(0.0, 0.0, 0.0, 0.0) == 0.0      # phi = 0 is conductor
    assert geometry.triangle_fraction(-1.0, 0.0, 0.0) == pytest.approx(1.0)


def test_halfspace_cut_exact():
    """phi = x - c is linear, so the piecewise-linear surface is the exact plane."""
    g = W.Grid(6, 5, 4, 0.5, 0.4, 0.3)
    c = 1.37
    X, Y, Z = W.node_coords(g)
    fr = geometry.fractions(X - c)
    # cell fraction = (c - x_i)/dx clipped
    xi = np.arange(g.nx) * g.dx
    vexp = np.clip((c - xi) / g.dx, 0.0, 1.0)
    assert np.allclose(fr["V"], vexp[None, None, :], atol=1e-14)
    # y-faces in the interior (not on walls) carry the same fraction
    assert np.allclose(fr["Ay"][:, 1:-1, :], vexp[None, None, :], atol=1e-14)
    # x-faces: open iff x_i < c, except the wall faces
    axp = (np.arange(g.nx + 1) * g.dx < c).astype(float)
    axp[0] = axp[-1] = 0.0
    assert np.array_equal(fr["Ax"], np.broadcast_to(axp, fr["Ax"].shape))


def test_corner_cut_exact():
    """phi = x + y + z - c on the unit cube: the vacuum is the corner simplex of
    volume c^3/6 (c <= 1), exact because phi is linear."""
    g = W.Grid(1, 1, 1, 1.0, 1.0, 1.0)
    X, Y, Z = W.node_coords(g)
    for c in (0.3, 0.7, 1.0):
        fr = geometry.fractions(X + Y + Z - c)
        assert fr["V"][0, 0, 0] == pytest.approx(c ** 3 / 6, abs=1e-14)
    # lower x-face of the cube (inside, if not a wall): triangle area c^2/2
    g = W.Grid(3, 3, 3, 1.0, 1.0, 1.0, (-1.0, -1.0, -1.0))
    X, Y, Z = W.node_coords(g)
    fr = geometry.fractions(X + Y + Z - 0.6)
    assert fr["Ax"][1, 1, 1] == pytest.approx(0.6 ** 2 / 2, abs=1e-14)
    assert fr["Lx"][1, 1, 1] == pytest.approx(0.6, abs=1e-14)


def test_box_fractions_binary():
    w = W.box_workload()
    fr = geometry.fractions(w.phi)
    for k, v in fr.items():
        assert set(np.unique(v)).issubset({0.0, 1.0}), k
    assert fr["V"].min() == 1.0


def test_sphere_volume_second_order():
    errs = []
    for n in (16, 32, 64):
        w = W.sphere_workload(n, offset_seed=W.SEED_BASE + 2)
        fr = geometry.fractions(w.phi)
        vol = fr["V"].sum() * w.grid.dx ** 3
        errs.append(abs(vol - analytic.sphere_volume()))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_sphere_divergence_theorem_of_a_constant_field():
    """Sum over a cut cell of the outward face fluxes of a constant field equals
    minus the flux through the cut surface; summed over every cell the interior
    faces cancel and the closed walls carry nothing, so the total is 0."""
    w = W.sphere_workload(16, offset_seed=W.SEED_BASE + 2)
    fr = geometry.fractions(w.phi)
    tot = (fr["Ax"][:, :, 1:] - fr["Ax"][:, :, :-1]).sum()
    assert abs(tot) < 1e-12


def test_paper_component_counts():
    """Tab. invPerf: magnetic components of a sphere of radius 0.49 L centred in a
    cube of side L, no faces neglected.  The open-face count (a > 0) equals the
    table's draft row exactly (kept commented out in the paper's source); the
    published row uses an unstated convention and agrees to ~8%."""
    ref = json.load(open(os.path.join(GOLDEN, "paper_tab_invperf.json")))
    for n, draft, pub in zip(ref["grid"], ref["draft_sphere_component_count"], ref["sphere_component_count"]):
        w = W.sphere_workload(n, radius=0.49, half_width=0.5)
        fr = geometry.fractions(w.phi)
        got = sum(int((fr[k] > 0).sum()) for k in ("Ax", "Ay", "Az"))
        assert got == draft, (n, got, draft)
        assert abs(got - pub) / pub < 0.08


def test_paper_cube_component_counts():
    """Draft row of Tab. invPerf for the PEC cube: 3 (N - 1) N^2 interior faces."""
    ref = json.load(open(os.path.join(GOLDEN, "paper_tab_invperf.json")))
    for n, draft in zip(ref["grid"][:2], ref["draft_cube_component_count"][:2]):
        w = W.box_workload(n, n, n, 1.0, 1.0, 1.0)
        fr = geometry.fractions(w.phi)
        assert sum(int((fr[k] > 0).sum()) for k in ("Ax", "Ay", "Az")) == draft


def test_smallest_area_fraction_scale():
    """Sec. 6.1: smallest area fraction on the sphere was 6e-4: tiny fractions occur."""
    w = W.sphere_workload(32, radius=0.49, half_width=0.5)
    fr = geometry.fractions(w.phi)
    a = np.concatenate([fr[k].ravel() for k in ("Ax", "Ay", "Az")])
    assert 0 < a[a > 0].min() < 1e-2
