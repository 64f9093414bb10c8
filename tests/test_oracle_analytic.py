"""Pins of the closed forms the oracle is checked against."""
import json
import math
import os

import numpy as np
import pytest

from oracle import analytic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_spherical_bessel_series_matches_library():
    sp = pytest.importorskip("scipy.special")
    for l in range(6):
        for x in np.linspace(0.3, 11.0, 37):
            assert abs(analytic.sph_jn(l, x) - sp.spherical_jn(l, x)) < 1e-11
            assert abs(analytic.sph_jn_prime(l, x) - sp.spherical_jn(l, x, derivative=True)) < 1e-11


def test_j0_closed_form():
    for x in (0.5, 2.0, 7.3):
        assert analytic.sph_jn(0, x) == pytest.approx(math.sin(x) / x, abs=1e-14)


def test_sphere_roots_golden():
    ref = json.load(open(os.path.join(GOLDEN, "sphere_roots.json")))
    modes = analytic.sphere_modes(xmax=7.0)
    tm1 = min(r for r, kind, l, _ in modes if kind == "TM" and l == 1)
    te1 = min(r for r, kind, l, _ in modes if kind == "TE" and l == 1)
    assert abs(tm1 - ref["TM1_first"]) < ref["tolerance"]
    assert abs(te1 - ref["TE1_first"]) < ref["tolerance"]
    # TE_1 zero is the root of tan x = x
    assert math.tan(te1) == pytest.approx(te1, rel=1e-9)
    j0 = analytic._roots(lambda x: analytic.sph_jn(0, x), 10.0, xmin=0.5)
    assert np.allclose(np.array(j0) / math.pi, ref["j0_zeros_over_pi"], atol=1e-10)


def test_sphere_lowest_eigenvalues_and_degeneracy():
    k2 = analytic.sphere_k2_list(1.0, 10)
    assert np.allclose(k2[:3], 2.743707269992269 ** 2, rtol=1e-12)
    assert np.allclose(k2[3:8], k2[3])       # TM_2 quintuplet
    assert k2[8] == pytest.approx(analytic.sphere_modes()[2][0] ** 2)


def test_box_mode_count_formula():
    for dims in ((4, 3, 3), (12, 10, 8), (5, 5, 2)):
        ev = analytic.box_eigenvalues(*dims, 0.1, 0.2, 0.3)
        assert ev.size == analytic.box_mode_count(*dims)


def _octant_points(rng, n, rmin, rmax):
    d = np.abs(rng.standard_normal((n, 3)))
    d /= np.linalg.norm(d, axis=1)[:, None]
    return d * rng.uniform(rmin, rmax, n)[:, None]


def test_octant_tm_mode_field_is_a_pec_cavity_mode():
    """The analytic field used for Eq. errorNorm's surface-field error: the TM
    mode of l = 3 with angular part x y z / r^3 at its TM root kR = 4.973420
    is divergence-free, solves curl curl B = k^2 B, has no tangential E on the
    sphere (perfect conductor) and none on the planes x, y, z = 0 (the octant's
    perfectly conducting symmetry planes), where B is tangential."""
    k = [r for r, kind, l, _ in analytic.sphere_modes(xmax=6.0) if kind == "TM" and l == 3][0]
    rng = np.random.default_rng(0)
    pts = _octant_points(rng, 40, 0.2, 0.9)
    B = analytic.tm_xyz_b(k, pts)
    E = analytic.tm_xyz_e(k, pts)
    scale = np.max(np.linalg.norm(B, axis=1))
    # div B = 0
    h = 1e-4
    div = sum((analytic.tm_xyz_b(k, pts + h * np.eye(3)[j])[:, j] - analytic.tm_xyz_b(k, pts - h * np.eye(3)[j])[:, j])
              / (2 * h) for j in range(3))
    assert np.max(np.abs(div)) < 1e-6 * scale * k
    # curl E = k B  (curl curl B = k^2 B for a divergence-free B)
    cE = analytic.curl_numeric(lambda p: analytic.tm_xyz_e(k, p), pts, h=1e-3)
    assert np.max(np.abs(cE - k * B)) < 1e-5 * k * scale
    # no tangential E on the sphere r = 1
    surf = _octant_points(rng, 40, 1.0, 1.0)
    Es = analytic.tm_xyz_e(k, surf)
    tang = Es - (Es * surf).sum(axis=1)[:, None] * surf
    assert np.max(np.linalg.norm(tang, axis=1)) < 1e-6 * np.max(np.linalg.norm(Es, axis=1))
    # on x = 0: E_y = E_z = 0 and B_x = 0 (likewise for y and z)
    for a in range(3):
        q = _octant_points(rng, 20, 0.2, 0.9)
        q[:, a] = 0.0
        Eq, Bq = analytic.tm_xyz_e(k, q), analytic.tm_xyz_b(k, q)
        others = [b for b in range(3) if b != a]
        assert np.max(np.abs(Eq[:, others])) < 1e-6 * np.max(np.abs(Eq)) + 1e-12
        assert np.max(np.abs(Bq[:, a])) < 1e-12 * scale + 1e-14
    # a wrong root fails the conductor condition: TE_2's k leaves tangential E
    Ew = analytic.tm_xyz_e(5.763459, surf)
    tw = Ew - (Ew * surf).sum(axis=1)[:, None] * surf
    assert np.max(np.linalg.norm(tw, axis=1)) > 1e-2 * np.max(np.linalg.norm(Ew, axis=1))
