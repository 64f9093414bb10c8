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
