"""Pins of the oracle eigensolve (the result the GPU eigensolver must reproduce)."""
import numpy as np
import pytest

import workloads as W
from oracle import analytic, eigen, geometry, operators


def _ops(w):
    return operators.DMOperators(w.grid, geometry.fractions(w.phi))


def test_box_shift_invert_matches_closed_form():
    w = W.box_workload()
    ops = _ops(w)
    k2, B, info = eigen.shift_invert_modes(ops, w.sigma, w.nev)
    g = w.grid
    ref = analytic.box_eigenvalues(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)
    order = eigen.wanted_order(ref, w.sigma)[:w.nev]
    assert np.allclose(np.sort(ref[order]), k2, rtol=1e-12)
    for i in range(w.nev):
        c = eigen.certificate(ops, k2[i], B[:, i])
        assert c["rho"] < 1e-10 and c["delta"] < 1e-10


def test_sparse_equals_dense_on_small_sphere():
    w = W.sphere_workload(8, offset_seed=11, sigma=5.0, nev=6)
    ops = _ops(w)
    kd, Bd = eigen.dense_modes(ops)
    ks, Bs, _ = eigen.shift_invert_modes(ops, w.sigma, w.nev)
    ref = np.sort(kd[eigen.wanted_order(kd, w.sigma)[:w.nev]])
    assert np.allclose(ks, ref, rtol=1e-11)


def test_sphere_16_close_to_analytic():
    """Sec. 6.2: the Dey--Mittra sphere reproduces the TM_1 triplet at 16^3 to
    well under 1% (second-order error)."""
    w = W.sphere_workload(16)
    ops = _ops(w)
    k2, B, _ = eigen.shift_invert_modes(ops, w.sigma, w.nev)
    ref = analytic.sphere_k2_list(1.0, 4)
    assert np.all(np.abs(k2[:3] - ref[:3]) / ref[:3] < 5e-3)
    for i in range(w.nev):
        assert eigen.certificate(ops, k2[i], B[:, i])["rho"] < 1e-10


@pytest.mark.slow
def test_frequency_convergence_second_order_and_first_order_with_face_neglect():
    """Sec. 6.2, Fig. freqErr3d: the unaltered Dey--Mittra method converges at
    second order in the frequency (the TM_1 error drops ~4x per refinement);
    dropping cut faces with a < a_min (Sec. 3; here a_min = 0.1 a_vac) leaves
    first-order convergence and larger errors."""
    ref = np.sqrt(analytic.sphere_k2_list(1.0, 3)[0])
    errs = {}
    for a_min in (0.0, 0.1):
        for n in (16, 32):
            w = W.sphere_workload(n, offset_seed=W.SEED_BASE + 2, sigma=7.0, nev=3)
            ops = operators.DMOperators(w.grid, geometry.fractions(w.phi, a_min=a_min))
            k2, _, _ = eigen.shift_invert_modes(ops, 7.0, 3)
            errs[a_min, n] = abs(np.sqrt(k2.mean()) - ref) / ref
    assert errs[0.0, 16] / errs[0.0, 32] > 2.8, errs
    order = {a: np.log2(errs[a, 16] / errs[a, 32]) for a in (0.0, 0.1)}
    assert order[0.1] < 1.5, (order, errs)
    assert errs[0.1, 32] > 3.0 * errs[0.0, 32], errs


def test_octant_lowest_mode_is_the_l3_tm_mode_at_second_order():
    """Sec. 6.2: with perfectly conducting planes at x, y, z = 0 (here the
    grid's own walls) the lowest mode of the sphere octant is the TM mode of
    l = 3 whose angular part is x y z / r^3 (kR = 4.973420, the only l = 3
    combination that vanishes tangentially on all three planes); the TM_1,
    TM_2 and TE_1 modes do not fit the planes.  It is not degenerate, and its
    eigenvalue converges at second order."""
    k3 = [r for r, kind, l, _ in analytic.sphere_modes(xmax=6.0) if kind == "TM" and l == 3][0]
    errs = {}
    for n in (12, 24):
        w = W.octant_sphere_workload(n)
        ops = operators.DMOperators(w.grid, geometry.fractions(w.phi))
        k2, _, _ = eigen.shift_invert_modes(ops, 20.0, 2)
        k2 = np.sort(k2)
        assert k2[1] > 1.3 * k2[0], k2                     # the next mode (TE_2) is far above
        errs[n] = abs(k2[0] - k3 ** 2) / k3 ** 2
    assert errs[24] < 3e-3, errs
    assert np.log2(errs[12] / errs[24]) > 1.8, errs


@pytest.mark.slow
def test_octant_surface_fields_converge_only_without_face_neglect():
    """Sec. 6.2, Eq. errorNorm / Fig. fieldErr3d on the oracle: the electric
    field of the octant's lowest mode on a shell 3 dx inside the surface
    converges (at about second order) when every cut face is kept, and does
    not converge when faces below a_min = 0.1 a_vac are neglected."""
    from field_sampling import surface_field_error
    err = {}
    for a_min in (0.0, 0.1):
        for n in (16, 24):
            w = W.octant_sphere_workload(n)
            ops = operators.DMOperators(w.grid, geometry.fractions(w.phi, a_min=a_min))
            _, B, _ = eigen.shift_invert_modes(ops, w.sigma, 1)
            err[a_min, n] = surface_field_error(w, a_min, B[:, 0])
    assert err[0.0, 16] / err[0.0, 24] > (24 / 16) ** 1.5, err     # ~ second order
    assert err[0.1, 16] / err[0.1, 24] < 1.2, err                   # no convergence
    assert err[0.1, 24] > 3.0 * err[0.0, 24], err
