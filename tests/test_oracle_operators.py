"""Pins of the oracle's assembled operators (Eq. farInt, divB, discWaveB,
discLaplB, discLaplDM, proj)."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import analytic, eigen, geometry, operators


def _ops(w):
    return operators.DMOperators(w.grid, geometry.fractions(w.phi))


def test_div_curl_is_exactly_zero():
    """Sec. 4.2: the Yee layout gives D C = 0 (div curl = 0), also with non-cubic cells."""
    ops = _ops(W.box_workload(5, 4, 3, 1.0, 0.7, 0.45))
    assert abs(ops.D @ ops.C).max() == 0.0


def test_dm_div_of_dm_curl_vanishes():
    """Sec. 5.1: D A (A^-1 C L e) = 0 for any edge field e (cut geometry)."""
    ops = _ops(W.sphere_workload(10, offset_seed=7))
    e = np.random.default_rng(0).standard_normal(ops.l.size)
    b = np.where(ops.open, (ops.C @ (ops.l * e)) / np.where(ops.open, ops.a, 1.0), 0.0)
    assert np.abs(ops.D @ (ops.a * b)).max() < 1e-9 * np.abs(ops.C @ (ops.l * e)).max() / min(ops.h)


def test_operator_symmetric():
    """Sec. 5.2: K - sigma A (Eq. discLaplDM) is symmetric."""
    ops = _ops(W.sphere_workload(10, offset_seed=7))
    K = ops.K(5.0)
    assert abs(K - K.T).max() < 1e-12 * abs(K).max()


@pytest.mark.parametrize("dims", [(4, 3, 3, 1.0, 0.8, 0.6), (12, 10, 8, 1.0, 0.8, 0.6)])
def test_box_curl_curl_closed_form(dims):
    """Grid-aligned PEC box: A^-1 C L C^T = C C^T on interior faces (Eq. discWaveB);
    its nonzero spectrum is the closed-form discrete Yee spectrum."""
    nx, ny, nz, lx, ly, lz = dims
    w = W.box_workload(nx, ny, nz, lx, ly, lz)
    ops = _ops(w)
    k2, _ = eigen.dense_modes(ops)
    g = w.grid
    ref = analytic.box_eigenvalues(nx, ny, nz, g.dx, g.dy, g.dz)
    assert k2.size == ref.size == analytic.box_mode_count(nx, ny, nz)
    assert np.max(np.abs(k2 - ref) / ref) < 1e-11


def test_box_vector_laplacian_spectrum():
    """Eq. discLaplB: K = C C^T + D^T D has the curl-curl spectrum plus the
    Neumann scalar spectrum (the divergent modes), nothing else."""
    w = W.box_workload(4, 3, 3, 1.0, 0.8, 0.6)
    ops = _ops(w)
    g = w.grid
    got = eigen.dense_spectrum_K(ops)
    ref = np.sort(np.concatenate([analytic.box_eigenvalues(4, 3, 3, g.dx, g.dy, g.dz),
                                  analytic.box_scalar_eigenvalues(4, 3, 3, g.dx, g.dy, g.dz)]))
    assert got.size == ref.size
    assert np.max(np.abs(got - ref) / ref) < 1e-11


def test_dm_vector_laplacian_splits_into_em_and_gradient_modes():
    """Sec. 5.1-5.2: the spectrum of (K, A) on a cut geometry is the
    electromagnetic spectrum of (C L C^T, A) plus the nonzero spectrum of the
    scalar pencil (D A D^T, V) on active cells, with the right multiplicities."""
    w = W.sphere_workload(8, offset_seed=11)
    ops = _ops(w)
    spec = eigen.dense_spectrum_K(ops)
    em, _ = eigen.dense_modes(ops)
    S = ops.scalar_laplacian()
    act = np.nonzero(np.asarray(abs(S).sum(axis=1)).ravel() > 0)[0]
    mu = sla.eigvalsh(S[act][:, act].toarray(), np.diag(ops.v[act]))
    ncomp = ops.vacuum_components()
    mu = np.sort(mu)[ncomp:]
    assert spec.size == em.size + mu.size
    ref = np.sort(np.concatenate([em, mu]))
    assert np.max(np.abs(spec - ref) / ref) < 1e-9


def test_projection_properties():
    """Eq. proj: P_DM^2 = P_DM, P_DM kills (masked) gradients D^T psi, keeps
    electromagnetic modes, and its output is A-orthogonal to gradients."""
    w = W.sphere_workload(10, offset_seed=3)
    ops = _ops(w)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(ops.a.size) * ops.open
    px = ops.project(x)
    assert np.linalg.norm(ops.project(px) - px) < 1e-10 * np.linalg.norm(px)
    psi = rng.standard_normal(ops.v.size)
    g = (ops.D.T @ psi) * ops.open
    assert np.linalg.norm(ops.project(g)) < 1e-10 * np.linalg.norm(g)
    # D A (P x) = 0
    assert np.linalg.norm(ops.D @ (ops.a * px)) < 1e-9 * np.linalg.norm(ops.D @ (ops.a * x))
    k2, B = eigen.dense_modes(ops)
    b = B[:, 0]
    assert np.linalg.norm(ops.project(b) - b) < 1e-9 * np.linalg.norm(b)


def test_sphere_spurious_modes_are_the_neumann_scalar_modes():
    """Sec. 5.1: the Dey--Mittra grad-div term adds the scalar Laplacian's
    spectrum as curl-free, divergent modes and leaves the electromagnetic ones
    alone.  On the cut-cell sphere the lowest eigenvalues of (K, A) are the
    l = 1 Neumann triplet (kR = 2.0816, the first zero of j_1') with curl-free
    eigenvectors, and the next is the divergence-free TM_1 mode (kR = 2.7437)."""
    import scipy.sparse.linalg as spla
    w = W.sphere_workload(16, sigma=5.0)
    ops = _ops(w)
    K = ops.restrict(ops.K(0.0)).tocsc()
    M = ops.restrict(ops.A).tocsc()
    lam, vec = spla.eigsh(K, k=4, M=M, sigma=-1.0, which="LM")
    o = np.argsort(lam)
    lam, vec = lam[o], vec[:, o]
    neumann = analytic.sphere_neumann_modes()[0]
    assert neumann[1] == 1 and neumann[2] == 3
    tm1 = analytic.sphere_k2_list(1.0, 1)[0]
    for c in range(4):
        b = np.zeros(ops.a.size)
        b[ops.open_idx] = vec[:, c]
        curl = np.linalg.norm(ops.l * (ops.C.T @ b)) / np.linalg.norm(b)
        div = eigen.divergence_ratio(ops, b)
        if c < 3:
            assert abs(lam[c] - neumann[0] ** 2) / neumann[0] ** 2 < 1e-2, lam
            assert curl < 1e-10 and div > 1e-2, (c, curl, div)
        else:
            assert abs(lam[c] - tm1) / tm1 < 5e-3, lam
            assert div < 1e-8, (c, div)
