"""Oracle: the eigenpairs the Dey--Mittra eigensolver converges to.

The paper's iteration (Eq. fullMat) is a shift-and-invert Krylov method on
P_DM (K - sigma A)^-1 A.  Its eigenvalues are 1/(k^2 - sigma) for the
electromagnetic modes -- the nonzero-k^2 solutions of the Dey--Mittra wave
equation A^-1 C L C^T b = k^2 b (Eq. discWaveBDM), which satisfy D A b = 0 -- and
0 for the divergent ones (Sec. 5.2).  The grad-div term and the projection only
change the speed of convergence (Sec. 5.1: electromagnetic modes are unchanged
by the added term).  So the result has a plain definition, written out here:

* dense path (tiny grids): the generalised symmetric-definite problem
  C L C^T b = k^2 A b on the open faces, keeping k^2 > 0;
* sparse path: shift-invert Lanczos (ARPACK) on K b = lambda A b with
  K = C L C^T + alpha A D^T V^-1 D A (Eq. discLaplDM with the grad-div term
  weighted), whose spectrum is the electromagnetic modes plus the spurious
  gradient modes; the latter are recognised by D A b != 0 and dropped.

The wanted modes are the ``nev`` electromagnetic eigenvalues nearest sigma (the
largest |1/(k^2 - sigma)| of Eq. shiftInv), ties broken towards lower k^2.

Eigenvectors are returned on the full face space, A-normalised (b^T A b = 1),
sign fixed so that the entry of largest magnitude is positive.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


def _normalise(ops, B):
    B = np.array(B, dtype=np.float64, copy=True)
    for c in range(B.shape[1]):
        b = B[:, c]
        b /= np.sqrt(b @ (ops.a * b))
        if b[np.argmax(np.abs(b))] < 0:
            b *= -1.0
    return B


def divergence_ratio(ops, b):
    """||D A b|| h / ||A b||: ~1e-15 for electromagnetic modes, O(1) for gradients."""
    h = min(ops.h)
    Ab = ops.a * b
    return np.linalg.norm(ops.D @ Ab) * h / max(np.linalg.norm(Ab), 1e-300)


def dense_modes(ops, rel_zero=1e-8):
    """All electromagnetic modes by dense eigh of (C L C^T, A) on the open faces.

    Returns (k2 ascending, B full-space A-normalised columns)."""
    o = ops.open_idx
    Kc = ops.CLCt.tocsr()[o][:, o].toarray()
    lam, vec = sla.eigh(Kc, np.diag(ops.a[o]))
    keep = lam > rel_zero * lam.max()
    B = np.zeros((ops.a.size, int(keep.sum())))
    B[o] = vec[:, keep]
    return lam[keep], _normalise(ops, B)


def dense_spectrum_K(ops, sigma=0.0):
    """Whole spectrum of (K - sigma A, A) on the open faces (dense eigh)."""
    o = ops.open_idx
    Kc = ops.K(sigma).tocsr()[o][:, o].toarray()
    return sla.eigvalsh(Kc, np.diag(ops.a[o]))


def wanted_order(k2, sigma):
    """Indices sorted by distance to sigma, ties towards lower k^2."""
    return np.lexsort((k2, np.round(np.abs(k2 - sigma), 12)))


def shift_invert_modes(ops, sigma, nev, extra=None, tol=1e-13, div_tol=1e-6, alpha=100.0):
    """The ``nev`` electromagnetic modes nearest sigma by sparse shift-invert.

    Lanczos (ARPACK, sparse LU) runs on C L C^T + alpha A D^T V^-1 D A against A.
    Sec. 5.1: the grad-div term leaves every electromagnetic mode unchanged
    (D A b = 0), whatever its weight; weighting it by alpha moves the divergent
    modes alpha times further from sigma, so they can no longer be degenerate
    with (and mix into) the wanted modes -- on a box they coincide exactly at
    alpha = 1.  Modes with D A b != 0 that still show up are dropped.

    Returns (k2 ascending, B full-space A-normalised, info dict)."""
    o = ops.open_idx
    Kal = ops.restrict((ops.CLCt + alpha * ops.GD).tocsr())
    M = ops.restrict(ops.A)
    n = o.size
    k = nev + (extra if extra is not None else max(6, nev // 2))
    while True:
        k = min(k, n - 2)
        lam, vec = spla.eigsh(Kal, k=k, M=M, sigma=sigma, which="LM", tol=tol)
        full = np.zeros((ops.a.size, k))
        full[o] = vec
        ratio = np.array([divergence_ratio(ops, full[:, c]) for c in range(k)])
        phys = ratio < div_tol
        lam_p, B_p = lam[phys], full[:, phys]
        if lam_p.size >= nev + 1 or k >= n - 2:
            break
        k = min(2 * k, n - 2)
    order = wanted_order(lam_p, sigma)[:nev]
    lam_w = lam_p[order]
    B_w = B_p[:, order]
    srt = np.argsort(lam_w)
    info = {"requested": k, "spurious_dropped": int((~phys).sum()),
            "next_physical": float(lam_p[wanted_order(lam_p, sigma)[nev]]) if lam_p.size > nev else None}
    return lam_w[srt], _normalise(ops, B_w[:, srt]), info


def certificate(ops, k2, b):
    """Residual certificate of one eigenpair (k2, b) of the original problem.

    rho   = ||K b - k2 A b|| / (k2 ||A b||)  with K = C L C^T + A D^T V^-1 D A,
    delta = ||D A b|| h / ||A b||           (divergence of the mode),
    rq    = b^T K b / b^T A b               (Rayleigh quotient).
    """
    Kb = ops.apply_K(b, 0.0)
    Ab = ops.a * b
    rho = np.linalg.norm(Kb - k2 * Ab) / (abs(k2) * np.linalg.norm(Ab))
    return {"rho": float(rho), "delta": float(divergence_ratio(ops, b)),
            "rq": float((b @ Kb) / (b @ Ab))}


def subspace_angle_max(ops, B1, B2):
    """Largest principal angle between span(B1) and span(B2) in the A inner product."""
    w = np.sqrt(ops.a)
    Q1, _ = np.linalg.qr(B1 * w[:, None])
    Q2, _ = np.linalg.qr(B2 * w[:, None])
    s = np.linalg.svd(Q1.T @ Q2, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))
