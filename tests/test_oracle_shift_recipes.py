"""Pins of the shift reading for the batch and 9-cell workloads.

Sec. 4.1 asks for a shift of the order of the operator's smallest nonzero
eigenvalue and warns that inverting K - sigma A becomes intractable as sigma
moves into the spectrum.  The recipes therefore keep every shift below the
cavity's lowest electromagnetic mode (batch) or below the whole spectrum of the
pencil (K, A) (9-cell cavity).  Both are checked here with the oracle on coarse
versions of the same cavities."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import eigen, geometry, operators


def _lowest_em_k2(w):
    ops = operators.DMOperators(w.grid, geometry.fractions(w.phi))
    k2, _, _ = eigen.shift_invert_modes(ops, 0.0, 1)
    return float(k2[0])


@pytest.mark.parametrize("index", [0, 1, 3, 5, 9, 22])
def test_batch_shifts_lie_below_the_lowest_mode(index):
    w, shifts, _ = W.batch_workloads(48)[index]
    n = 20
    if w.name.startswith("sphere"):
        wc = W.sphere_workload(n, sigma=shifts[0], offset_seed=w.seed)
    else:
        wc = W.ellipsoid_workload(n, seed=w.seed, sigma=shifts[0])
    lowest = _lowest_em_k2(wc)
    # the coarse grid moves the mode by O(h^2); keep a margin of 5%
    assert max(shifts) < 0.95 * lowest, (w.name, shifts, lowest)


def test_ninecell_shift_keeps_the_pencil_definite():
    w = W.nine_cell_workload(nxy=12, nz=144)
    ops = operators.DMOperators(w.grid, geometry.fractions(w.phi))
    K = ops.restrict(ops.K(0.0)).tocsc()
    M = ops.restrict(ops.A).tocsc()
    lam = spla.eigsh(K, k=1, M=M, sigma=-1.0, which="LM", return_eigenvectors=False)
    lowest = float(np.min(lam))
    assert 0.0 < w.sigma < lowest, (w.sigma, lowest)
