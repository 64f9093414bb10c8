"""The cut-cell volumes in the grad-div term decide the multigrid's speed (Sec. 6.1).

The paper reports that without V^-1 in K (Eq. discLaplDM) the multigrid-
preconditioned GMRES needs more than 400 iterations, and that random errors in
the cut-cell volumes, v~ = 10^(f eps) v with f ~ U[-1, 1] on cut cells only
(Eq. volPert1), raise the average iteration count from 10 (eps = 0.1) to 24
(eps = 1) and 220 (eps = 3) (Tab. volPert1, 32^3 sphere, tolerance 1e-6).
Both effects are pinned here on the oracle's V-cycle inside FGMRES; the
electromagnetic modes do not depend on V (Sec. 5.1), only the solver does."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import geometry, multigrid as MG


def _iterations(w, fine, maxiter):
    levels = MG.build_vector_hierarchy(w.grid, w.phi, w.sigma, fine=fine)
    om = []
    for lev in levels:
        idx = np.nonzero(lev.mask)[0]
        Kd = lev.K.tocsr()[idx][:, idx]
        dinv = lev.inv_d[idx]
        op = spla.LinearOperator(Kd.shape, matvec=lambda v, Kd=Kd, dinv=dinv: dinv * (Kd @ v))
        om.append(1.7 / abs(spla.eigs(op, k=1, which="LM", return_eigenvectors=False, tol=1e-6)[0]))
    lev = levels[0]
    b = np.random.default_rng(0).standard_normal(lev.K.shape[0]) * lev.mask
    _, hist = MG.fgmres(lambda v: lev.K @ v, b, lambda v: MG.vcycle(levels, v, om), tol=1e-6, maxiter=maxiter)
    return len(hist), hist[-1]


@pytest.fixture(scope="module")
def sphere():
    w = W.sphere_workload(16, sigma=5.0, offset_seed=W.SEED_BASE + 2)
    return w, geometry.fractions(w.phi)


def _with_volumes(fr, v):
    out = dict(fr)
    out["V"] = v
    return out


def test_leaving_out_inverse_volumes_stalls_the_solver(sphere):
    w, fr = sphere
    it_v, res_v = _iterations(w, fr, 60)
    # V = 1 on every active cell: V^-1 left out of K
    it_no, res_no = _iterations(w, _with_volumes(fr, (fr["V"] > 0).astype(float)), 60)
    assert res_v <= 1e-6 and it_v <= 15, (it_v, res_v)
    assert it_no == 60 and res_no > 1e-3, (it_no, res_no)


def test_volume_errors_slow_the_solver(sphere):
    w, fr = sphere
    v = fr["V"]
    cut = (v > 0) & (v < 1)
    f = np.random.default_rng(7).uniform(-1.0, 1.0, v.shape)
    its = {}
    for eps in (0.1, 1.0, 3.0):
        its[eps], res = _iterations(w, _with_volumes(fr, np.where(cut, 10.0 ** (f * eps) * v, v)), 60)
        if eps < 3.0:
            assert res <= 1e-6, (eps, its[eps], res)
    assert its[0.1] <= its[1.0] < its[3.0], its
    assert its[3.0] >= 4 * its[0.1], its
