"""Plain FP64 CPU oracle of the Dey--Mittra shift-and-invert eigensolver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
CUDA path never calls into it and shares no code with it; both take their
inputs from the ``workloads`` module, which holds none of the method's
arithmetic.

Modules and the passages of Bauer, Werner & Cary (arXiv:1301.3794) they follow:

* ``geometry``   cut lengths l, areas a and volumes v *outside* the conductor
                 (Sec. 2, Eq. farInt / Fig. dmFace; Sec. 5.1, Eq. divBInt /
                 Fig. dmVol), measured on the piecewise-linear level set of a
                 conforming tetrahedral split of every cell (Sec. 6.1, the
                 "tetrahedral subvolumes" of the cut-cell volume routine).
* ``operators``  curl C (Eq. farInt, Eq. discWaveB), divergence D (Eq. divB),
                 the Dey--Mittra curl-curl A^-1 C L C^T (Eq. discWaveBDM), the
                 A-scaled shifted vector Laplacian K - sigma A (Eq. discLaplDM),
                 the projection P_DM (Eq. proj) -- assembled as sparse matrices.
* ``eigen``      the eigenpairs the method converges to: the generalised
                 symmetric-definite problem C L C^T b = k^2 A b restricted to the
                 divergence-free (D A b = 0) modes (Eq. discWaveBDM, Eq. fullMat),
                 by dense eigh on tiny grids and sparse shift-invert otherwise;
                 the residual certificate of a computed eigenpair.
* ``analytic``   closed-form discrete Yee eigenvalues of a PEC box and the
                 spherical-cavity wavenumbers from Bessel-function zeros (Sec.
                 6.2), used to pin the oracle itself.
* ``multigrid``  the library's geometric V-cycle, the preconditioner of
                 the inner solve (the paper used algebraic multigrid, Sec. 6):
                 written out as plain sparse-matrix steps in the order the
                 V-cycle takes them.
"""
