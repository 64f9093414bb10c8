"""The C-ABI library builds, loads and exports every symbol include/dmeig.h
declares; argument checks that need no GPU."""
import ctypes as C
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1301_3794_gb300 import _lib
    return _lib.load()


def test_header_symbols_exported(lib):
    from paper_1301_3794_gb300 import _lib
    declared = _lib.header_symbols()
    assert len(declared) >= 25
    for name in declared:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_binding_covers_only_declared_symbols():
    from paper_1301_3794_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(_lib.header_symbols())


def test_struct_layouts_match_defaults(lib):
    from paper_1301_3794_gb300._lib import EigParams, MGParams
    p = EigParams()
    lib.dm_eig_params_default(C.byref(p))
    assert p.tol == 1e-10 and p.inner_tol == 1e-9 and p.nev == 4 and p.inner_restart == 40 and p.seed == 1301
    assert p.mg.max_coarse == 4 and p.mg.band_sweeps == 24 and p.mg.band_brick == 8 and p.mg.omega_scale == 1.7
    m = MGParams()
    lib.dm_mg_params_default(C.byref(m))
    assert m.power_iters == 30 and m.precision == 0
    assert m.autotune == 1 and m.stencil_shape == -1 and m.band_sweeps_coarse == 16 and m.symmetric_transform == 0
    assert m.dense_coarse == 2048 and m.krylov_ff == 1 and m.jacobi_sweeps == 2
    # the field after the embedded multigrid settings lands where the C struct has it
    assert p.mg.autotune == 1 and p.mg.stencil_shape == -1 and not p.learned


def test_null_arguments_rejected_without_gpu(lib):
    h = C.c_void_p()
    assert lib.dm_context_create(0, None, None) == 1          # DM_ERR_INVALID_ARG
    assert lib.dm_geometry_num_levels(None) == 0
    assert lib.dm_operator_num_levels(None) == 0
    assert lib.dm_last_error(None) == b"null context"
    assert lib.dm_eigensolve(None, None, None, None, None, 0, None) == 1


def test_no_cpu_fallback_in_package():
    """The product path has no CPU compute route: the package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1301_3794_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "oracle" not in src.replace("oracle.", ""), f
            assert "import oracle" not in src and "from oracle" not in src, f


def test_eig_params_tail_fields_keep_their_c_offsets(lib):
    """max_seconds, the last field, sits where the C struct has it: the C
    default routine overwrites a value planted there through ctypes."""
    from paper_1301_3794_gb300._lib import EigParams
    p = EigParams()
    p.max_seconds = 5.0
    p.rho_tol = 5.0
    p.learned = 1234
    lib.dm_eig_params_default(C.byref(p))
    assert p.max_seconds == 0.0 and not p.learned and p.rho_tol == 1e-8


def test_allocation_counter_needs_no_gpu(lib):
    assert lib.dm_debug_allocation_count() >= 0


def test_apply_noalloc_checks_both_tensors_before_any_library_call():
    """x and out must be contiguous float64 tensors of the level's face count on
    the operator's device; anything else is refused on the host, before the
    library (and the GPU) sees a pointer."""
    import types

    import numpy as np
    import torch

    import paper_1301_3794_gb300 as dm
    calls = []
    op = dm.Operator.__new__(dm.Operator)
    op.ctx = types.SimpleNamespace(device=0, check=lambda *a: calls.append(a))
    op.h = None
    op._faces = lambda level: 10
    good = torch.zeros(10, dtype=torch.float64)   # a CPU tensor: refused as not on cuda:0
    for bad_x in (np.zeros(10), good, torch.zeros(10, dtype=torch.float32), torch.zeros(12, dtype=torch.float64)):
        with pytest.raises(ValueError):
            op.apply_noalloc(bad_x)
    with pytest.raises(ValueError):
        op.apply_noalloc(good, out=torch.zeros(10, dtype=torch.float32))
    assert calls == []
