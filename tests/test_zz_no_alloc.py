"""dm_operator_apply_noalloc: the operator apply for callers that must not
allocate once running (it stages through a static device scratch instead of
cudaMalloc).  Its output must equal dm_operator_apply's on consecutive calls,
whether this file runs alone in a fresh process or after the other tests
(which leave other contents in the shared scratch)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("make", [lambda: W.sphere_workload(24, offset_seed=W.SEED_BASE + 2, sigma=5.0),
                                  lambda: W.box_workload(12, 10, 8, 1.0, 0.8, 0.6, sigma=7.0)])
def test_noalloc_matches_apply_on_consecutive_calls(dm, ctx, make):
    import torch
    w = make()
    geom = dm.Geometry.from_workload(ctx, w)
    op = dm.Operator(ctx, geom, w.sigma)
    rng = np.random.default_rng(7)
    for level in range(op.num_levels):
        F = geom.level_info(level)["faces"]
        for _ in range(2):   # two calls in a row: the second sees the first call's scratch contents
            x = torch.from_numpy(rng.standard_normal(F)).cuda()
            ref = op.apply(x, level=level).cpu().numpy()
            got = op.apply_noalloc(x, level=level).cpu().numpy()
            assert _rel(got, ref) < 1e-13, (level, _rel(got, ref))


def test_noalloc_rejects_levels_beyond_the_scratch(dm, ctx):
    import torch
    w = W.sphere_workload(112, sigma=5.0)
    geom = dm.Geometry.from_workload(ctx, w)
    op = dm.Operator(ctx, geom, w.sigma, autotune=0)
    F = geom.level_info(0)["faces"]
    x = torch.zeros(F, dtype=torch.float64, device="cuda")
    with pytest.raises(dm.DMError) as err:
        op.apply_noalloc(x, level=0)
    assert "scratch" in str(err.value)
    # a coarser level of the same operator fits
    F1 = geom.level_info(1)["faces"]
    x1 = torch.from_numpy(np.random.default_rng(1).standard_normal(F1)).cuda()
    assert _rel(op.apply_noalloc(x1, level=1).cpu().numpy(), op.apply(x1, level=1).cpu().numpy()) < 1e-13


def test_noalloc_creates_no_buffer_event_or_stream(dm, ctx):
    """The property the entry point exists for: after its first call on the
    device (which only looks up the scratch's address), further calls leave the
    library's count of created device buffers, pinned buffers, events, streams
    and graphs unchanged, even while kernel tracing is on."""
    import torch
    w = W.sphere_workload(16, offset_seed=W.SEED_BASE + 1, sigma=5.0)
    geom = dm.Geometry.from_workload(ctx, w)
    op = dm.Operator(ctx, geom, w.sigma)
    F = geom.level_info(0)["faces"]
    x = torch.from_numpy(np.random.default_rng(3).standard_normal(F)).cuda()
    y = torch.empty_like(x)
    op.apply_noalloc(x, out=y)
    ctx.trace(True)
    try:
        before = dm.lib.dm_debug_allocation_count()
        for _ in range(3):
            op.apply_noalloc(x, out=y)
        after = dm.lib.dm_debug_allocation_count()
    finally:
        ctx.trace(False)
    assert after == before, (before, after)
    # the calls were not traced (tracing would have created events)
    assert ctx.trace_stats() == {}
    assert _rel(y.cpu().numpy(), op.apply(x).cpu().numpy()) < 1e-13
