"""lim_run_batch_static: batch runs for callers that cannot allocate device memory.

A real-time control loop that must not block on the allocator, or a process
whose GPU memory belongs to another framework's pool, cannot call cudaMalloc
while it runs trajectories.  lim_run_batch_static uses a 64 MiB workspace built
into the library instead of a caller buffer.  These tests check, through the C
ABI, that it returns exactly what lim_run_batch returns (records, tallies and
final residuals of the same shots, bit for bit), twice in a row on the shared
array, and that a batch too large for the array is refused.  This file is
collected last.
"""
import numpy as np
import pytest

from paper_2609_38139_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_38139_b300 import build, lim
    build.build()
    return lim


def _points(ctx, shot0):
    t8 = ctx.from_inputs(I.toric2d(8))
    t40 = ctx.from_inputs(I.toric2d(40))
    bb = ctx.from_inputs(I.bb_code(12, 6))
    return [(t40, 0.06, 40, shot0, 0, 160), (t8, 0.05, 300, shot0, 1, 32),
            (bb, 0.04, 200, shot0, 2, 200)], (t8, t40, bb)


def test_static_workspace_matches_caller_workspace(L):
    ctx = L.Context(0)
    # four 256-thread blocks per SM: the L=40 messages do not fit in shared
    # memory and live in the workspace's per-team slots
    prm = L.params(precision="f32", tick_budget=32, variant="cta", block_threads=256,
                   blocks_per_sm=4)
    pts, keep = _points(ctx, 0)
    ws = L.workspace_size(ctx, pts, prm)
    assert 1 << 20 < ws <= 64 << 20
    for call, shot0 in enumerate((0, 1000)):  # two calls in a row share the array
        pts, keep = _points(ctx, shot0)
        tal_ref, rec_ref, fin_ref = L.run_batch(ctx, pts, prm, 17, e_final=True)
        tal, rec, fin = L.run_batch_static(ctx, pts, prm, 17, e_final=True)
        assert np.array_equal(rec, rec_ref), call
        assert np.array_equal(tal, tal_ref), call
        assert np.array_equal(fin, fin_ref), call
        assert int(tal["errors"].sum()) == 0 and int(tal["shots"].sum()) == 540


def test_static_workspace_refuses_oversized_batch(L):
    ctx = L.Context(0)
    big = ctx.from_inputs(I.toric2d(128))
    prm = L.params(precision="f32", tick_budget=100, variant="cta")
    assert L.workspace_size(ctx, [(big, 0.05, 10, 0, 0)], prm) > 64 << 20
    with pytest.raises(L.LimError, match="LIM_E_NOMEM"):
        L.run_batch_static(ctx, [(big, 0.05, 10, 0, 0)], prm, 1)
