"""traj_solve_noalloc: the solve for callers that cannot allocate device memory.

Such callers (code under an allocator or memory pool that another framework
owns, plugins limited to the buffers they are handed, real-time paths where an
allocation could stall) cannot create a traj_batch, whose workspace is
allocated. This entry point keeps its intermediates in one fixed-size array
that the library reserves at load time. The test calls it through the C ABI
twice in a row, on two different batches, and compares each result with the
handle-based solve at the parity tolerance of the other GPU tests. It lives in
a file that pytest collects last, so that a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

from paper_2408_10731_b300 import scenes
from tests.gpu_helpers import POS_TOL, gpu_solve, position_error

pytestmark = pytest.mark.gpu


def _noalloc(batch, iters, tol):
    import torch
    from paper_2408_10731_b300 import trajbatch as tb
    dev = torch.device("cuda", 0)
    t = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    B, D = batch.n_traj, batch.dim
    out = dict(xi=torch.full((B, D, 11), float("nan"), device=dev),
               residual=torch.full((B, 3), float("nan"), device=dev),
               iters=torch.full((B,), -1, dtype=torch.int32, device=dev),
               status=torch.full((B,), -1, dtype=torch.int8, device=dev))
    tb.solve_noalloc(D, batch.vmax, batch.amax, batch.rho, batch.n_steps, batch.duration,
                     batch.start, batch.goal, batch.offsets, t(batch.centers, torch.float32),
                     t(batch.semi_axes, torch.float32), t(batch.velocities, torch.float32),
                     t(batch.traj_problem, torch.int32), t(batch.xi0, torch.float32), iters, tol,
                     out["xi"], out["residual"], out["iters"], out["status"])
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_noalloc_matches_handle_solve_on_two_calls_in_a_row():
    first = scenes.config2(11, n_scenes=16, inits=8)
    second = scenes.config4(3, n_problems=24, inits=4)  # uneven horizons and obstacle counts
    for batch, iters, tol in ((first, 150, 1e-3), (second, 60, -1.0)):
        got = _noalloc(batch, iters, tol)
        ref = gpu_solve(batch, iters, tol=tol)
        err = position_error(batch, got["xi"], ref["xi"])
        assert err.max() <= POS_TOL, err.max()
        np.testing.assert_allclose(got["residual"], ref["residual"], atol=2e-5, rtol=1e-4)
        np.testing.assert_array_equal(got["iters"], ref["iters"])
        np.testing.assert_array_equal(got["status"], ref["status"])


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.config2(0, n_scenes=1, inits=2)
    dev = torch.device("cuda", 0)
    dummy = torch.zeros(16, device=dev)
    many = np.zeros(8193, np.int32)
    with pytest.raises(tb.TrajBatchError) as e:
        tb.solve_noalloc(2, 1.5, 2.0, 1.0, b.n_steps, b.duration, b.start, b.goal, b.offsets,
                         dummy, dummy, dummy, torch.as_tensor(many, device=dev), dummy, 10, 1e-3,
                         dummy, dummy, dummy.int(), dummy.to(torch.int8))
    assert e.value.code == -4 and "8192" in str(e.value)
