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


def _args(batch, n_traj):
    import torch
    dev = torch.device("cuda", 0)
    n_obs, D = int(batch.offsets[-1]), batch.dim
    t = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    return dict(centers=t(batch.centers, torch.float32), semi_axes=t(batch.semi_axes, torch.float32),
                velocities=t(batch.velocities, torch.float32),
                traj_problem=torch.zeros(n_traj, dtype=torch.int32, device=dev),
                coeffs0=torch.zeros(n_traj, D, 11, device=dev),
                coeffs=torch.zeros(n_traj, D, 11, device=dev),
                residual=torch.zeros(n_traj, 3, device=dev),
                iters=torch.zeros(n_traj, dtype=torch.int32, device=dev),
                status=torch.zeros(n_traj, dtype=torch.int8, device=dev))


def _call(batch, a, iters=10, tol=1e-3):
    from paper_2408_10731_b300 import trajbatch as tb
    tb.solve_noalloc(batch.dim, batch.vmax, batch.amax, batch.rho, batch.n_steps, batch.duration,
                     batch.start, batch.goal, batch.offsets, a["centers"], a["semi_axes"],
                     a["velocities"], a["traj_problem"], a["coeffs0"], iters, tol, a["coeffs"],
                     a["residual"], a["iters"], a["status"])


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.config2(0, n_scenes=1, inits=2)
    with pytest.raises(tb.TrajBatchError) as e:
        _call(b, _args(b, 8193))
    assert e.value.code == -4 and "8192" in str(e.value)


def test_noalloc_rejects_a_problem_index_out_of_range_on_the_device():
    """traj_problem lives in device memory; an entry outside [0, n_problems) is found
    by a range check on the device before any kernel indexes the problem records, and
    the call returns TRAJ_EINVAL with the outputs untouched."""
    import torch
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.config2(0, n_scenes=2, inits=2)
    for bad in (2, -1, 255):
        a = _args(b, 4)
        a["traj_problem"] = torch.tensor([0, 1, bad, 0], dtype=torch.int32, device="cuda")
        a["coeffs0"].copy_(torch.as_tensor(b.xi0, device="cuda"))
        a["iters"].fill_(-7)
        with pytest.raises(tb.TrajBatchError) as e:
            _call(b, a)
        assert e.value.code == -1 and "traj_problem" in str(e.value)
        assert bool((a["iters"] == -7).all())
    # a valid map right after works (the flag does not stick)
    a = _args(b, 4)
    a["traj_problem"] = torch.tensor([0, 1, 1, 0], dtype=torch.int32, device="cuda")
    a["coeffs0"].copy_(torch.as_tensor(b.xi0, device="cuda"))
    _call(b, a)
    assert bool((a["iters"] >= 1).all())


def test_noalloc_binding_refuses_a_short_output_tensor():
    import torch
    b = scenes.config2(0, n_scenes=1, inits=2)
    a = _args(b, 2)
    a["coeffs"] = torch.zeros(2, 2, 10, device="cuda")
    with pytest.raises(ValueError, match="coeffs holds 40 values, needs 44"):
        _call(b, a)
