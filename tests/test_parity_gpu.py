"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar: max coefficient-evaluated position error <= 1e-5 m (grid points and
1000 uniform tau) after a fixed iteration count; residuals and iteration
decisions agree up to FP32 rounding. Inputs are the seeded scenes of
paper_2408_10731_b300.scenes (FP32-exact, so both sides see identical data).
"""
import dataclasses

import numpy as np
import pytest

from oracle import am
from paper_2408_10731_b300 import scenes
from tests.gpu_helpers import POS_TOL, gpu_solve, position_error, reduced_config4

pytestmark = pytest.mark.gpu


def _check(batch, iters, cost_mode=0, tol_pos=POS_TOL, **kw):
    g = gpu_solve(batch, iters, cost_mode=["smooth_track", "project"][cost_mode], **kw)
    o = am.solve(batch, iters, tol=-1.0, cost_mode=cost_mode)
    err = position_error(batch, g["xi"], o["xi"])
    assert err.max() <= tol_pos, (err.max(), np.argmax(err))
    np.testing.assert_allclose(g["residual"], o["residual"], atol=2e-5, rtol=1e-4)
    assert np.all(g["iters"] == iters)
    return g, o, err


def test_config1_parity_100_iterations():
    _check(scenes.config1(), 100)


def test_config1_feasible_parity_100_iterations():
    _check(scenes.config1(feasible=True), 100)


def test_config2_reduced_parity_20_iterations():
    b = scenes.config2(1, n_scenes=8, inits=8)
    g, o, _ = _check(b, 20)


def test_uneven_batch_parity_20_iterations():
    # every horizon of the uneven generator (50/75/100/150 steps) and obstacle counts 4..256
    b = reduced_config4(12, seed=2)
    assert set(int(n) for n in b.n_steps) == {50, 75, 100, 150}
    _check(b, 20)


def test_3d_projection_mode_parity_20_iterations():
    c3 = scenes.config3(0, n_traj=32)
    b = c3["batch"]
    z = scenes.normal_draws(7, (32, 33))
    L = np.linalg.cholesky(c3["sigma0"])
    xi0 = scenes.f32((c3["mu0"][None] + z @ L.T).reshape(32, 3, 11))
    _check(dataclasses.replace(b, xi0=xi0), 20, cost_mode=1)


def test_multipliers_and_contraction_parity():
    b = scenes.config2(4, n_scenes=4, inits=4)
    g = gpu_solve(b, 20, state=True)
    o = am.solve(b, 20, tol=-1.0, want_lambda=True)
    scale = np.abs(o["lam"]).max()
    assert np.abs(g["lam"] - o["lam"]).max() <= 1e-4 * scale


def test_early_stop_decisions_match_oracle():
    b = scenes.config2(0, n_scenes=6, inits=8)
    tol, cap = 1e-3, 200
    g = gpu_solve(b, cap, tol=tol)
    o = am.solve(b, cap, tol=-1.0, want_hist=True)
    h = o["hist"].max(axis=2)  # worst of the three residuals after each iteration
    slack = 5e-6
    for k in range(b.n_traj):
        it = int(g["iters"][k])
        if g["status"][k] == 0:
            assert 1 <= it <= cap
            assert h[k, it] <= tol + slack
            assert np.all(h[k, 1:it] > tol - slack)
        else:
            assert it == cap and np.all(h[k, 1:cap + 1] > tol - slack)
    assert (g["status"] == 0).sum() > 0


def test_full_size_config2_sampled_parity():
    """The bench workload (1024 trajectories, one launch); 24 sampled trajectories
    recomputed by the oracle one by one."""
    b = scenes.config2(0)
    g = gpu_solve(b, 20)
    pick = np.random.default_rng(5).choice(b.n_traj, 24, replace=False)
    sub = b.subset(pick)
    o = am.solve(sub, 20, tol=-1.0)
    err = position_error(sub, g["xi"][pick], o["xi"])
    assert err.max() <= POS_TOL, err.max()
    # properties that hold at any size: boundary rows, finite outputs, iteration counts
    assert np.all(np.isfinite(g["xi"])) and np.all(g["iters"] == 20)
    P, Pd, Pdd = am.bernstein(100, 10.0)
    np.testing.assert_allclose(g["xi"] @ P[0], b.start[b.traj_problem], atol=1e-4)
    np.testing.assert_allclose(g["xi"] @ P[-1], b.goal[b.traj_problem], atol=1e-4)


def test_full_size_uneven_sampled_parity():
    """The uneven workload at full size (2048 problems x 8 = 16384 trajectories, one
    launch) in the launch shapes the bench uses; 32 sampled trajectories, spread over
    every horizon, recomputed by the oracle one by one."""
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.config4(0)
    rng = np.random.default_rng(11)
    pick = np.concatenate([rng.choice(np.nonzero(b.n_steps[b.traj_problem] == n_p)[0], 8, replace=False)
                           for n_p in (50, 75, 100, 150)])
    o_full = am.solve(b.subset(pick), 20, tol=-1.0)
    h = tb.from_batch(b)
    try:
        for w, bps, team in ((8, 0, 2), (4, 0, 1)):
            h.set_launch_shape(w, bps, team)
            h.solve(20, tol=-1.0)
            g = h.get_trajectories()
            assert np.all(np.isfinite(g["xi"])) and np.all(g["iters"] == 20)
            err = position_error(b.subset(pick), g["xi"][pick], o_full["xi"])
            assert err.max() <= POS_TOL, (team, err.max())
    finally:
        h.close()


def test_determinism_and_shard_equivalence():
    """Trajectories are independent: a batch split into two shards (as replicas on
    two GPUs would run it) gives bitwise the same results as one launch."""
    b = scenes.config2(3, n_scenes=8, inits=8)
    full = gpu_solve(b, 30)
    again = gpu_solve(b, 30)
    np.testing.assert_array_equal(full["xi"], again["xi"])
    half = b.n_traj // 2
    for sl in (slice(0, half), slice(half, b.n_traj)):
        idx = np.arange(b.n_traj)[sl]
        part = gpu_solve(b.subset(idx), 30)
        np.testing.assert_array_equal(part["xi"], full["xi"][idx])
        np.testing.assert_array_equal(part["residual"], full["residual"][idx])


# ----------------------------------------------------------------------------- edge cases
def _problem(start, goal, n_p, T, centers, axes, xi0, vel=None, vmax=1.5, amax=2.0):
    dim = len(start)
    centers = np.asarray(centers, float).reshape(-1, dim)
    n_o = centers.shape[0]
    return scenes.Batch(
        dim=dim, n_steps=np.array([n_p], np.int32), duration=np.array([float(T)]),
        start=np.asarray(start, float)[None], goal=np.asarray(goal, float)[None],
        offsets=np.array([0, n_o], np.int32), centers=scenes.f32(centers),
        semi_axes=scenes.f32(np.asarray(axes, float).reshape(-1, dim)),
        velocities=np.zeros((n_o, dim)) if vel is None else scenes.f32(vel),
        traj_problem=np.zeros(xi0.shape[0], np.int32), xi0=scenes.f32(xi0), vmax=vmax, amax=amax)


def test_point_at_obstacle_centre_and_no_obstacles():
    """A grid point exactly at an obstacle centre: alpha = atan2(0, 0) = 0, so the
    target is the centre plus the x semi-axis. p(0) = xi_0 holds exactly, so an
    obstacle centred at the start puts t = 0 at ||u|| = 0 in the initial
    projection; its residual is the semi-axis and the first QP step is
    well-defined (later iterates sit at a non-zero but rounding-sized offset
    whose direction is arbitrary, so only iterate 1 is compared)."""
    start, goal = np.array([0.0, 0.0]), np.array([6.0, 1.0])
    line = scenes.straight_line_coeffs(start, goal)[None]
    xi0 = line + np.random.default_rng(0).normal(0, 0.3, (3, 2, 11))
    xi0[:, :, 0] = start
    b = _problem(start, goal, 40, 8.0, [[0.0, 0.0], [3.0, 0.4]], [[0.3, 0.5], [0.6, 0.4]], xi0)
    g0 = gpu_solve(b, 0)
    o0 = am.solve(b, 0, tol=-1.0)
    np.testing.assert_allclose(g0["residual"], o0["residual"], atol=2e-5)
    assert np.all(np.abs(g0["residual"][:, 0] - 0.3) < 1e-6) or np.all(g0["residual"][:, 0] >= 0.3)
    g1 = gpu_solve(b, 1)
    o1 = am.solve(b, 1, tol=-1.0)
    assert position_error(b, g1["xi"], o1["xi"]).max() <= POS_TOL
    b0 = _problem(start, goal, 33, 8.0, np.zeros((0, 2)), np.zeros((0, 2)), xi0)
    _check(b0, 15)


def test_ragged_and_maximum_horizons():
    rng = np.random.default_rng(1)
    for n_p, n_o in ((32, 3), (33, 5), (64, 7), (256, 256)):
        start, goal = np.array([0.0, 0.0]), np.array([8.0, 6.0])
        T = 0.1 * n_p if n_p > 40 else 6.0
        cen = rng.uniform(0, 8, (n_o, 2))
        ax = rng.uniform(0.2, 0.6, (n_o, 2))
        vel = rng.uniform(-0.3, 0.3, (n_o, 2))
        xi0 = scenes.straight_line_coeffs(start, goal)[None] + rng.normal(0, 0.5, (4, 2, 11))
        _check(_problem(start, goal, n_p, T, cen, ax, xi0, vel=vel), 10)


def test_zero_iterations_returns_initial_projection():
    b = scenes.config2(2, n_scenes=2, inits=4)
    g = gpu_solve(b, 0)
    o = am.solve(b, 0, tol=-1.0)
    np.testing.assert_array_equal(g["xi"], b.xi0.astype(np.float32))
    np.testing.assert_allclose(g["residual"], o["residual"], atol=2e-5, rtol=1e-4)
    assert np.all(g["iters"] == 0) and np.all(g["status"] == 1)


def test_nan_input_is_isolated():
    b = scenes.config2(5, n_scenes=2, inits=4)
    xi0 = b.xi0.copy(); xi0[3, 1, 4] = np.nan
    g = gpu_solve(b, 10, xi0=xi0)
    assert g["status"][3] == 2 and g["stats"].get("error") == -6
    ok = np.arange(b.n_traj) != 3
    ref = gpu_solve(b.subset(np.nonzero(ok)[0]), 10)
    np.testing.assert_array_equal(g["xi"][ok], ref["xi"])


def test_deadline_stops_every_trajectory():
    b = scenes.config2(6, n_scenes=2, inits=4)
    g = gpu_solve(b, 100000, tol=-1.0, timeout_ms=1e-6)
    assert g["stats"].get("error") == -5
    assert np.all(g["status"] == 3) and np.all(g["iters"] < 100000)


def test_launch_shape_graph_replay_and_autotune_do_not_change_results():
    """Uneven batch in one persistent launch: every launch shape with one warp per
    trajectory, a replayed CUDA graph and the autotuned shape give bitwise the same
    trajectories; two or four warps per trajectory add their contraction parts in
    another order, so they agree bitwise among shapes with the same team size and
    with the oracle at the parity tolerance."""
    from paper_2408_10731_b300 import trajbatch as tb
    b = reduced_config4(16, seed=4, inits=3)
    o = am.solve(b, 25, tol=-1.0)
    h = tb.from_batch(b)
    try:
        refs = {}
        for w, bps, team in ((1, 0, 1), (4, 1, 1), (8, 2, 1), (2, 0, 1), (2, 0, 2), (8, 0, 2),
                             (4, 2, 2), (4, 0, 4), (8, 1, 4)):
            h.set_launch_shape(w, bps, team)
            for _ in range(2):  # capture, then replay
                h.solve(25, tol=-1.0)
                out = h.get_trajectories()
                ref = refs.setdefault(team, out)
                np.testing.assert_array_equal(out["xi"], ref["xi"])
                np.testing.assert_array_equal(out["iters"], ref["iters"])
        for team, ref in refs.items():
            assert position_error(b, ref["xi"], o["xi"]).max() <= POS_TOL, team
        choice = h.autotune(5)
        assert 0 <= choice["warps_per_block"] <= 8 and choice["ms"] > 0  # 0: the default shape
        h.solve(25, tol=-1.0)
        np.testing.assert_array_equal(h.get_trajectories()["xi"],
                                      refs[choice["warps_per_trajectory"]]["xi"])
    finally:
        h.close()


@pytest.mark.parametrize("precision,shape", [("fp32", (4, 0, 1)), ("fp32", (8, 0, 2)),
                                             ("mixed", (0, 0, 1))])
def test_checkpoint_resume_continues_bitwise(precision, shape):
    """Solving N iterations, exporting (xi, lambda, u) and resuming for M more gives
    bitwise the iterate of N + M iterations in one solve; traj_set_initial returns
    to fresh starts."""
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.config2(2, n_scenes=8, inits=8)
    h = tb.from_batch(b, precision=precision)
    try:
        h.set_launch_shape(*shape)
        h.solve(40, tol=-1.0)
        direct = h.get_trajectories()
        direct.update(h.get_state())
        h.set_initial(b.traj_problem, b.xi0)
        h.solve(25, tol=-1.0)
        mid = h.get_trajectories()
        mid.update(h.get_state())
        h.set_state(mid["xi"], mid["lam"], mid["u"])
        h.solve(15, tol=-1.0)
        res = h.get_trajectories()
        res.update(h.get_state())
        assert np.all(res["iters"] == 15)
        for key in ("xi", "lam", "u", "residual"):
            np.testing.assert_array_equal(res[key], direct[key], err_msg=key)
        h.set_initial(b.traj_problem, b.xi0)  # fresh start again
        h.solve(40, tol=-1.0)
        np.testing.assert_array_equal(h.get_trajectories()["xi"], direct["xi"])
    finally:
        h.close()


def test_resume_is_refused_in_projection_mode():
    from paper_2408_10731_b300 import trajbatch as tb
    c3 = scenes.config3(0, n_traj=16)
    h = tb.from_batch(c3["batch"], cost_mode="project")
    try:
        z = np.zeros((16, 3, 11), np.float32)
        with pytest.raises(tb.TrajBatchError) as e:
            h.set_state(z, z, z)
        assert e.value.code == -1
    finally:
        h.close()


def test_penalty_continuation_parity():
    """The penalty ladder (reading R10) against the oracle with the same ladder after
    a fixed iteration count that crosses four switches (every 5 iterations, up to
    16 rho), for one and two warps per trajectory; levels = 1 returns bitwise to the
    fixed penalty. (The count is kept short: past ~30 iterations a few
    trajectories of this nonconvex iteration amplify FP32 rounding beyond the
    tolerance with or without the ladder.)"""
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.config2(4, n_scenes=8, inits=8)
    sched = dict(rho_levels=5, rho_growth=2.0, rho_every=5)
    o = am.solve(b, 25, tol=-1.0, **sched)
    plain = gpu_solve(b, 25)
    h = tb.from_batch(b)
    try:
        h.set_rho_schedule(5, 2.0, 5)
        for shape in ((4, 0, 1), (8, 0, 2)):
            h.set_launch_shape(*shape)
            h.solve(25, tol=-1.0)
            g = h.get_trajectories()
            err = position_error(b, g["xi"], o["xi"])
            assert err.max() <= POS_TOL, (shape, err.max())
        h.set_rho_schedule(1)
        h.set_launch_shape(4, 0, 1)
        h.solve(25, tol=-1.0)
        np.testing.assert_array_equal(h.get_trajectories()["xi"], plain["xi"])
    finally:
        h.close()


def test_penalty_continuation_early_stop_and_tensor_core_form():
    """With the stop test on, the ladder's trajectories stop where the oracle's do
    (iteration counts within one, for decisions that are not at the tolerance's
    edge); the tensor-core form follows the same ladder within its error bound."""
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.config2(5, n_scenes=8, inits=8)
    o = am.solve(b, 300, tol=1e-3, rho_levels=6, rho_growth=1.5, rho_every=40)
    for precision in ("fp32", "mixed"):
        h = tb.from_batch(b, precision=precision)
        try:
            h.set_rho_schedule(6, 1.5, 40)
            h.solve(300, tol=1e-3)
            g = h.get_trajectories()
        finally:
            h.close()
        same = np.abs(g["iters"] - o["iters"]) <= 1
        assert same.mean() >= 0.9, (precision, same.mean())
        if precision == "fp32":
            agree = (g["status"] == 0) == (o["iters"] < 300)
            assert agree.mean() >= 0.95


def test_workspace_bounds_parity():
    """Workspace bounds (reading R11) against the oracle: 2D smoothness/tracking with a
    box that cuts through the initialisations (one and two warps per trajectory), and
    3D projection mode with the sampler scene's 20 x 20 x 5 m workspace; removing the
    bounds returns bitwise to the unbounded solve."""
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.config2(6, n_scenes=8, inits=8)
    lo = np.tile([-0.2, -0.2], (b.n_problems, 1)); hi = np.tile([7.5, 7.0], (b.n_problems, 1))
    o = am.solve(b, 20, tol=-1.0, box_lo=lo, box_hi=hi)
    free = gpu_solve(b, 20)
    h = tb.from_batch(b)
    try:
        h.set_workspace(lo, hi)
        for shape in ((4, 0, 1), (8, 0, 2)):
            h.set_launch_shape(*shape)
            h.solve(20, tol=-1.0)
            g = h.get_trajectories()
            assert position_error(b, g["xi"], o["xi"]).max() <= POS_TOL, shape
            np.testing.assert_allclose(g["residual"][:, 0], o["residual"][:, 0], atol=1e-4)
        assert np.abs(g["xi"] - free["xi"]).max() > 1e-3  # the bounds changed the solve
        h.set_workspace(None, None)
        h.set_launch_shape(4, 0, 1)
        h.solve(20, tol=-1.0)
        np.testing.assert_array_equal(h.get_trajectories()["xi"], free["xi"])
    finally:
        h.close()

    c3 = scenes.config3(1, n_traj=24)
    b3 = c3["batch"]
    lo3 = np.array([[0.0, 0.0, 0.0]]); hi3 = np.array([[20.0, 20.0, 5.0]])
    o3 = am.solve(b3, 20, tol=-1.0, cost_mode=1, box_lo=lo3, box_hi=hi3)
    h = tb.from_batch(b3, cost_mode="project")
    try:
        h.set_workspace(lo3, hi3)
        h.solve(20, tol=-1.0)
        g3 = h.get_trajectories()
    finally:
        h.close()
    assert position_error(b3, g3["xi"], o3["xi"]).max() <= POS_TOL


@pytest.mark.parametrize("prec,batch", [("fp32", "uneven"), ("mixed", "uneven"),
                                        ("mixed_split", "config2")])
def test_register_capped_build_is_bitwise_the_default_one(prec, batch):
    """The occupancy build (registers capped so that more warps stay resident) runs the
    same arithmetic as the default build: identical results, bit for bit."""
    from paper_2408_10731_b300 import trajbatch as tb
    b = reduced_config4(12, seed=5, inits=2) if batch == "uneven" else \
        scenes.config2(8, n_scenes=6, inits=4)
    h = tb.from_batch(b, precision=prec)
    try:
        out = {}
        for occ in (0, 1):
            h.set_launch_shape(4, 0, 1, occ)
            h.solve(40, tol=1e-3)
            out[occ] = h.get_trajectories()
            info = h.launch_info()
            assert info["occupancy"] == occ and info["warps_per_block"] == 4
        for k in ("xi", "residual", "iters", "status"):
            np.testing.assert_array_equal(out[0][k], out[1][k])
        with pytest.raises(tb.TrajBatchError):
            h.set_launch_shape(8, 0, 1, 1)  # more warps per block than the capped build takes
    finally:
        h.close()
