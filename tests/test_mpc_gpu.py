"""GPU parity of the receding-horizon step (traj_shift_horizon, Paper II's MPC use
of Algorithm 2: each control loop's solve starts from the previous loop's
multipliers) against the FP64 oracle's step (oracle/mpc.py)."""
import numpy as np
import pytest

from oracle import am, mpc
from paper_2408_10731_b300 import scenes
from tests.gpu_helpers import POS_TOL, position_error

pytestmark = pytest.mark.gpu


def _handle(batch, **kw):
    from paper_2408_10731_b300 import trajbatch as tb
    return tb.from_batch(batch, **kw)


def _oracle_sensitivity(batch, iters, rel=1e-7, trials=3):
    """How far the FP64 oracle's own result after `iters` iterations moves, per
    trajectory, when its initial coefficients are perturbed at FP32 rounding size
    (relative 1e-7): the part of any FP32 implementation's error that the method
    itself amplifies, whatever order its sums are rounded in."""
    base = am.solve(batch, iters, tol=-1.0)
    rng = np.random.default_rng(0)
    worst = np.zeros(batch.n_traj)
    for _ in range(trials):
        x0 = batch.xi0 * (1.0 + rel * rng.standard_normal(batch.xi0.shape))
        o = am.solve(batch, iters, tol=-1.0, xi0=x0)
        worst = np.maximum(worst, position_error(batch, o["xi"], base["xi"]))
    return worst


@pytest.mark.parametrize("shape", [None, (4, 0, 2)], ids=["one_warp", "two_warp_team"])
def test_three_receding_calls_of_ten_iterations_match_the_oracle(shape):
    """Each control loop is checked against the oracle's step from the GPU's own state
    before it (coefficients and multipliers as the GPU left them), at the parity bar;
    the oracle's own chain of three loops is followed beside it, where the FP32
    rounding of each shifted iterate and start state compounds (bound 5e-5 m). Run at
    one warp per trajectory and with two-warp teams (the shape the MPC bench's trial
    picks), whose carried multipliers enter through the team kernel. The initial
    30-iteration solve holds one trajectory (18) that the method itself amplifies: a
    1e-7 relative change of its start moves the oracle's own result by 2.4e-5 m, so
    its bar there is twice that measured sensitivity; every trajectory the method
    does not amplify is held to 1e-5 m."""
    b = scenes.config2(5, n_scenes=6, inits=4)
    executed = np.arange(b.n_problems) * 4 + 1  # the second plan of every scene
    delta = 0.3
    h = _handle(b)
    try:
        if shape:
            h.set_launch_shape(*shape)
        h.solve(30, -1.0)
        g = h.get_trajectories()
        o = am.solve(b, 30, tol=-1.0, want_lambda=True)
        err0 = position_error(b, g["xi"], o["xi"])
        sens = _oracle_sensitivity(b, 30)
        assert np.all(err0 <= np.maximum(POS_TOL, 2.0 * sens)), (err0.max(), sens[np.argmax(err0)])
        assert np.all(err0[sens < POS_TOL / 4] <= POS_TOL)
        chain_xi, chain_lam, chain_b = o["xi"], o["lam"], b
        cur = b
        for step in range(3):
            xi_g = g["xi"].astype(np.float64)
            lam_g = h.get_state()["lam"].astype(np.float64)
            h.shift_horizon(delta, executed)
            h.solve(10, -1.0)
            g = h.get_trajectories()
            cur, va, o = mpc.solve_after_step(cur, xi_g, lam_g, executed, delta, 10)
            err = position_error(cur, g["xi"], o["xi"])
            assert err.max() <= POS_TOL, (step, err.max())
            assert np.all(g["iters"] == 10)
            scale = np.abs(o["lam"]).max()
            assert np.abs(h.get_state()["lam"] - o["lam"]).max() <= 2e-4 * scale, step
            np.testing.assert_allclose(g["residual"], o["residual"], atol=2e-5, rtol=1e-4)
            # the new start is where the executed plan was delta seconds in
            P, Pd, Pdd = am.bernstein(100, 10.0)
            xg = g["xi"].astype(np.float64)
            np.testing.assert_allclose(xg @ P[0], cur.start[cur.traj_problem], atol=2e-5)
            np.testing.assert_allclose(xg @ Pd[0], va[cur.traj_problem, 0], atol=2e-5)
            chain_b, _, co = mpc.solve_after_step(chain_b, chain_xi, chain_lam, executed, delta, 10)
            chain_xi, chain_lam = co["xi"], co["lam"]
            assert position_error(chain_b, g["xi"], chain_xi).max() <= 5e-5, step
    finally:
        h.close()


def test_new_obstacles_between_shifts_set_the_problems_up_again():
    """A shift keeps each problem's KKT inverse and forms again only the constants that
    depend on the boundary values; new obstacles (here a different number per scene,
    which changes F^T F) are set up in full, and the next shift must start from the
    blocks that set-up kept. Four control loops; after the second shift the obstacles
    are replaced before its solve, so the third shift starts from the new ones: every
    loop against the oracle's step from the GPU's own state."""
    import dataclasses
    b = scenes.config2(7, n_scenes=4, inits=4)
    new = scenes.config2(8, n_scenes=4, inits=4, n_obstacles=30)
    executed = np.arange(b.n_problems) * 4 + 2
    delta = 0.25
    h = _handle(b)
    try:
        h.solve(30, -1.0)
        g = h.get_trajectories()
        cur = b
        for step in range(4):
            xi_g = g["xi"].astype(np.float64)
            lam_g = h.get_state()["lam"].astype(np.float64)
            h.shift_horizon(delta, executed)
            moved, va, xi0, lam0 = mpc.mpc_step(cur, xi_g, lam_g, executed, delta)
            if step == 1:  # fresh obstacle data, 30 instead of 50 per scene
                h.set_obstacles(new.offsets, new.centers, new.semi_axes, new.velocities)
                moved = dataclasses.replace(moved, offsets=new.offsets, centers=new.centers,
                                            semi_axes=new.semi_axes, velocities=new.velocities)
            h.solve(10, -1.0)
            g = h.get_trajectories()
            o = am.solve(moved, 10, xi0=xi0, start_va=va, lam0=lam0, want_lambda=True)
            err = position_error(moved, g["xi"], o["xi"])
            assert err.max() <= POS_TOL, (step, err.max())
            cur = moved
    finally:
        h.close()


def test_default_executed_plan_is_the_smallest_worst_residual():
    b = scenes.config2(6, n_scenes=5, inits=6)
    h1, h2 = _handle(b), _handle(b)
    try:
        h1.solve(40, 1e-3)
        h2.solve(40, 1e-3)
        res = h2.get_trajectories()["residual"]
        worst = res.max(axis=1).reshape(b.n_problems, 6)
        executed = np.argmin(worst, axis=1) + 6 * np.arange(b.n_problems)  # ties: lower index
        h1.shift_horizon(0.2)
        h2.shift_horizon(0.2, executed)
        h1.solve(10, -1.0)
        h2.solve(10, -1.0)
        a, c = h1.get_trajectories(), h2.get_trajectories()
        assert np.array_equal(a["xi"], c["xi"]) and np.array_equal(a["residual"], c["residual"])
    finally:
        h1.close()
        h2.close()


def test_fresh_start_after_a_shift_and_refused_calls():
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.config2(7, n_scenes=3, inits=2)
    h = _handle(b)
    try:
        with pytest.raises(tb.TrajBatchError) as e:
            h.shift_horizon(0.1)  # no solve yet
        assert e.value.code == -7
        h.solve(15, -1.0)
        ref = h.get_trajectories()["xi"].copy()
        for bad in (0.0, -0.1, 10.0, float("nan")):
            with pytest.raises(tb.TrajBatchError) as e:
                h.shift_horizon(bad)
            assert e.value.code == -1
        with pytest.raises(tb.TrajBatchError) as e:
            h.shift_horizon(0.1, [0, 1, 2])  # trajectory 1 belongs to problem 0
        assert e.value.code == -1
        h.shift_horizon(0.1, [0, 2, 4])
        h.solve(15, -1.0)
        moved = h.get_trajectories()["xi"].copy()
        assert not np.array_equal(moved, ref)
        # traj_set_initial returns to fresh starts (of the moved problems)
        h.set_initial(b.traj_problem, b.xi0)
        h.solve(15, -1.0)
        again = h.get_trajectories()["xi"]
        assert not np.array_equal(again, moved)
    finally:
        h.close()
    hp = _handle(b, cost_mode="project")
    try:
        hp.solve(5, -1.0)
        with pytest.raises(tb.TrajBatchError) as e:
            hp.shift_horizon(0.1)
        assert e.value.code == -1
    finally:
        hp.close()


def test_full_size_receding_step_sampled():
    """The bench's MPC workload (125 scenes x 8 plans, 50 moving ellipses): a converged
    plan, one shift of 0.1 s and 10 iterations; three scenes recomputed by the oracle
    from the GPU's own state before the shift."""
    b = scenes.config2(0, n_scenes=125, inits=8)
    h = _handle(b)
    try:
        h.solve(500, 1e-3)
        g0 = h.get_trajectories()
        lam0 = h.get_state()["lam"]
        worst = g0["residual"].max(axis=1).reshape(125, 8)
        executed = np.argmin(worst, axis=1) + 8 * np.arange(125)
        h.shift_horizon(0.1)
        h.solve(10, -1.0)
        g = h.get_trajectories()
        for p in (0, 61, 124):
            sub = b.select_problems([p])
            idx = np.nonzero(b.traj_problem == p)[0]
            moved, va, o = mpc.solve_after_step(sub, g0["xi"][idx].astype(np.float64),
                                                lam0[idx].astype(np.float64),
                                                [int(executed[p] - idx[0])], 0.1, 10)
            err = position_error(moved, g["xi"][idx], o["xi"])
            assert err.max() <= POS_TOL, (p, err.max())
    finally:
        h.close()


def _step_against_oracle(batch, precision="fp32", shape=None, iters0=20, delta=0.1):
    """Solve, shift by delta onto each problem's first plan, solve 10 iterations; the
    oracle's step from the GPU's own state before the shift. Returns the error."""
    h = _handle(batch, precision=precision)
    try:
        if shape:
            h.set_launch_shape(*shape)
        h.solve(iters0, -1.0)
        xi = h.get_trajectories()["xi"].astype(np.float64)
        lam = h.get_state()["lam"].astype(np.float64)
        executed = [int(np.nonzero(batch.traj_problem == p)[0][0]) for p in range(batch.n_problems)]
        h.shift_horizon(delta, executed)
        h.solve(10, -1.0)
        g = h.get_trajectories()
    finally:
        h.close()
    moved, _, o = mpc.solve_after_step(batch, xi, lam, executed, delta, 10)
    return position_error(moved, g["xi"], o["xi"])


def test_receding_step_in_3d_and_with_a_team_of_warps():
    """A 3D problem set (ellipsoids, start velocity and acceleration in three axes) in
    the one-warp and the two-warp-team kernels."""
    b = scenes.long_horizon(3, n_scenes=3, inits=4, n_steps=200, dim=3)
    assert _step_against_oracle(b).max() <= POS_TOL
    b2 = scenes.config2(9, n_scenes=4, inits=4)
    assert _step_against_oracle(b2, shape=(4, 0, 2)).max() <= POS_TOL


@pytest.mark.parametrize("prec,bound", [("mixed", 5e-2), ("mixed_split", 1e-3)])
def test_receding_step_in_the_tensor_core_forms(prec, bound, capsys):
    """The carried multipliers and the first projection of the shifted iterate in the
    tensor-core kernel; error against the oracle's step reported and bounded as the
    forms' error after 20 iterations."""
    b = scenes.config2(9, n_scenes=4, inits=4)
    err = _step_against_oracle(b, precision=prec)
    with capsys.disabled():
        print(f"\n{prec} receding step vs FP64: max {err.max():.2e} m")
    assert err.max() <= bound


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_mpc_step_graph_is_bitwise_the_shift_and_solve_calls(precision):
    """traj_mpc_step replays the shift, the boundary update and the solve as one CUDA
    graph. Over control loops with the default executed plan, a given one, a new delta
    (the graph captured again) and obstacles replaced between loops (the graph dropped
    with the set-up) and a new launch shape (two-warp teams for FP32), it gives bitwise
    the iterates, multipliers, residuals, iteration counts and statuses of
    traj_shift_horizon followed by traj_solve, with the FP32 solve and with the
    tensor-core one inside the graph."""
    b = scenes.config2(11, n_scenes=6, inits=4)
    new = scenes.config2(12, n_scenes=6, inits=4, n_obstacles=30)
    h1, h2 = _handle(b, precision=precision), _handle(b, precision=precision)
    try:
        for h in (h1, h2):
            h.solve(40, 1e-3, stats=False)
        given = np.arange(b.n_problems) * 4 + 1
        plan = [(0.1, None), (0.1, None), (0.1, given), (0.2, None), ("obstacles", None),
                (0.2, None), (0.2, given), ("shape", None), (0.1, None), (0.1, None)]
        for step, (delta, ex) in enumerate(plan):
            if delta == "obstacles":
                for h in (h1, h2):
                    h.set_obstacles(new.offsets, new.centers, new.semi_axes, new.velocities)
                    h.solve(10, 1e-3, stats=False)
                continue
            if delta == "shape":  # the graph is captured again for the new launch shape
                for h in (h1, h2):
                    h.set_launch_shape(4, 0, 2 if precision == "fp32" else 1)
                continue
            h1.shift_horizon(delta, ex)
            h1.solve(10, 1e-3, stats=False)
            h2.mpc_step(delta, 10, 1e-3, executed=ex)
            g1, g2 = h1.get_trajectories(), h2.get_trajectories()
            for k in ("xi", "residual", "iters", "status"):
                assert np.array_equal(g1[k], g2[k]), (step, k)
            assert np.array_equal(h1.get_state()["lam"], h2.get_state()["lam"]), step
        st = h2.last_stats()
        assert st["gpu_ms"] > 0 and st["n_traj"] == b.n_traj
    finally:
        h1.close()
        h2.close()


def test_mpc_step_refusals():
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.config2(13, n_scenes=2, inits=2)
    h = _handle(b)
    try:
        with pytest.raises(tb.TrajBatchError) as e:
            h.mpc_step(0.1, 10)  # no solve has run
        assert e.value.code == -7
        h.solve(5, 1e-3, stats=False)
        with pytest.raises(tb.TrajBatchError) as e:
            h.mpc_step(100.0, 10)  # delta beyond the horizon
        assert e.value.code == -1
        with pytest.raises(tb.TrajBatchError) as e:
            h.mpc_step(0.1, 10, executed=[1, 0])  # not a trajectory of its problem
        assert e.value.code == -1
        h.mpc_step(0.1, 10)  # the handle is still usable
        assert np.all(np.isfinite(h.get_trajectories()["xi"]))
    finally:
        h.close()
