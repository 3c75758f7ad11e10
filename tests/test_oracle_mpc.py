"""Pins of the receding-horizon step's oracle (oracle/mpc.py and the start-state
and carried-multiplier inputs of am.solve), against scipy's BPoly, brute-force
equality-constrained QPs and invariants."""
import dataclasses

import numpy as np
import pytest
from scipy.interpolate import BPoly

from oracle import am, mpc
from paper_2408_10731_b300 import scenes
from tests.test_oracle_am import _qp_bruteforce, _single_problem, _tables


@pytest.mark.parametrize("frac", [0.0, 0.01, 0.1, 0.37])
def test_shift_is_the_polynomial_on_the_shifted_window(frac):
    """q(tau') = p(frac + tau'), checked by evaluating both with BPoly (the old one
    extrapolated past tau = 1) at points of the new window."""
    rng = np.random.default_rng(3)
    xi = rng.normal(0, 2.0, (4, 11))
    q = mpc.shift_coeffs(xi, frac)
    t = np.concatenate([rng.uniform(0, 1, 50), [0.0, 1.0]])
    for k in range(4):
        p_old = BPoly(xi[k][:, None], [0.0, 1.0], extrapolate=True)
        p_new = BPoly(q[k][:, None], [0.0, 1.0])
        np.testing.assert_allclose(p_new(t), p_old(frac + t), atol=1e-10 * np.abs(xi).max())
    if frac == 0.0:
        np.testing.assert_allclose(q, xi, atol=1e-12)


def test_shifts_compose():
    rng = np.random.default_rng(4)
    xi = rng.normal(0, 1.0, (3, 2, 11))
    np.testing.assert_allclose(mpc.shift_coeffs(mpc.shift_coeffs(xi, 0.05), 0.12),
                               mpc.shift_coeffs(xi, 0.17), atol=1e-9)


def test_start_state_is_position_velocity_acceleration_at_delta():
    rng = np.random.default_rng(5)
    xi = rng.normal(0, 2.0, (3, 11))
    T, delta = 7.5, 0.6
    st = mpc.start_state(xi, T, delta)
    for a in range(3):
        bp = BPoly(xi[a][:, None], [0.0, T])
        for d in range(3):
            np.testing.assert_allclose(st[d, a], bp.derivative(d)(delta) if d else bp(delta),
                                       rtol=1e-12, atol=1e-12)


def test_repose_moves_each_obstacle_along_its_velocity():
    c = np.array([[1.0, 2.0], [3.0, -1.0]], np.float32)
    v = np.array([[0.5, -0.25], [0.0, 1.0]], np.float32)
    out = mpc.repose_obstacles(c, v, 0.4)
    assert out.dtype == np.float32
    np.testing.assert_array_equal(out, np.array([[1.2, 1.9], [3.0, -0.6]], np.float32))


def test_start_state_boundary_rows_give_the_brute_force_qp_optimum():
    """Obstacle-free, bounds inactive, start velocity and acceleration given: the
    fixed point is the QP optimum with b = (start, v0, a0, goal)."""
    n_p, T = 50, 5.0
    start, goal = np.array([0.0, 1.0]), np.array([4.0, -2.0])
    va = np.array([[[0.8, -0.3], [0.2, 0.5]]])  # [P][2][dim]
    rng = np.random.default_rng(0)
    xi0 = scenes.straight_line_coeffs(start, goal)[None] + rng.normal(0, 0.5, (3, 2, 11))
    b = _single_problem(start, goal, n_p, T, np.zeros((0, 2)), np.zeros((0, 2)), B=3, xi0=xi0,
                        rho=0.05)
    out = am.solve(b, 6000, tol=-1.0, start_va=va)
    P, Pd, Pdd = _tables(n_p, T)
    Q = Pdd.T @ Pdd + P.T @ P
    A = np.stack([P[0], Pd[0], Pdd[0], P[-1]])
    tau = np.linspace(0, 1, n_p)
    for a in range(2):
        xdes = start[a] + (goal[a] - start[a]) * tau
        ref = _qp_bruteforce(Q, -P.T @ xdes, A,
                             np.array([start[a], va[0, 0, a], va[0, 1, a], goal[a]]))
        np.testing.assert_allclose(out["xi"][:, a], np.broadcast_to(ref, (3, 11)), atol=1e-10)
    # and every iterate meets the start state (A xi = b)
    one = am.solve(b, 3, iters_fixed=np.full(3, 3), start_va=va)["xi"]
    np.testing.assert_allclose(one @ Pd[0], np.broadcast_to(va[0, 0], (3, 2)), atol=1e-10)
    np.testing.assert_allclose(one @ Pdd[0], np.broadcast_to(va[0, 1], (3, 2)), atol=1e-10)


def test_one_step_from_carried_multipliers_is_the_brute_force_proximal_qp():
    """Without obstacles and with bounds inactive the projection leaves F xi0 as its
    own target, so the first xi-step from imported multipliers lam0 solves
    min 1/2 xi^T Q xi + q^T xi - lam0^T xi + rho/2 ||F (xi - xi0)||^2  s.t.  A xi = b
    (reading R1 with lambda = lam0): a wrong sign or a dropped lam0 moves it."""
    n_p, T, rho = 40, 6.0, 0.7
    start, goal = np.array([1.0, -1.0]), np.array([5.0, 2.0])
    rng = np.random.default_rng(7)
    xi0 = scenes.straight_line_coeffs(start, goal)[None] + rng.normal(0, 0.3, (2, 2, 11))
    lam0 = rng.normal(0, 0.5, (2, 2, 11))
    b = _single_problem(start, goal, n_p, T, np.zeros((0, 2)), np.zeros((0, 2)), B=2, xi0=xi0,
                        rho=rho)
    out = am.solve(b, 1, iters_fixed=np.full(2, 1), lam0=lam0, want_lambda=True)
    P, Pd, Pdd = _tables(n_p, T)
    FtF = Pd.T @ Pd + Pdd.T @ Pdd
    Q = Pdd.T @ Pdd + P.T @ P + rho * FtF
    A = np.stack([P[0], Pd[0], Pdd[0], P[-1]])
    tau = np.linspace(0, 1, n_p)
    for k in range(2):
        for a in range(2):
            q = -P.T @ (start[a] + (goal[a] - start[a]) * tau) - lam0[k, a] - rho * FtF @ xi0[k, a]
            ref = _qp_bruteforce(Q, q, A, np.array([start[a], 0.0, 0.0, goal[a]]))
            np.testing.assert_allclose(out["xi"][k, a], ref, atol=1e-9)
    # zero carried multipliers are a fresh start, bit for bit
    fresh = am.solve(b, 5, iters_fixed=np.full(2, 5), want_lambda=True)
    zero = am.solve(b, 5, iters_fixed=np.full(2, 5), want_lambda=True, lam0=np.zeros_like(lam0))
    assert np.array_equal(fresh["xi"], zero["xi"]) and np.array_equal(fresh["lam"], zero["lam"])


def test_receding_step_keeps_the_new_boundary_rows_at_every_iterate():
    b = scenes.config2(3, n_scenes=2, inits=3)
    first = am.solve(b, 30, tol=-1.0, want_lambda=True)
    executed = np.array([0, 3])
    moved, va, out = mpc.solve_after_step(b, first["xi"], first["lam"], executed, 0.4, 7)
    P, Pd, Pdd = _tables(100, 10.0)
    xi = out["xi"]
    tp = b.traj_problem
    np.testing.assert_allclose(xi @ P[0], moved.start[tp], atol=1e-10)
    np.testing.assert_allclose(xi @ Pd[0], va[tp, 0], atol=1e-10)
    np.testing.assert_allclose(xi @ Pdd[0], va[tp, 1], atol=1e-10)
    np.testing.assert_allclose(xi @ P[-1], b.goal[tp], atol=1e-10)
    # the new start is where the executed plan was at delta
    for p, e in enumerate(executed):
        np.testing.assert_allclose(moved.start[p], first["xi"][e] @ am.bernstein(101, 10.0)[0][4],
                                   atol=1e-12)
