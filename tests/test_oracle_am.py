"""Pins of the oracle's AM loop (Algorithm 2) by invariants and special cases.

- Obstacle-free, bounds inactive: the iteration's fixed point is the
  brute-force solution of the equality-constrained QP (eq. qp_cost / qp_sol),
  computed here by the null-space method with an independent basis (BPoly).
- Projection mode (eq. projection_cost) without obstacles: the Euclidean
  projection onto {A xi = b}, a textbook closed form.
- A xi = b holds at every iterate.
- A feasible QP optimum is a fixed point: r = 0, lambda = 0, xi unchanged.
- Multiplier sign: a single penetrating obstacle is pushed out and the
  residual goes to zero only with lambda <- lambda - rho F^T r.
- Early stop: the first k >= 1 whose three residuals are all <= tol.
"""
import dataclasses

import numpy as np
import pytest
from scipy.interpolate import BPoly
from scipy.linalg import null_space

from oracle import am
from paper_2408_10731_b300 import scenes


def _tables(n_p, T):
    t = np.linspace(0.0, T, n_p)
    P = np.zeros((n_p, 11)); Pd = np.zeros_like(P); Pdd = np.zeros_like(P)
    for i in range(11):
        c = np.zeros((11, 1)); c[i, 0] = 1.0
        bp = BPoly(c, [0.0, T])
        P[:, i] = bp(t); Pd[:, i] = bp.derivative()(t); Pdd[:, i] = bp.derivative(2)(t)
    return P, Pd, Pdd


def _single_problem(start, goal, n_p, T, centers, axes, vel=None, B=1, xi0=None, vmax=1e6,
                    amax=1e6, rho=1.0):
    dim = len(start)
    centers = np.asarray(centers, float).reshape(-1, dim)
    n_o = centers.shape[0]
    return scenes.Batch(
        dim=dim, n_steps=np.array([n_p], np.int32), duration=np.array([T]),
        start=np.asarray(start, float)[None], goal=np.asarray(goal, float)[None],
        offsets=np.array([0, n_o], np.int32), centers=centers,
        semi_axes=np.asarray(axes, float).reshape(-1, dim),
        velocities=np.zeros((n_o, dim)) if vel is None else np.asarray(vel, float).reshape(-1, dim),
        traj_problem=np.zeros(B, np.int32),
        xi0=np.zeros((B, dim, 11)) if xi0 is None else np.asarray(xi0, float),
        vmax=vmax, amax=amax, rho=rho)


def _qp_bruteforce(Q, q, A, b):
    xp = np.linalg.lstsq(A, b, rcond=None)[0]
    N = null_space(A)
    z = -np.linalg.solve(N.T @ Q @ N, N.T @ (Q @ xp + q))
    return xp + N @ z


@pytest.mark.parametrize("n_p,T", [(50, 5.0), (1000, 10.0)])
def test_obstacle_free_fixed_point_is_the_qp_optimum(n_p, T):
    """The obstacle-free iteration converges to the QP optimum found by a
    null-space solve; n_p = 1000 is Paper I's long horizon."""
    start, goal = np.array([0.0, 1.0]), np.array([4.0, -2.0])
    rng = np.random.default_rng(0)
    xi0 = scenes.straight_line_coeffs(start, goal)[None] + rng.normal(0, 0.5, (3, 2, 11))
    b = _single_problem(start, goal, n_p, T, np.zeros((0, 2)), np.zeros((0, 2)), B=3, xi0=xi0,
                        rho=0.05)
    out = am.solve(b, 6000, tol=-1.0)
    P, Pd, Pdd = _tables(n_p, T)
    Q = Pdd.T @ Pdd + P.T @ P
    A = np.stack([P[0], Pd[0], Pdd[0], P[-1]])
    tau = np.linspace(0, 1, n_p)
    for a in range(2):
        xdes = start[a] + (goal[a] - start[a]) * tau
        ref = _qp_bruteforce(Q, -P.T @ xdes, A, np.array([start[a], 0, 0, goal[a]]))
        np.testing.assert_allclose(out["xi"][:, a], np.broadcast_to(ref, (3, 11)), atol=1e-10)
    np.testing.assert_allclose(out["residual"], 0.0, atol=1e-12)


def test_projection_mode_without_obstacles_is_affine_projection():
    n_p, T = 60, 6.0
    start, goal = np.array([1.0, 2.0, 0.5]), np.array([5.0, -1.0, 2.0])
    rng = np.random.default_rng(1)
    xi0 = rng.normal(0, 1.0, (4, 3, 11))
    b = _single_problem(start, goal, n_p, T, np.zeros((0, 3)), np.zeros((0, 3)), B=4, xi0=xi0,
                        rho=0.01)
    # the proximal iteration converges to the projection; run it to its fixed point
    out = am.solve(b, 20000, tol=-1.0, cost_mode=1)
    P, Pd, Pdd = _tables(n_p, T)
    A = np.stack([P[0], Pd[0], Pdd[0], P[-1]])
    for a in range(3):
        bb = np.array([start[a], 0, 0, goal[a]])
        x = xi0[:, a]
        ref = x - (A.T @ np.linalg.solve(A @ A.T, A @ x.T - bb[:, None])).T
        np.testing.assert_allclose(out["xi"][:, a], ref, atol=1e-11)


def test_boundary_equalities_hold_at_every_iterate():
    b = scenes.config2(3, n_scenes=2, inits=3)
    P, Pd, Pdd = _tables(100, 10.0)
    for k in (1, 4, 17):
        out = am.solve(b, k, iters_fixed=np.full(b.n_traj, k))
        xi = out["xi"]
        np.testing.assert_allclose(xi @ P[0], b.start[b.traj_problem], atol=1e-10)
        np.testing.assert_allclose(xi @ Pd[0], 0.0, atol=1e-10)
        np.testing.assert_allclose(xi @ Pdd[0], 0.0, atol=1e-10)
        np.testing.assert_allclose(xi @ P[-1], b.goal[b.traj_problem], atol=1e-10)


def test_feasible_qp_optimum_is_a_fixed_point():
    n_p, T = 50, 10.0
    start, goal = np.array([0.0, 0.0]), np.array([5.0, 3.0])
    P, Pd, Pdd = _tables(n_p, T)
    Q = Pdd.T @ Pdd + P.T @ P
    A = np.stack([P[0], Pd[0], Pdd[0], P[-1]])
    tau = np.linspace(0, 1, n_p)
    xi_star = np.stack([_qp_bruteforce(Q, -P.T @ (start[a] + (goal[a] - start[a]) * tau), A,
                                       np.array([start[a], 0, 0, goal[a]])) for a in range(2)])
    # obstacles well away from the optimum; bounds satisfied (1.5 m/s, 2 m/s^2)
    centers = [[0.0, 4.0], [4.0, -2.0], [1.0, 3.0]]
    b = _single_problem(start, goal, n_p, T, centers, [[0.5, 0.4]] * 3, B=1,
                        xi0=xi_star[None], vmax=1.5, amax=2.0)
    out = am.solve(b, 25, tol=-1.0, want_lambda=True)
    np.testing.assert_allclose(out["xi"][0], xi_star, atol=1e-10)
    np.testing.assert_allclose(out["lam"], 0.0, atol=1e-10)
    np.testing.assert_allclose(out["residual"], 0.0, atol=1e-12)


def test_multiplier_sign_pushes_out_of_a_single_obstacle():
    n_p, T = 50, 10.0
    start, goal = np.array([0.0, 0.0]), np.array([6.0, 0.0])
    line = scenes.straight_line_coeffs(start, goal)[None]
    # one circle sitting on the straight line, slightly off-axis so the push is +y
    b = _single_problem(start, goal, n_p, T, [[3.0, -0.05]], [[0.5, 0.5]], B=1, xi0=line,
                        vmax=1.5, amax=2.0)
    out = am.solve(b, 400, tol=-1.0, want_hist=True)
    h = out["hist"][0, :, 0]
    assert h[0] > 0.4 and h[1] > 0.0
    assert h[50] < 0.5 * h[1]
    assert h[-1] < 1e-3
    # every iterate after the first moves the midpoint further from the centre (+y)
    ys = []
    for k in (1, 2, 5, 20):
        xi = am.solve(b, k, iters_fixed=[k])["xi"][0]
        P, _, _ = _tables(n_p, T)
        ys.append((P @ xi[1])[n_p // 2])
    assert all(np.diff(ys) > 0), ys


def test_early_stop_is_first_iteration_under_tolerance():
    b = scenes.config2(0, n_scenes=2, inits=4)
    tol = 1e-3
    out = am.solve(b, 300, tol=tol, want_hist=True)
    for k in range(b.n_traj):
        h = out["hist"][k]
        under = np.nonzero(np.all(h[1:] <= tol, axis=1))[0]
        expect = (under[0] + 1) if under.size else 300
        assert out["iters"][k] == expect
        np.testing.assert_array_equal(out["residual"][k], h[out["iters"][k]])


def test_penalty_continuation_plumbing_and_fixed_point():
    """Reading R10: a ladder with growth 1, or whose first switch lies past the last
    iteration, is bitwise the fixed-penalty run; a real ladder changes the iterates;
    and without obstacles the continued iteration still converges to the
    equality-constrained QP optimum (a wrong K inverse or rho at a level would move
    the fixed point)."""
    b = scenes.config2(3, n_scenes=2, inits=3)
    base = am.solve(b, 60, tol=-1.0, want_lambda=True)
    same = am.solve(b, 60, tol=-1.0, want_lambda=True, rho_levels=10, rho_growth=1.0, rho_every=5)
    np.testing.assert_array_equal(base["xi"], same["xi"])
    np.testing.assert_array_equal(base["lam"], same["lam"])
    late = am.solve(b, 60, tol=-1.0, rho_levels=10, rho_growth=2.0, rho_every=100)
    np.testing.assert_array_equal(base["xi"], late["xi"])
    switched = am.solve(b, 60, tol=-1.0, rho_levels=3, rho_growth=2.0, rho_every=20)
    assert np.abs(switched["xi"] - base["xi"]).max() > 1e-6

    n_p, T = 50, 5.0
    start, goal = np.array([0.0, 1.0]), np.array([4.0, -2.0])
    rng = np.random.default_rng(0)
    xi0 = scenes.straight_line_coeffs(start, goal)[None] + rng.normal(0, 0.5, (3, 2, 11))
    bq = _single_problem(start, goal, n_p, T, np.zeros((0, 2)), np.zeros((0, 2)), B=3, xi0=xi0,
                         rho=0.05)
    out = am.solve(bq, 6000, tol=-1.0, rho_levels=4, rho_growth=2.0, rho_every=1000)
    P, Pd, Pdd = _tables(n_p, T)
    Q = Pdd.T @ Pdd + P.T @ P
    A = np.stack([P[0], Pd[0], Pdd[0], P[-1]])
    tau = np.linspace(0, 1, n_p)
    for a in range(2):
        xdes = start[a] + (goal[a] - start[a]) * tau
        ref = _qp_bruteforce(Q, -P.T @ xdes, A, np.array([start[a], 0, 0, goal[a]]))
        np.testing.assert_allclose(out["xi"][:, a], np.broadcast_to(ref, (3, 11)), atol=1e-10)


def test_workspace_bounds_inactive_fixed_point_and_active_feasibility():
    """Reading R11 (PRIEST's G xi <= tau with slack, G = [-P; P] per axis).
    Inactive box: the obstacle-free fixed point is still the equality-constrained QP
    optimum; this fails if G^T G = 2 P^T P were missing from the KKT matrix while the
    rows enter the multiplier update (or the reverse). Active box (projection mode,
    samples leaving it): the iteration converges to a point whose grid positions
    satisfy the bounds, with some of them on a bound, and the rows' residual folds
    into the obstacle column."""
    n_p, T = 50, 5.0
    start, goal = np.array([0.0, 1.0]), np.array([4.0, -2.0])
    rng = np.random.default_rng(0)
    xi0 = scenes.straight_line_coeffs(start, goal)[None] + rng.normal(0, 0.5, (3, 2, 11))
    b = _single_problem(start, goal, n_p, T, np.zeros((0, 2)), np.zeros((0, 2)), B=3, xi0=xi0,
                        rho=0.05)
    big_lo, big_hi = np.array([[-50.0, -50.0]]), np.array([[50.0, 50.0]])
    out = am.solve(b, 6000, tol=-1.0, box_lo=big_lo, box_hi=big_hi)
    P, Pd, Pdd = _tables(n_p, T)
    Q = Pdd.T @ Pdd + P.T @ P
    A = np.stack([P[0], Pd[0], Pdd[0], P[-1]])
    tau = np.linspace(0, 1, n_p)
    for a in range(2):
        xdes = start[a] + (goal[a] - start[a]) * tau
        ref = _qp_bruteforce(Q, -P.T @ xdes, A, np.array([start[a], 0, 0, goal[a]]))
        np.testing.assert_allclose(out["xi"][:, a], np.broadcast_to(ref, (3, 11)), atol=1e-10)

    n_p, T = 40, 4.0
    start, goal = np.array([0.0, 0.0]), np.array([3.0, 1.0])
    lo, hi = np.array([-0.5, -0.3]), np.array([3.2, 1.2])
    xi0 = scenes.straight_line_coeffs(start, goal)[None] + np.random.default_rng(7).normal(0, 1.0, (2, 2, 11))
    b = _single_problem(start, goal, n_p, T, np.zeros((0, 2)), np.zeros((0, 2)), B=2, xi0=xi0,
                        rho=0.05)
    h = am.solve(b, 3000, tol=-1.0, cost_mode=1, box_lo=lo[None], box_hi=hi[None], want_hist=True)
    free = am.solve(b, 3000, tol=-1.0, cost_mode=1)
    P, _, _ = _tables(n_p, T)
    pos = np.einsum("ti,kai->kta", P, h["xi"])
    assert np.all(pos >= lo - 1e-9) and np.all(pos <= hi + 1e-9)
    on_bound = np.minimum(np.abs(pos - lo), np.abs(pos - hi)).min()
    assert on_bound < 1e-9
    assert np.all(h["residual"] < 1e-12)
    pos_free = np.einsum("ti,kai->kta", P, free["xi"])
    assert np.any(pos_free > hi + 1e-3) or np.any(pos_free < lo - 1e-3)  # the box mattered
    assert h["hist"][:, 0, 0].max() > 1e-3  # the initial projection saw the violation


@pytest.mark.parametrize("dim,moving", [(2, True), (2, False), (3, True)])
def test_long_horizon_scenes_follow_their_recipe(dim, moving):
    """Long-horizon inputs: n_p grid points over T = 0.01 n_p, the goal within the
    rest-to-rest reach vmax (T - vmax / amax), no obstacle covering the start at
    t = 0 or the goal at t = T, speeds in [0, 1] m/s (zero when static)."""
    b = scenes.long_horizon(seed=2, n_scenes=6, inits=3, n_steps=[257, 300, 500, 640, 1000, 1000],
                            dim=dim, moving=moving)
    assert b.n_traj == 18 and b.xi0.shape == (18, dim, 11)
    np.testing.assert_allclose(b.duration, 0.01 * b.n_steps)
    reach = np.linalg.norm(b.goal - b.start, axis=1)
    assert np.all(reach <= b.vmax * (b.duration - b.vmax / b.amax))
    for p in range(b.n_problems):
        sl = slice(b.offsets[p], b.offsets[p + 1])
        c, a, v = b.centers[sl], b.semi_axes[sl], b.velocities[sl]
        assert c.shape == (10, dim) and np.all((a >= 0.2) & (a <= 0.8))
        speed = np.linalg.norm(v, axis=1)
        assert np.all(speed <= 1.0 + 1e-6) and (moving or np.all(speed == 0))
        assert np.all((((b.start[p] - c) / a) ** 2).sum(1) > 1.0)
        assert np.all((((b.goal[p] - (c + v * b.duration[p])) / a) ** 2).sum(1) > 1.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_first_iterations_equal_brute_force_composition(dim):
    """Two full iterations on a small problem with moving obstacles and active bounds,
    rebuilt step by step outside the oracle's loop: the targets g from the projection
    functions (pinned against dense grids above) applied to each iterate, the
    xi-steps as brute-force equality-constrained QPs (null-space method, BPoly
    tables, a literal stacked F per axis), and the multiplier update
    lambda <- lambda - rho F^T (F xi - g). A dropped term, a wrong sign, an index off
    by one or a step out of Algorithm 2's order moves the result."""
    n_p, T, rho, vmax, amax = 20, 4.0, 0.8, 1.2, 1.5
    rng = np.random.default_rng(21 + dim)
    start = rng.uniform(-1, 1, dim)
    goal = start + rng.uniform(3, 5, dim)
    n_o = 3
    centers = start + (goal - start) * rng.uniform(0.3, 0.7, (n_o, 1)) + rng.normal(0, 0.2, (n_o, dim))
    axes = rng.uniform(0.4, 0.8, (n_o, dim))
    vel = rng.normal(0, 0.3, (n_o, dim))
    xi0 = scenes.straight_line_coeffs(start, goal)[None] + rng.normal(0, 0.4, (2, dim, 11))
    b = _single_problem(start, goal, n_p, T, centers, axes, vel=vel, B=2, xi0=xi0, vmax=vmax,
                        amax=amax, rho=rho)
    P, Pd, Pdd = _tables(n_p, T)
    t = np.linspace(0.0, T, n_p)
    F = np.vstack([P] * n_o + [Pd, Pdd])                  # one axis's stacked rows
    Q = Pdd.T @ Pdd + P.T @ P
    A = np.stack([P[0], Pd[0], Pdd[0], P[-1]])
    tau = np.linspace(0, 1, n_p)

    def targets(xi):  # g [dim][rows] for coefficients xi [dim][11]
        pos, v, a = xi @ P.T, xi @ Pd.T, xi @ Pdd.T
        g = np.zeros((dim, F.shape[0]))
        for j in range(n_o):
            o = centers[j][:, None] + vel[j][:, None] * t[None]
            for k in range(n_p):
                g[:, j * n_p + k] = o[:, k] + am.project_obstacle(pos[:, k] - o[:, k], axes[j])
        for k in range(n_p):
            g[:, n_o * n_p + k] = am.project_bound(v[:, k], vmax)
            g[:, (n_o + 1) * n_p + k] = am.project_bound(a[:, k], amax)
        return g

    for kk in range(2):
        xi, lam = xi0[kk].copy(), np.zeros((dim, 11))
        g = targets(xi)
        ref = []
        for it in range(2):
            new = np.zeros_like(xi)
            for ax in range(dim):
                q = -P.T @ (start[ax] + (goal[ax] - start[ax]) * tau)
                new[ax] = _qp_bruteforce(Q + rho * F.T @ F, q - lam[ax] - rho * F.T @ g[ax], A,
                                         np.array([start[ax], 0.0, 0.0, goal[ax]]))
            xi = new
            g = targets(xi)
            lam = lam - rho * np.stack([F.T @ (F @ xi[ax] - g[ax]) for ax in range(dim)])
            ref.append((xi.copy(), lam.copy()))
        for it in (1, 2):
            out = am.solve(b, it, iters_fixed=np.full(2, it), want_lambda=True)
            np.testing.assert_allclose(out["xi"][kk], ref[it - 1][0], atol=1e-9, rtol=0)
            np.testing.assert_allclose(out["lam"][kk], ref[it - 1][1], atol=1e-8, rtol=0)
