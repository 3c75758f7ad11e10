"""Pins of the footprint-and-heading oracle (Paper II, Algorithm 2 with the
heading variables)."""
import numpy as np
import pytest

from oracle import am, footprint as fp
from paper_2408_10731_b300 import scenes
from tests.test_oracle_am import _qp_bruteforce, _tables


def _from_batch(b, p=0, offsets=(0.0,), r_circle=0.0, psi0=0.0, psif=0.0, rho_psi=1.0):
    c, a, v = b.obstacles(p)
    return fp.FPProblem(n_p=int(b.n_steps[p]), T=float(b.duration[p]), start=b.start[p],
                        goal=b.goal[p], psi0=psi0, psif=psif, centers=np.asarray(c, float),
                        semi_axes=np.asarray(a, float), velocities=np.asarray(v, float),
                        offsets=np.asarray(offsets, float), r_circle=r_circle, vmax=b.vmax,
                        amax=b.amax, rho=b.rho, rho_psi=rho_psi)


def test_one_circle_at_the_centre_is_the_single_agent_method():
    """With one circle at offset 0 and radius 0 the collision, speed and
    acceleration rows of each half are those of the single-agent F, and the copy
    rows touch only the slack coefficients: x and y must follow am.solve."""
    b = scenes.config2(4, n_scenes=1, inits=4)
    prob = _from_batch(b, psi0=0.3, psif=-0.2)
    xi0 = np.concatenate([b.xi0, np.zeros((4, 1, 11))], 1)
    xi0[:, 2] = np.linspace(0.3, -0.2, 11)
    out = fp.solve(prob, xi0, 30)
    ref = am.solve(b, 30, tol=-1.0)
    np.testing.assert_allclose(out["xi"][:, 0], ref["xi"][:, 0], atol=1e-9)
    np.testing.assert_allclose(out["xi"][:, 2], ref["xi"][:, 1], atol=1e-9)
    np.testing.assert_allclose(out["residual"][:, 0], ref["residual"][:, 0], atol=1e-9)


def test_obstacle_free_fixed_point_with_a_constant_heading():
    """No obstacles, inactive bounds, heading theta at both ends and initially:
    the fixed point is the brute-force QP optimum of x and y (null-space method
    on BPoly tables) with heading theta and copies cos theta, sin theta; from a
    noisy initial heading the copies still become consistent with psi."""
    n_p, T, th = 40, 6.0, 0.7
    start, goal = np.array([0.0, 1.0]), np.array([5.0, 4.0])
    prob = fp.FPProblem(n_p=n_p, T=T, start=start, goal=goal, psi0=th, psif=th,
                        centers=np.zeros((0, 2)), semi_axes=np.zeros((0, 2)),
                        velocities=np.zeros((0, 2)), offsets=np.array([-0.3, 0.0, 0.3]),
                        r_circle=0.2, vmax=1e3, amax=1e3, rho=0.5, rho_psi=0.5)
    rng = np.random.default_rng(0)
    xi0 = np.zeros((3, 3, 11))
    for a in range(2):
        xi0[:, a] = start[a] + (goal[a] - start[a]) * np.arange(11) / 10 + rng.normal(0, 0.3, (3, 11))
    xi0[:, 2] = th
    out = fp.solve(prob, xi0, 3000)
    P, Pd, Pdd = _tables(n_p, T)
    A = np.stack([P[0], Pd[0], Pdd[0], P[-1]])
    tau = np.linspace(0, 1, n_p)
    for a, col in ((0, 0), (1, 2)):
        xdes = start[a] + (goal[a] - start[a]) * tau
        ref = _qp_bruteforce(Pdd.T @ Pdd + P.T @ P, -P.T @ xdes, A,
                             np.array([start[a], 0, 0, goal[a]]))
        np.testing.assert_allclose(out["xi"][:, col], np.broadcast_to(ref, (3, 11)), atol=1e-8)
    np.testing.assert_allclose(out["xi"][:, 1], np.cos(th), atol=1e-10)
    np.testing.assert_allclose(out["xi"][:, 3], np.sin(th), atol=1e-10)
    np.testing.assert_allclose(out["xi_psi"], th, atol=1e-10)
    assert out["residual"].max() < 1e-8
    xi0[:, 2] += rng.normal(0, 0.2, (3, 11))
    xi0[:, 2, 0] = xi0[:, 2, -1] = th
    out = fp.solve(prob, xi0, 1000)
    assert out["residual"][:, 3].max() < 1e-9
    psi = out["xi_psi"] @ P.T
    np.testing.assert_allclose(psi[:, [0, -1]], th, atol=1e-10)


def test_psi_step_is_the_surrogate_least_squares_optimum():
    rng = np.random.default_rng(3)
    n_p, T, rp = 30, 5.0, 1.7
    prob = fp.FPProblem(n_p=n_p, T=T, start=np.zeros(2), goal=np.ones(2), psi0=0.4, psif=-1.1,
                        centers=np.zeros((0, 2)), semi_axes=np.zeros((0, 2)),
                        velocities=np.zeros((0, 2)), offsets=np.array([0.0]), r_circle=0.0,
                        vmax=1.0, amax=1.0, rho_psi=rp)
    P, _, _ = am.bernstein(n_p, T)
    lp = rng.normal(size=(2, 11)); ph = rng.normal(size=(2, n_p))
    out = fp.psi_step(fp.kkt_psi(prob), P, lp, ph, rp, np.array([0.4, -1.1]))
    Pb, _, Pddb = _tables(n_p, T)
    A = np.stack([Pb[0], Pb[-1]])
    for i in range(2):
        ref = _qp_bruteforce(Pddb.T @ Pddb + rp * Pb.T @ Pb, -lp[i] - rp * Pb.T @ ph[i], A,
                             np.array([0.4, -1.1]))
        np.testing.assert_allclose(out[i], ref, atol=1e-9)


def test_xi_step_is_the_stacked_least_squares_optimum():
    """One xi-step with arbitrary targets and multipliers equals the brute-force
    minimiser of 1/2 xi^T Q xi + q^T xi - lambda^T xi + rho/2 ||F xi - g||^2 s.t.
    the boundary rows, with F built here from BPoly tables."""
    rng = np.random.default_rng(1)
    n_p, T, offs, n_o, rho = 30, 4.0, np.array([-0.4, 0.1, 0.5]), 2, 1.3
    prob = fp.FPProblem(n_p=n_p, T=T, start=np.array([0.0, 0.0]), goal=np.array([4.0, 2.0]),
                        psi0=0.0, psif=0.0, centers=rng.normal(size=(n_o, 2)),
                        semi_axes=np.ones((n_o, 2)), velocities=np.zeros((n_o, 2)),
                        offsets=offs, r_circle=0.1, vmax=1.0, amax=1.0, rho=rho)
    Ki, F = fp.kkt_half(prob)
    q = rng.normal(size=22); bnd = np.array([0.0, 0.0, 0.0, 4.0])
    lam = rng.normal(size=(2, 22)); g = rng.normal(size=(2, F.shape[0]))
    xi = fp.xi_step_half(Ki, F, q, bnd, lam, g, rho)
    Pb, Pdb, Pddb = _tables(n_p, T)
    Z = np.zeros((n_p, 11))
    rows = [np.hstack([Pdb, Z]), np.hstack([Pddb, Z])]
    rows += [np.hstack([Pb, o * Pb]) for o in offs for _ in range(n_o)]
    rows.append(np.hstack([Z, Pb]))
    Fb = np.vstack(rows)
    Q = np.zeros((22, 22)); Q[:11, :11] = Pddb.T @ Pddb + Pb.T @ Pb
    A = np.zeros((4, 22)); A[:, :11] = np.stack([Pb[0], Pdb[0], Pddb[0], Pb[-1]])
    for i in range(2):
        ref = _qp_bruteforce(Q + rho * Fb.T @ Fb, q - lam[i] - rho * Fb.T @ g[i], A, bnd)
        np.testing.assert_allclose(xi[i], ref, atol=1e-8)


def test_wrap_and_a_turn_through_pi():
    x = np.array([-np.pi, np.pi, 3 * np.pi, -3 * np.pi + 0.1, 0.0, 7.0])
    w = fp.wrap(x)
    assert np.all(w > -np.pi) and np.all(w <= np.pi)
    np.testing.assert_allclose(np.cos(w), np.cos(x), atol=1e-12)
    np.testing.assert_allclose(np.sin(w), np.sin(x), atol=1e-12)
    # heading from 2.8 rad to -2.8 rad (through +-pi the long way, as fixed by the
    # end rows): the unwrapped surrogate converges with consistent copies
    prob = fp.FPProblem(n_p=40, T=6.0, start=np.array([0.0, 0.0]), goal=np.array([3.0, 0.0]),
                        psi0=2.8, psif=-2.8, centers=np.zeros((0, 2)), semi_axes=np.zeros((0, 2)),
                        velocities=np.zeros((0, 2)), offsets=np.array([0.0]), r_circle=0.0,
                        vmax=1e3, amax=1e3, rho=1.0, rho_psi=1.0)
    xi0 = np.zeros((1, 3, 11))
    xi0[0, 0] = np.linspace(0, 3, 11)
    xi0[0, 2] = np.linspace(2.8, -2.8, 11)
    out = fp.solve(prob, xi0, 2000)
    P, _, _ = _tables(40, 6.0)
    psi = out["xi_psi"][0] @ P.T
    assert abs(psi[0] - 2.8) < 1e-9 and abs(psi[-1] + 2.8) < 1e-9
    assert out["residual"][0, 3] < 1e-4


def test_rectangle_clears_the_obstacles_after_convergence():
    """A three-circle footprint through a config-2-style scene: at convergence
    every circle keeps its inflated ellipse distance and the copies match the
    heading."""
    b = scenes.config2(7, n_scenes=1, inits=6, n_obstacles=12)
    prob = _from_batch(b, offsets=(-0.35, 0.0, 0.35), r_circle=0.15, psi0=np.pi / 4,
                       psif=np.pi / 4)
    xi0 = np.concatenate([b.xi0, np.full((6, 1, 11), np.pi / 4)], 1)
    out = fp.solve(prob, xi0, 1500, tol=1e-3)
    ok = np.all(out["residual"] <= 1e-3, axis=1)
    assert ok.sum() >= 1
    P, _, _ = am.bernstein(prob.n_p, prob.T)
    t = np.linspace(0, prob.T, prob.n_p)
    ob = fp.obstacle_positions(prob, t)
    ax = prob.semi_axes[:, None, :] + prob.r_circle
    for i in np.nonzero(ok)[0]:
        x, c, y, s = (out["xi"][i, k] @ P.T for k in range(4))
        for r in prob.offsets:
            foot = np.stack([x + r * c, y + r * s], -1)
            u = (foot[None] - ob) / ax
            assert np.sqrt((u ** 2).sum(-1)).min() >= 1 - 2e-3
