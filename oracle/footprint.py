"""Oracle of the batch optimizer for a robot with a multi-circle footprint and a
heading (Paper II, Algorithm 2 with the heading variables) -- TEST
INFRASTRUCTURE ONLY, FP64 numpy.

Problem (eqs. acc_cost .. coll_multiagent, 2D): per trajectory, positions
x(t), y(t) and heading psi(t) as degree-10 Bernstein polynomials; cost
sum_t (x''^2 + y''^2 + psi''^2 + (x - x_des)^2 + (y - y_des)^2) with x_des, y_des
the constant-velocity line from start to goal; the footprint is n_c circles at
offsets r_m along the heading, each kept outside every obstacle ellipse
(inflated by the circle radius); speed and acceleration bounded.

Reformulation (eqs. cos_ref .. fc1, reform_cost .. d_bound, Q_matrix and the
F / g of the paper): slack copies c(t), s(t) of cos psi, sin psi with their own
coefficients, xi = (xi_x, xi_c, xi_y, xi_s); per half h in {x, y} the rows of F
are [Pdot 0] (speed), [Pddot 0] (acceleration), [P r_m P] for every circle m
and obstacle j (collision), and [0 P] (the copy of cos / sin psi).

Algorithm 2, in the paper's order: xi-step (eq. zeta_1_sepration_1, the KKT of
eq. over_2 per half), psi-step (eq. compute_convex_surrogate), alpha-step
(eqs. zeta_2, alpha_v, alpha_a), d-step (eqs. compute_d_mij, compute_dv,
compute_da), multiplier updates (eqs. update_lambda2_1, update_lambda2_2).

Readings (besides R1-R9 of the single-agent oracle, which carry over: the
xi-step right-hand side -q + lambda + rho F^T g, lambda <- lambda - rho F^T
(F xi - g), alpha = atan2(y~/b, x~/a), d_v, d_a over [0, 1], the boundary rows
of R8 for x and y, L-infinity residuals over the grid):
  H1  the collision rows use the slack copies, x~ = x + r_m c - x_o, as F does
      (the alpha-step text writes cos psi); the ellipse axes are the obstacle's
      semi-axes plus the circle radius;
  H2  the psi-step target atan2(s, c) is unwrapped against the current heading:
      psi^ = psi + wrap(atan2(s, c) - psi), wrap to (-pi, pi], so that the
      surrogate never sees a 2 pi jump;
  H3  A_psi fixes the heading at both ends (first and last row of P);
  H4  lambda_psi <- lambda_psi - rho_psi P^T (P xi_psi - psi^) (the printed
      update reuses F's residual, which has the wrong dimension);
  H5  initialisation: xi_x, xi_y and xi_psi are given; the targets of the first
      xi-step use c, s = cos psi, sin psi on the grid, lambda = 0; the copy
      coefficients start as cos / sin of the heading coefficients (they are
      returned after zero iterations and do not enter the first xi-step);
  H6  a fourth residual, max_t ||(c, s) - (cos psi, sin psi)||, joins the stop
      test.

Parity status: pinned by (i) one circle at offset 0 and radius 0, which reduces
each half's speed, acceleration and collision rows to the single-agent F, so
x and y must follow the single-agent oracle iterate for iterate; (ii) the
xi-step and the psi-step against brute-force minimisers of their stacked
objectives on BPoly tables; (iii) an obstacle-free run from a constant
heading, whose fixed point is the brute-force QP optimum of x, y with a
constant heading and exact copies; (iv) a turn through +-pi, where the
unwrapped surrogate converges with consistent copies; (v) a three-circle
footprint that clears every inflated ellipse at convergence.
The heading multiplier keeps what it gathered in the transient: from a noisy
initial heading the iteration reaches a consistent (c, s, psi) whose psi is
not the minimiser of sum psi''^2, the same kind of feasible non-optimal point
as the workspace slack of the single-agent method.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import am

NC = 11


@dataclasses.dataclass
class FPProblem:
    n_p: int
    T: float
    start: np.ndarray        # [2]
    goal: np.ndarray         # [2]
    psi0: float
    psif: float
    centers: np.ndarray      # [n_o, 2] at t = 0
    semi_axes: np.ndarray    # [n_o, 2]
    velocities: np.ndarray   # [n_o, 2]
    offsets: np.ndarray      # [n_c] circle offsets along the heading
    r_circle: float
    vmax: float
    amax: float
    rho: float = 1.0
    rho_psi: float = 1.0


def wrap(x):
    """Angle to (-pi, pi]."""
    return x - 2.0 * np.pi * np.ceil((x - np.pi) / (2.0 * np.pi))


def tables(n_p, T):
    return am.bernstein(n_p, T)


def build_F_half(P, Pd, Pdd, offsets, n_o):
    """Rows of F for one half (eq. F of the paper): speed, acceleration, one block
    per (circle m, obstacle j), cos / sin copy. Columns (xi_h, xi_copy)."""
    n_p = P.shape[0]
    Z = np.zeros((n_p, NC))
    rows = [np.hstack([Pd, Z]), np.hstack([Pdd, Z])]
    for m in range(len(offsets)):
        for j in range(n_o):
            rows.append(np.hstack([P, offsets[m] * P]))
    rows.append(np.hstack([Z, P]))
    return np.vstack(rows)


def kkt_half(prob: FPProblem):
    """Inverse of [[Q + rho F^T F, A^T], [A, 0]] for one half (eq. over_2) with
    Q = blockdiag(Pdd^T Pdd + P^T P, 0) (eq. Q_matrix) and A the boundary rows of
    xi_h (reading R8)."""
    P, Pd, Pdd = tables(prob.n_p, prob.T)
    F = build_F_half(P, Pd, Pdd, prob.offsets, len(prob.centers))
    Q = np.zeros((2 * NC, 2 * NC))
    Q[:NC, :NC] = Pdd.T @ Pdd + P.T @ P
    A = np.zeros((4, 2 * NC))
    A[:, :NC] = np.stack([P[0], Pd[0], Pdd[0], P[-1]])
    K = np.block([[Q + prob.rho * F.T @ F, A.T], [A, np.zeros((4, 4))]])
    return np.linalg.inv(K), F


def xi_step_half(Ki, F, q, b, lam, g, rho):
    """eq. zeta_1_sepration_1 for one half (reading R1 of the single-agent oracle):
    the KKT solution with right-hand side (-q + lambda + rho F^T g, b); [B, 22]."""
    B = lam.shape[0]
    rhs = np.concatenate([-q[None] + lam + rho * g @ F, np.broadcast_to(b, (B, len(b)))], 1)
    return (rhs @ Ki.T)[:, :F.shape[1]]


def kkt_psi(prob: FPProblem):
    """Inverse of [[Pdd^T Pdd + rho_psi P^T P, A_psi^T], [A_psi, 0]] (eq.
    compute_convex_surrogate, reading H3)."""
    P, Pd, Pdd = tables(prob.n_p, prob.T)
    A = np.stack([P[0], P[-1]])
    K = np.block([[Pdd.T @ Pdd + prob.rho_psi * P.T @ P, A.T], [A, np.zeros((2, 2))]])
    return np.linalg.inv(K)


def psi_step(Kp, P, lpsi, psi_hat, rho_psi, bpsi):
    """eq. compute_convex_surrogate: argmin 1/2 xi^T Pdd^T Pdd xi - lambda_psi^T xi
    + rho_psi/2 ||psi^ - P xi||^2 s.t. the end headings; [B, 11]."""
    B = lpsi.shape[0]
    rhs = np.concatenate([lpsi + rho_psi * psi_hat @ P, np.broadcast_to(bpsi, (B, 2))], 1)
    return (rhs @ Kp.T)[:, :NC]


def obstacle_positions(prob, t):
    """[n_o, n_p, 2] centres of the moving ellipses on the grid."""
    return prob.centers[:, None, :] + prob.velocities[:, None, :] * t[None, :, None]


def project_obstacles(xt, ax):
    """Targets g - o for every (.., 2) offset x~ and axes (.., 2) (eqs. zeta_2 and
    compute_d_mij with reading R4 of the single-agent oracle)."""
    alpha = np.arctan2(xt[..., 1] / ax[..., 1], xt[..., 0] / ax[..., 0])
    ca, sa = np.cos(alpha), np.sin(alpha)
    d = (ax[..., 0] * xt[..., 0] * ca + ax[..., 1] * xt[..., 1] * sa) / (
        ax[..., 0] ** 2 * ca ** 2 + ax[..., 1] ** 2 * sa ** 2)
    d = np.maximum(d, 1.0)
    return np.stack([ax[..., 0] * d * ca, ax[..., 1] * d * sa], -1)


def project_bound(w, bound):
    """eqs. alpha_v / compute_dv (reading R5): d over [0, 1]."""
    alpha = np.arctan2(w[..., 1], w[..., 0])
    ca, sa = np.cos(alpha), np.sin(alpha)
    d = np.clip((w[..., 0] * ca + w[..., 1] * sa) / bound, 0.0, 1.0)
    return np.stack([d * bound * ca, d * bound * sa], -1)


def solve(prob: FPProblem, xi0, iters, tol=-1.0, want_hist=False):
    """Algorithm 2 with the heading for a batch of initial guesses.
    xi0: [B, 3, 11] coefficients of x, y, psi. Returns xi [B, 4, 11] in the order
    (x, c, y, s), xi_psi [B, 11], residual [B, 4] (obstacle, speed, acceleration,
    heading copy), iterations [B]."""
    P, Pd, Pdd = tables(prob.n_p, prob.T)
    n_p, n_o, n_c = prob.n_p, len(prob.centers), len(prob.offsets)
    t = np.linspace(0.0, prob.T, n_p)
    Ki, F = kkt_half(prob)
    Kp = kkt_psi(prob)
    rho, rp = prob.rho, prob.rho_psi
    xi0 = np.asarray(xi0, float)
    B = xi0.shape[0]
    tau = np.linspace(0.0, 1.0, n_p)
    des = [prob.start[a] + (prob.goal[a] - prob.start[a]) * tau for a in range(2)]
    qh = [np.concatenate([-P.T @ des[a], np.zeros(NC)]) for a in range(2)]   # eq. Q_matrix
    bh = [np.array([prob.start[a], 0.0, 0.0, prob.goal[a]]) for a in range(2)]
    bpsi = np.array([prob.psi0, prob.psif])
    ob = obstacle_positions(prob, t)                                      # [n_o, n_p, 2]
    ax = prob.semi_axes[:, None, :] + prob.r_circle                       # reading H1
    xh = [np.concatenate([xi0[:, 0], np.cos(xi0[:, 2])], 1),
          np.concatenate([xi0[:, 1], np.sin(xi0[:, 2])], 1)]             # (xi_x, xi_c), (xi_y, xi_s)
    xpsi = xi0[:, 2].copy()
    lam = [np.zeros((B, 2 * NC)), np.zeros((B, 2 * NC))]
    lpsi = np.zeros((B, NC))

    def targets(pos, vel, acc, cs, psi):
        """g for both halves: rows (speed, acceleration, collisions, copy)."""
        gv = project_bound(vel, prob.vmax)
        ga = project_bound(acc, prob.amax)
        go = []
        for m in range(n_c):
            foot = pos + prob.offsets[m] * cs                            # reading H1
            xt = foot[:, None, :, :] - ob[None]                           # [B, n_o, n_p, 2]
            go.append(ob[None] + project_obstacles(xt, np.broadcast_to(ax[None], xt.shape)))
        go = np.stack(go, 1)                                              # [B, n_c, n_o, n_p, 2]
        cp = np.stack([np.cos(psi), np.sin(psi)], -1)
        g = []
        for a in range(2):
            g.append(np.concatenate([gv[..., a], ga[..., a], go[..., a].reshape(B, -1),
                                     cp[..., a]], 1))
        return g, (gv, ga, go, cp)

    def evaluate():
        x, c = xh[0][:, :NC], xh[0][:, NC:]
        y, s = xh[1][:, :NC], xh[1][:, NC:]
        pos = np.stack([x @ P.T, y @ P.T], -1)
        vel = np.stack([x @ Pd.T, y @ Pd.T], -1)
        acc = np.stack([x @ Pdd.T, y @ Pdd.T], -1)
        cs = np.stack([c @ P.T, s @ P.T], -1)
        return pos, vel, acc, cs

    def residuals(pos, vel, acc, cs, parts):
        gv, ga, go, cp = parts
        r_o = 0.0
        if n_o:
            foot = pos[:, None] + prob.offsets[None, :, None, None] * cs[:, None]   # [B, n_c, n_p, 2]
            d = foot[:, :, None] - go                                   # [B, n_c, n_o, n_p, 2]
            r_o = np.linalg.norm(d, axis=-1).max(axis=(1, 2, 3))
        r_v = np.linalg.norm(vel - gv, axis=-1).max(1)
        r_a = np.linalg.norm(acc - ga, axis=-1).max(1)
        r_c = np.linalg.norm(cs - cp, axis=-1).max(1)
        return np.stack([np.broadcast_to(r_o, (B,)), r_v, r_a, r_c], 1)

    # initialisation (reading H5)
    psi = xpsi @ P.T
    pos0 = np.stack([xi0[:, 0] @ P.T, xi0[:, 1] @ P.T], -1)
    vel0 = np.stack([xi0[:, 0] @ Pd.T, xi0[:, 1] @ Pd.T], -1)
    acc0 = np.stack([xi0[:, 0] @ Pdd.T, xi0[:, 1] @ Pdd.T], -1)
    g, _ = targets(pos0, vel0, acc0, np.stack([np.cos(psi), np.sin(psi)], -1), psi)
    iters_done = np.zeros(B, np.int32)
    active = np.ones(B, bool)
    res = np.full((B, 4), np.inf)
    hist = []
    for k in range(1, iters + 1):
        # xi-step (eq. zeta_1_sepration_1 per half; reading R1)
        new = [xi_step_half(Ki, F, qh[a], bh[a], lam[a], g[a], rho) for a in range(2)]
        # psi-step (eq. compute_convex_surrogate; readings H2, H3)
        c_new, s_new = new[0][:, NC:] @ P.T, new[1][:, NC:] @ P.T
        psi_cur = xpsi @ P.T
        psi_hat = psi_cur + wrap(np.arctan2(s_new, c_new) - psi_cur)
        xpsi_new = psi_step(Kp, P, lpsi, psi_hat, rp, bpsi)
        # only active trajectories move
        for a in range(2):
            xh[a] = np.where(active[:, None], new[a], xh[a])
        xpsi = np.where(active[:, None], xpsi_new, xpsi)
        # alpha, d (eqs. zeta_2, alpha_v, alpha_a, compute_d_mij, compute_dv, compute_da)
        pos, vel, acc, cs = evaluate()
        psi = xpsi @ P.T
        g_new, parts = targets(pos, vel, acc, cs, psi)
        # multipliers (eq. update_lambda2_1; reading H4)
        for a in range(2):
            r = xh[a] @ F.T - g_new[a]
            lam[a] = np.where(active[:, None], lam[a] - rho * r @ F, lam[a])
        lpsi = np.where(active[:, None], lpsi - rp * (psi - psi_hat) @ P, lpsi)
        g = [np.where(active[:, None], g_new[a], g[a]) for a in range(2)]
        r_now = residuals(pos, vel, acc, cs, parts)
        res = np.where(active[:, None], r_now, res)
        iters_done = np.where(active, k, iters_done)
        if want_hist:
            hist.append(res.copy())
        if tol >= 0:
            active = active & ~np.all(res <= tol, axis=1)
            if not active.any():
                break
    xi = np.stack([xh[0][:, :NC], xh[0][:, NC:], xh[1][:, :NC], xh[1][:, NC:]], 1)
    out = dict(xi=xi, xi_psi=xpsi, residual=res, iterations=iters_done)
    if want_hist:
        out["hist"] = np.array(hist)
    return out
