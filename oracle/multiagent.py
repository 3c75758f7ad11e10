"""Oracle of the joint multi-agent trajectory optimizer (Paper IV, Algorithm 5) --
TEST INFRASTRUCTURE ONLY, FP64 numpy/scipy.

Problem (eqs. cost_multiagent .. quadratic_multiagent): N agents, each a degree-10
Bernstein polynomial per axis on an n_p-point grid over [0, T]; cost
1/2 sum_i xi_i^T Pdd^T Pdd xi_i per axis (the QP form printed with eq.
eq_step_x); start and goal position, velocity and acceleration fixed (zero
velocity and acceleration); agents are spheroids (r, r, h) that must keep every
other agent outside the spheroid (a, a, b) = (2r, 2r, 2h) around them, and
static obstacles are circumscribing spheres of radius r_o, kept outside
(r + r_o, r + r_o, h + r_o).

Algorithm 5, in the paper's order and notation, over ORDERED pairs (i, j), i != j,
with the constraint x_i - x_j - a d_ij cos(alpha_ij) sin(beta_ij) = 0 per axis
(eq. sphere_proposed) and multipliers lambda_ij(t) per axis:
  x-step   eq. kkt_step_x: the stacked KKT system over all agents, with A_fo the
           literal rows P xi_i - P xi_j (one block row per ordered pair and time
           step; eq. A_f) and P xi_i (static obstacles), solved with its inverse
           cached once per penalty;
  alpha    eq. com_alpha_i: atan2(dy, dx);
  beta     eq. com_beta_i: atan2(dx / (a cos alpha), dz / b);
  d        eq. com_d_i: the one-variable least-squares minimiser, then d >= 1;
  lambda   eqs. update_lamda_xi .. update_lamda_zi.

Readings (where the print is silent or inconsistent):
  M1  the bound is d >= 1 (eq. sphere_proposed); the text's "clip to [0, 1]"
      would allow overlap and is read as a slip;
  M2  dx / (a cos alpha) is read as sqrt(dx^2 + dy^2) / a, its value wherever
      cos alpha != 0 (cos alpha has the sign of dx), so that the 0/0 at dx = 0 is
      defined; at dx = dy = dz = 0, atan2(0, 0) = 0 gives alpha = beta = 0, i.e.
      e = (0, 0, b) (2D: (a, 0)) for the pair (i, j) with i < j and the opposite
      direction for (j, i), so that the two agents are pushed apart rather than
      both the same way (every other e is already odd in delta);
  M3  initialisation: xi^0 is the obstacle-free optimum of each agent's QP;
      alpha^0, beta^0, d^0 follow from xi^0 with lambda^0 = 0;
  M4  the residual of iteration k is max over pairs, obstacles and grid points
      of || delta - d e(alpha, beta) ||_2 after the d-step; a scene stops at the
      first k with residual <= tol;
  M5  penalty ladder (the paper caches the inverse for ten increasing rho_o
      used in later iterations): rho growth^l, one level up after every
      rho_every-th unconverged iteration, as in the single-agent solver; the
      x-step uses lambda / rho of the level it runs at.
  M6  2D: the same with alpha only (circles of radius a = 2r and r + r_o).

Parity status: pinned by (i) the fixed point of agents that never come close,
which must be each agent's brute-force equality-constrained QP optimum with
zero residual; (ii) the d-step against a dense-grid minimisation of its
one-variable objective with the bound; (iii) the alpha/beta step: e lies on the
spheroid and is parallel to delta; (iv) the x-step's KKT inverse against
scipy's sparse least-squares of the same stacked objective; (v) convergence of
a crossing scene to pairwise distances >= a up to the residual and antipodal
symmetry of a symmetric two-agent swap.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import am

NC = 11


@dataclasses.dataclass
class MAProblem:
    dim: int
    n_p: int
    T: float
    start: np.ndarray            # [N, dim]
    goal: np.ndarray             # [N, dim]
    radius: float                # agent horizontal radius r
    height: float = 0.0          # agent vertical half-size h (3D)
    obs_centers: np.ndarray = None   # [n_o, dim]
    obs_radii: np.ndarray = None     # [n_o]
    rho: float = 1.0
    rho_levels: int = 1
    rho_growth: float = 1.0
    rho_every: int = 0

    @property
    def n_agents(self):
        return self.start.shape[0]

    @property
    def n_obs(self):
        return 0 if self.obs_centers is None else len(self.obs_centers)


def boundary_rows(P, Pd, Pdd):
    """A of eq. kkt_step_x: position, velocity, acceleration at both ends (6 x 11)."""
    return np.stack([P[0], Pd[0], Pdd[0], P[-1], Pd[-1], Pdd[-1]])


def boundary_values(start, goal):
    """b_eq per agent and axis: (start, 0, 0, goal, 0, 0) -> [N, dim, 6]."""
    N, dim = start.shape
    e = np.zeros((N, dim, 6))
    e[:, :, 0] = start
    e[:, :, 3] = goal
    return e


def pair_lists(N, n_o):
    """Ordered agent pairs (i, j), i != j, then (agent, obstacle) pairs."""
    ag = [(i, j) for i in range(N) for j in range(N) if i != j]
    ob = [(i, o) for i in range(N) for o in range(n_o)]
    return ag, ob


def build_A_fo(P, N, n_o):
    """A_fo of eq. A_f (one axis), sparse: a block of n_p rows per ordered pair
    (+P at agent i, -P at agent j), then per (agent, obstacle) (+P at agent i)."""
    n_p = P.shape[0]
    ag, ob = pair_lists(N, n_o)
    blocks = []
    for (i, j) in ag:
        row = [None] * N
        for k in range(N):
            row[k] = sp.csr_matrix((n_p, NC))
        row[i] = sp.csr_matrix(P)
        row[j] = sp.csr_matrix(-P)
        blocks.append(row)
    for (i, o) in ob:
        row = [sp.csr_matrix((n_p, NC)) for _ in range(N)]
        row[i] = sp.csr_matrix(P)
        blocks.append(row)
    if not blocks:
        return sp.csr_matrix((0, N * NC))
    return sp.bmat(blocks, format="csr")


def kkt_inverse(Q0, A_fo, Aeq, rho, N):
    """Inverse of [[I (x) Q0 + rho A_fo^T A_fo, I (x) A^T], [I (x) A, 0]] (eq. kkt_step_x)."""
    H = np.kron(np.eye(N), Q0) + rho * (A_fo.T @ A_fo).toarray()
    Ab = np.kron(np.eye(N), Aeq)
    m = Ab.shape[0]
    K = np.block([[H, Ab.T], [Ab, np.zeros((m, m))]])
    return np.linalg.inv(K)


def direction(delta, a, b, dim, sign=1.0):
    """e(alpha, beta) of eq. sphere_proposed from eqs. com_alpha_i and com_beta_i
    (readings M2, M6): delta [..., dim] -> e [..., dim]; `sign` (broadcast to
    delta[..., 0]) orients e where delta = 0."""
    alpha = np.arctan2(delta[..., 1], delta[..., 0])
    if dim == 2:
        e = np.stack([a * np.cos(alpha), a * np.sin(alpha)], -1)
    else:
        rxy = np.hypot(delta[..., 0], delta[..., 1])
        beta = np.arctan2(rxy / a, delta[..., 2] / b)
        e = np.stack([a * np.cos(alpha) * np.sin(beta), a * np.sin(alpha) * np.sin(beta),
                      b * np.cos(beta) * np.ones_like(alpha)], -1)
    zero = np.all(delta == 0.0, axis=-1)
    if np.any(zero):
        e = np.where(zero[..., None], e * np.broadcast_to(np.asarray(sign, float),
                                                           zero.shape)[..., None], e)
    return e


def d_step(e, delta, lam, rho):
    """eq. com_d_i: argmin_d ||delta - d e + lam / rho||^2, then d >= 1 (reading M1)."""
    d = (e * (delta + lam / rho)).sum(-1) / (e * e).sum(-1)
    return np.maximum(d, 1.0)


def x_step(Kinv, A_fo, rho, target_rows, e_bd, N):
    """eq. kkt_step_x per axis: rhs = [rho A_fo^T b; b_eq], xi = top of Kinv rhs.
    target_rows: list of [pairs, n_p, dim] target blocks in A_fo's row order."""
    dim = e_bd.shape[1]
    xi = np.zeros((N, dim, NC))
    for a in range(dim):
        bvec = np.concatenate([r[..., a].reshape(-1) for r in target_rows])
        top = rho * (A_fo.T @ bvec) if bvec.size else np.zeros(N * NC)
        rhs = np.concatenate([top, e_bd[:, a, :].reshape(-1)])
        xi[:, a, :] = (Kinv @ rhs)[:N * NC].reshape(N, NC)
    return xi


def free_init(prob: MAProblem):
    """Reading M3: each agent's obstacle-free optimum, [N, dim, 11]."""
    P, Pd, Pdd = am.bernstein(prob.n_p, prob.T)
    A = boundary_rows(P, Pd, Pdd)
    Q0 = Pdd.T @ Pdd
    K = np.block([[Q0, A.T], [A, np.zeros((6, 6))]])
    e = boundary_values(prob.start, prob.goal)
    rhs = np.concatenate([np.zeros(e.shape[:2] + (NC,)), e], -1)
    return np.linalg.solve(K, rhs[..., None])[..., :NC, 0]


def _deltas(prob, pos):
    """delta for every agent pair and obstacle pair, with their (a, b):
    pos [N, n_p, dim] -> (delta_ag [Nag, n_p, dim], delta_ob [Nob, n_p, dim])."""
    N, n_o = prob.n_agents, prob.n_obs
    ag, ob = pair_lists(N, n_o)
    dag = np.stack([pos[i] - pos[j] for (i, j) in ag]) if ag else np.zeros((0, prob.n_p, prob.dim))
    dob = (np.stack([pos[i] - prob.obs_centers[o][None, :] for (i, o) in ob]) if ob
           else np.zeros((0, prob.n_p, prob.dim)))
    return dag, dob


def solve(prob: MAProblem, iters: int, tol: float = -1.0, xi0=None, want_hist=False):
    """Algorithm 5 for `iters` iterations (or until the residual <= tol).
    Returns xi [N, dim, 11], residual (last), iterations, and optionally the
    residual history and the per-iteration xi."""
    N, dim, n_p, n_o = prob.n_agents, prob.dim, prob.n_p, prob.n_obs
    P, Pd, Pdd = am.bernstein(n_p, prob.T)
    Aeq = boundary_rows(P, Pd, Pdd)
    Q0 = Pdd.T @ Pdd
    A_fo = build_A_fo(P, N, n_o)
    levels = max(1, prob.rho_levels)
    rhos = [prob.rho * prob.rho_growth ** l for l in range(levels)]
    Kinv = [kkt_inverse(Q0, A_fo, Aeq, r, N) for r in rhos]
    e_bd = boundary_values(prob.start, prob.goal)          # [N, dim, 6]
    a_ag, b_ag = 2.0 * prob.radius, 2.0 * prob.height
    ag_pairs, _ = pair_lists(N, n_o)
    sgn = np.array([1.0 if i < j else -1.0 for (i, j) in ag_pairs])[:, None]
    if n_o:
        a_ob = prob.radius + np.asarray(prob.obs_radii, float)
        b_ob = prob.height + np.asarray(prob.obs_radii, float)
        ag, ob = pair_lists(N, n_o)
        a_ob_rows = np.array([a_ob[o] for (_, o) in ob])[:, None]
        b_ob_rows = np.array([b_ob[o] for (_, o) in ob])[:, None]
    xi = free_init(prob) if xi0 is None else np.array(xi0, float)

    # initialisation (reading M3): alpha, beta, d from xi^0, lambda^0 = 0
    pos = np.einsum("tk,iak->ita", P, xi)
    dag, dob = _deltas(prob, pos)
    lam_ag = np.zeros_like(dag)
    lam_ob = np.zeros_like(dob)
    level = 0
    rho = rhos[level]
    e_ag = direction(dag, a_ag, b_ag, dim, sgn)
    d_ag = d_step(e_ag, dag, lam_ag, rho)
    if n_o:
        e_ob = direction(dob, a_ob_rows, b_ob_rows, dim)
        d_ob = d_step(e_ob, dob, lam_ob, rho)
    hist, xis = [], []
    k_done, res = 0, np.inf
    for k in range(1, iters + 1):
        # x-step (eq. kkt_step_x), per axis; targets b = d e - lambda / rho
        bt_ag = d_ag[..., None] * e_ag - lam_ag / rho
        rhs_rows = [bt_ag]
        if n_o:
            bt_ob = d_ob[..., None] * e_ob - lam_ob / rho + prob.obs_centers[
                np.array([o for (_, o) in ob])][:, None, :]
            rhs_rows.append(bt_ob)
        new = x_step(Kinv[level], A_fo, rho, rhs_rows, e_bd, N)
        xi = new
        pos = np.einsum("tk,iak->ita", P, xi)
        dag, dob = _deltas(prob, pos)
        # alpha, beta (eqs. com_alpha_i, com_beta_i), d (eq. com_d_i) with lambda^k
        e_ag = direction(dag, a_ag, b_ag, dim, sgn)
        d_ag = d_step(e_ag, dag, lam_ag, rho)
        r_ag = dag - d_ag[..., None] * e_ag
        lam_ag = lam_ag + rho * r_ag                      # eqs. update_lamda_*
        res = np.linalg.norm(r_ag, axis=-1).max() if r_ag.size else 0.0
        if n_o:
            e_ob = direction(dob, a_ob_rows, b_ob_rows, dim)
            d_ob = d_step(e_ob, dob, lam_ob, rho)
            r_ob = dob - d_ob[..., None] * e_ob
            lam_ob = lam_ob + rho * r_ob
            res = max(res, np.linalg.norm(r_ob, axis=-1).max())
        hist.append(res)
        if want_hist:
            xis.append(xi.copy())
        k_done = k
        if tol >= 0 and res <= tol:
            break
        if levels > 1 and prob.rho_every > 0 and k % prob.rho_every == 0 and level < levels - 1:
            level += 1
            rho = rhos[level]
    out = dict(xi=xi, residual=res, iterations=k_done, lam_ag=lam_ag, d_ag=d_ag)
    if want_hist:
        out.update(hist=np.array(hist), xis=np.array(xis))
    return out


def positions(prob: MAProblem, xi):
    """Grid positions [N, n_p, dim] of coefficients [N, dim, 11]."""
    P, _, _ = am.bernstein(prob.n_p, prob.T)
    return np.einsum("tk,iak->ita", P, xi)
