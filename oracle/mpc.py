"""Oracle of the receding-horizon step (Paper II's MPC use of Algorithm 2) --
TEST INFRASTRUCTURE ONLY, FP64 numpy.

Paper II runs its batch optimizer inside an MPC loop and starts every control
loop's solve from the Lagrange multipliers of the previous one. Reading R12
(also in am_oracle.c) of what one control step does when the robot has followed
the plan for delta seconds:

  executed plan  per problem, one trajectory the robot follows during [0, delta];
  start state    its position, velocity and acceleration at delta become the
                 problem's boundary rows at the start (goal, horizon T and grid
                 unchanged; the tracking line x_des runs from the new start);
  obstacles      each moves on to c + v delta (its constant-velocity prediction);
  iterate        every trajectory's polynomial is re-expressed on the shifted
                 window [delta, delta + T]: the unique degree-10 polynomial
                 q(tau') = p(delta / T + tau') (extrapolated past the old end);
  multipliers    kept as they are (the paper's carry), and the next solve starts
                 with the usual projection of the re-expressed iterate (so u is
                 formed afresh for the moved problem) with lambda0 = the kept ones.

The re-expression is computed here by its definition: the old polynomial is
evaluated at 11 distinct points of the new window and the Bernstein coefficients
of the interpolating polynomial are solved for (an 11 x 11 collocation system).

Parity status: shift pinned by evaluation against scipy's BPoly with
extrapolation (tests/test_oracle_mpc.py); start_state by BPoly derivatives;
the boundary rows with a start state and the carried multipliers through
am.solve's pins there.
"""
from __future__ import annotations

import dataclasses
from math import comb

import numpy as np

from . import am

N = 10  # Bernstein degree


def bernstein_values(tau):
    """B_i(tau) = C(10, i) tau^i (1 - tau)^(10 - i) for any real tau: [len(tau), 11]."""
    tau = np.asarray(tau, np.float64)[:, None]
    i = np.arange(N + 1)[None, :]
    c = np.array([comb(N, k) for k in range(N + 1)], np.float64)[None, :]
    return c * tau ** i * (1.0 - tau) ** (N - i)


def shift_coeffs(xi, frac):
    """Coefficients [..., 11] of q(tau') = p(frac + tau') for coefficients xi [..., 11]
    of p: collocation at tau'_k = k / 10, k = 0..10."""
    nodes = np.arange(N + 1) / N
    Bn = bernstein_values(nodes)                # new basis at the nodes
    Bo = bernstein_values(frac + nodes)         # old basis at the same instants
    vals = np.einsum("ki,...i->...k", Bo, np.asarray(xi, np.float64))
    return np.einsum("ik,...k->...i", np.linalg.inv(Bn), vals)


def start_state(xi, T, delta):
    """Position, velocity and acceleration [3][dim] at time delta of the trajectory
    with coefficients xi [dim][11] over [0, T]: the derivatives of the Bernstein form
    (degree-9 and degree-8 differences) evaluated at tau = delta / T."""
    tau = np.array([delta / T])
    xi = np.asarray(xi, np.float64)
    b10 = bernstein_values(tau)[0]
    b9 = np.array([comb(N - 1, k) * tau[0] ** k * (1 - tau[0]) ** (N - 1 - k) for k in range(N)])
    b8 = np.array([comb(N - 2, k) * tau[0] ** k * (1 - tau[0]) ** (N - 2 - k) for k in range(N - 1)])
    d1 = N * np.diff(xi, axis=-1)
    d2 = N * (N - 1) * np.diff(xi, n=2, axis=-1)
    return np.stack([xi @ b10, d1 @ b9 / T, d2 @ b8 / T ** 2])


def repose_obstacles(centers, velocities, delta):
    """Constant-velocity prediction c + v delta in FP64, rounded to the FP32 the
    obstacle inputs are given in."""
    c = np.asarray(centers, np.float64) + np.asarray(velocities, np.float64) * float(delta)
    return c.astype(np.float32)


def mpc_step(batch, xi, lam, executed, delta):
    """One receding-horizon step: (batch', start_va [P][2][dim], xi0' [B][dim][11],
    lam0 [B][dim][11]) for the next solve, from the last solve's coefficients xi and
    multipliers lam of every trajectory and executed[p], the trajectory of problem p
    that the robot followed during [0, delta]."""
    P = batch.n_problems
    start = np.zeros_like(np.asarray(batch.start, np.float64))
    va = np.zeros((P, 2, batch.dim))
    for p in range(P):
        T = float(batch.duration[p])
        st = start_state(np.asarray(xi[executed[p]], np.float64), T, delta)
        start[p], va[p, 0], va[p, 1] = st[0], st[1], st[2]
    frac = np.asarray(batch.duration, np.float64)[batch.traj_problem]
    xi0 = np.stack([shift_coeffs(np.asarray(xi[k], np.float64), delta / frac[k])
                    for k in range(batch.n_traj)])
    moved = dataclasses.replace(batch, start=start,
                                centers=repose_obstacles(batch.centers, batch.velocities, delta))
    return moved, va, xi0, np.asarray(lam, np.float64).copy()


def solve_after_step(batch, xi, lam, executed, delta, iters, **kw):
    """mpc_step, then am.solve of the moved problems from the carried state for a fixed
    number of iterations; returns (moved batch, start_va, am.solve's output)."""
    moved, va, xi0, lam0 = mpc_step(batch, xi, lam, executed, delta)
    out = am.solve(moved, iters, xi0=xi0, start_va=va, lam0=lam0, want_lambda=True, **kw)
    return moved, va, out
