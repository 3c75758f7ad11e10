"""ctypes wrapper of the FP64 AM oracle (am_oracle.c) -- TEST INFRASTRUCTURE ONLY.

Parity status:
  bernstein    pinned: partition of unity, endpoint interpolation, linear
               precision, central differences (tests/test_oracle_basis.py)
  kkt          pinned: LAPACK solve of the same KKT system; obstacle-free QP
               fixed point equals the brute-force equality-constrained QP
  projection   pinned: dense-grid minimisation of each (alpha, beta, d)
               subproblem; closed form d = max(1, ||u||) (eq. d_max)
  start state  pinned: with a start velocity and acceleration in the boundary
  and carry    rows the obstacle-free fixed point is the brute-force QP with those
               rows; one iteration from imported multipliers equals the
               brute-force proximal QP step with them (tests/test_oracle_mpc.py)
  am_solve     pinned: the first two iterations (moving obstacles, active
               bounds, 2D and 3D) equal their step-by-step brute-force
               composition -- targets from the dense-grid-pinned projections,
               xi-steps as null-space QP solves on BPoly tables with a literal
               stacked F, lambda <- lambda - rho F^T (F xi - g); plus the fixed
               point of a feasible QP optimum, the obstacle-free QP optimum,
               A xi = b at every iterate and the multiplier sign. The paper
               prints no iterate values, so later iterates are checked only
               through these steps.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIBS = {}
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _lib(real: str = "f64"):
    if real not in _LIBS:
        paths = _build.build()
        lib = ctypes.CDLL(paths[real])
        lib.orc_am_solve_flat.restype = ctypes.c_int
        lib.orc_am_solve_flat.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp, _dp, _dp,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double, _ip, _dp, _dp, _dp,
            _ip, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp,
            _dp]
        lib.orc_kkt_flat.restype = ctypes.c_int
        lib.orc_kkt_flat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, _dp, _dp]
        lib.orc_bernstein.restype = None
        lib.orc_bernstein.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
        lib.orc_invert.restype = ctypes.c_int
        lib.orc_invert.argtypes = [ctypes.c_int, _dp, _dp]
        real_p = _dp if real == "f64" else ctypes.POINTER(ctypes.c_float)
        lib.orc_project_obstacle.restype = None
        lib.orc_project_obstacle.argtypes = [ctypes.c_int, real_p, real_p, real_p]
        lib.orc_project_bound.restype = None
        lib.orc_project_bound.argtypes = [ctypes.c_int, real_p,
                                          ctypes.c_double if real == "f64" else ctypes.c_float,
                                          real_p]
        _LIBS[real] = lib
    return _LIBS[real]


def _p(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def bernstein(n_p: int, T: float):
    """P, Pdot, Pddot [n_p, 11] (eq. parameter with the Bernstein basis)."""
    P = np.zeros((n_p, 11)); Pd = np.zeros((n_p, 11)); Pdd = np.zeros((n_p, 11))
    _lib().orc_bernstein(n_p, float(T), _p(P), _p(Pd), _p(Pdd))
    return P, Pd, Pdd


def invert(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.zeros_like(A)
    rc = _lib().orc_invert(A.shape[0], _p(A), _p(out))
    if rc:
        raise np.linalg.LinAlgError("singular")
    return out


def kkt(dim, n_p, T, n_o, rho=1.0, w_smooth=1.0, w_track=1.0, cost_mode=0):
    """(K, K^-1), 15x15: [[Q + rho F^T F, A^T], [A, 0]] (eq. over_2)."""
    K = np.zeros((15, 15)); Ki = np.zeros((15, 15))
    rc = _lib().orc_kkt_flat(dim, n_p, float(T), n_o, rho, w_smooth, w_track, cost_mode,
                             _p(K), _p(Ki))
    if rc:
        raise np.linalg.LinAlgError("singular KKT")
    return K, Ki


def project_obstacle(xt, axes, real="f64"):
    """Target offset g - o for one point offset x~ (eqs. zeta_2, compute_d_mij)."""
    dt = np.float64 if real == "f64" else np.float32
    pt = _dp if real == "f64" else ctypes.POINTER(ctypes.c_float)
    xt = np.ascontiguousarray(xt, dtype=dt); ax = np.ascontiguousarray(axes, dtype=dt)
    out = np.zeros_like(xt)
    _lib(real).orc_project_obstacle(xt.shape[0], _p(xt, pt), _p(ax, pt), _p(out, pt))
    return out


def project_bound(w, bound, real="f64"):
    """Target for a velocity/acceleration vector (eqs. alpha_v, compute_dv)."""
    dt = np.float64 if real == "f64" else np.float32
    pt = _dp if real == "f64" else ctypes.POINTER(ctypes.c_float)
    w = np.ascontiguousarray(w, dtype=dt)
    out = np.zeros_like(w)
    _lib(real).orc_project_bound(w.shape[0], _p(w, pt), bound, _p(out, pt))
    return out


def solve(batch, max_iters: int, tol: float = -1.0, cost_mode: int = 0, w_smooth: float = 1.0,
          w_track: float = 1.0, iters_fixed=None, want_lambda: bool = False,
          want_hist: bool = False, n_threads: int = 0, real: str = "f64", xi0=None,
          rho_levels: int = 1, rho_growth: float = 1.0, rho_every: int = 0,
          box_lo=None, box_hi=None, start_va=None, lam0=None):
    """Run Algorithm 2 on every trajectory of a scenes.Batch.

    Returns dict(xi [B,dim,11], residual [B,3], iters [B], lam?, hist?).
    tol < 0 disables the early stop; iters_fixed[B] runs exactly that many
    iterations per trajectory (no stop test). rho_levels / rho_growth / rho_every:
    the penalty continuation of reading R10 (rho_levels = 1: a fixed rho).
    box_lo / box_hi [n_problems][dim]: workspace bounds of reading R11 (None: none).
    start_va [n_problems][2][dim]: start velocity and acceleration of the boundary rows
    (reading R12; None: at rest). lam0 [B][dim][11]: multipliers the loop starts from
    (reading R12's carry; None: zero).
    """
    lib = _lib(real)
    dim = batch.dim
    xi0_all = np.ascontiguousarray(batch.xi0 if xi0 is None else xi0, dtype=np.float64)
    B = xi0_all.shape[0]
    xi = np.zeros((B, dim, 11)); lam = np.zeros((B, dim, 11)) if want_lambda else None
    res = np.zeros((B, 3)); its = np.zeros(B, np.int32)
    hist = np.full((B, max_iters + 1, 3), np.nan) if want_hist else None
    fixed_all = None if iters_fixed is None else np.asarray(iters_fixed, np.int32)
    for p in range(batch.n_problems):
        idx = np.nonzero(batch.traj_problem == p)[0]
        if idx.size == 0:
            continue
        c, a, v = (np.ascontiguousarray(x, dtype=np.float64) for x in batch.obstacles(p))
        st = np.ascontiguousarray(batch.start[p], dtype=np.float64)
        gl = np.ascontiguousarray(batch.goal[p], dtype=np.float64)
        x0 = np.ascontiguousarray(xi0_all[idx])
        xo = np.zeros_like(x0); lo = np.zeros_like(x0) if want_lambda else None
        ro = np.zeros((idx.size, 3)); io = np.zeros(idx.size, np.int32)
        ho = np.full((idx.size, max_iters + 1, 3), np.nan) if want_hist else None
        fx = None if fixed_all is None else np.ascontiguousarray(fixed_all[idx])
        sva = None if start_va is None else np.ascontiguousarray(start_va[p], np.float64)
        l0 = None if lam0 is None else np.ascontiguousarray(np.asarray(lam0, np.float64)[idx])
        rc = lib.orc_am_solve_flat(
            dim, int(batch.n_steps[p]), float(batch.duration[p]), c.shape[0], _p(c), _p(a),
            _p(v), _p(st), _p(gl), float(batch.vmax), float(batch.amax), float(batch.rho),
            float(w_smooth), float(w_track), int(cost_mode), idx.size, _p(x0), int(max_iters),
            float(tol), _p(fx, _ip), _p(xo), _p(lo), _p(ro), _p(io, _ip), _p(ho),
            int(n_threads), int(rho_levels), float(rho_growth), int(rho_every),
            _p(None if box_lo is None else np.ascontiguousarray(box_lo[p], np.float64)),
            _p(None if box_hi is None else np.ascontiguousarray(box_hi[p], np.float64)),
            _p(sva), _p(l0))
        if rc:
            raise RuntimeError(f"oracle solve failed for problem {p}: {rc}")
        xi[idx] = xo; res[idx] = ro; its[idx] = io
        if want_lambda:
            lam[idx] = lo
        if want_hist:
            hist[idx] = ho
    out = dict(xi=xi, residual=res, iters=its)
    if want_lambda:
        out["lam"] = lam
    if want_hist:
        out["hist"] = hist
    return out


def positions(xi, n_p: int, T: float):
    """Evaluate p(t) = P xi at the n_p grid points: [B, n_p, dim]."""
    P, _, _ = bernstein(n_p, T)
    return np.einsum("ti,bdi->btd", P, xi)
