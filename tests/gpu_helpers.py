"""Shared helpers of the GPU parity tests (run the CUDA path, compare positions)."""
import numpy as np

from oracle import am
from paper_2408_10731_b300 import scenes

POS_TOL = 1e-5  # metres: max coefficient-evaluated position error, FP32 GPU vs FP64 oracle


def gpu_solve(batch, iters, tol=-1.0, precision="fp32", cost_mode="smooth_track",
              timeout_ms=0.0, xi0=None, state=False):
    from paper_2408_10731_b300 import trajbatch as tb
    b = batch if xi0 is None else __import__("dataclasses").replace(batch, xi0=xi0)
    h = tb.from_batch(b, precision=precision, cost_mode=cost_mode)
    try:
        try:
            stats = h.solve(iters, tol, timeout_ms=timeout_ms)
        except tb.TrajBatchError as e:
            if e.code not in (-5, -6):
                raise
            stats = dict(error=e.code)
        out = h.get_trajectories()
        out["stats"] = stats
        if state:
            out.update(h.get_state())
        return out
    finally:
        h.close()


def position_error(batch, xi_a, xi_b, dense=1000):
    """Max |p_a - p_b| over axes, the n_p grid and `dense` uniform tau, per trajectory."""
    xi_a = np.asarray(xi_a, np.float64); xi_b = np.asarray(xi_b, np.float64)
    err = np.zeros(xi_a.shape[0])
    for p in range(batch.n_problems):
        idx = np.nonzero(batch.traj_problem == p)[0]
        if idx.size == 0:
            continue
        for n in (int(batch.n_steps[p]), dense):
            P, _, _ = am.bernstein(n, float(batch.duration[p]))
            d = np.einsum("ti,bdi->btd", P, xi_a[idx] - xi_b[idx])
            err[idx] = np.maximum(err[idx], np.abs(d).max(axis=(1, 2)))
    return err


def reduced_config4(n_problems=12, seed=0, inits=2):
    full = scenes.config4(seed, n_problems=256, inits=inits)
    # pick problems spanning every horizon and small/large obstacle counts
    picks = []
    for n_p in (50, 75, 100, 150):
        cand = [p for p in range(full.n_problems) if int(full.n_steps[p]) == n_p]
        cand.sort(key=lambda p: full.n_obstacles(p))
        k = max(1, n_problems // 4)
        sel = [cand[int(round(i * (len(cand) - 1) / max(1, k - 1)))] for i in range(k)]
        picks.extend(sel)
    return full.select_problems(sorted(set(picks)))
