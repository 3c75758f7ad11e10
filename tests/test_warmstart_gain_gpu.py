"""What the trained warm-start network gains: 4096 held-out scenes solved from the
network's K = 8 proposals versus the initialisations the optimizer uses without
it -- the straight line (zero offsets, the fallback) and 8 random draws
N(straight line, 0.5 m). The network is trained on the GPU by the library's own
kernels on scenes that the optimizer itself solved, with labels that cover each
scene's homotopy classes first."""
import dataclasses

import numpy as np
import pytest

from paper_2408_10731_b300 import scenes

pytestmark = pytest.mark.gpu


def _solve(batch, xi0, tp, cap=500, tol=1e-3):
    from paper_2408_10731_b300 import trajbatch as tb
    b = dataclasses.replace(batch, xi0=scenes.f32(xi0), traj_problem=tp)
    h = tb.from_batch(b)
    try:
        st = h.solve(cap, tol)
        out = h.get_trajectories()
    finally:
        h.close()
    ok = (out["status"] == 0).reshape(batch.n_problems, 8)
    return ok, out["iters"].reshape(batch.n_problems, 8), st["gpu_ms"]


def test_trained_network_gains_over_the_fallback_initialisation(capsys):
    import torch
    from paper_2408_10731_b300 import warmstart
    ws, info = warmstart.trained(seed=1000, n_scenes=200000, epochs=20)
    try:
        if info is not None:  # trained in this process: the loss must fall well below the start
            assert info["losses"][-1] < 0.5 * info["losses"][0], info["losses"]
        held = scenes.ellipse_scenes(99, 4096)
        P = held.n_problems
        xi_l, tp = warmstart.proposals(ws, held)
        ws.sync()
        line = np.stack([scenes.straight_line_coeffs(held.start[k], held.goal[k]) for k in range(P)])
        rng = np.random.default_rng(5)
        res = {}
        for name, x in (("learned", xi_l.cpu().numpy()), ("straight", np.repeat(line, 8, 0)),
                        ("random", np.repeat(line, 8, 0) + rng.normal(0, 0.5, (P * 8, 2, 11)))):
            ok, it, ms = _solve(held, x, tp)
            res[name] = dict(scenes=float(ok.any(1).mean()), traj=int(ok.sum()),
                             it_med=float(np.median(it[ok])) if ok.any() else np.inf,
                             it_p90=float(np.percentile(it[ok], 90)) if ok.any() else np.inf,
                             solved_per_s=float(ok.sum() / (ms * 1e-3)))
        with capsys.disabled():
            print("\nwarm-start gain on 4096 held-out scenes:", res)
        # against the zero-offset fallback: more scenes and more trajectories solved
        # (the median iteration count of the solved ones is not compared: the fallback
        # solves only the easy scenes)
        assert res["learned"]["scenes"] >= 1.3 * res["straight"]["scenes"], res
        assert res["learned"]["traj"] >= res["straight"]["traj"], res
        # against random draws: more trajectories solved and more solved per second (the
        # share of scenes with at least one solution stays below the random draws':
        # the eight heads cover fewer homotopy classes than eight independent draws,
        # with or without class-diverse labels; recorded above)
        assert res["learned"]["traj"] >= res["random"]["traj"], res
        assert res["learned"]["solved_per_s"] >= res["random"]["solved_per_s"], res
    finally:
        ws.close()
