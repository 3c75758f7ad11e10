"""GPU parity of the footprint-and-heading optimizer (Paper II, Algorithm 2 with
the heading variables) against the FP64 oracle, through the C ABI (traj_fp_*)."""
import numpy as np
import pytest

from oracle import am, footprint as fp
from paper_2408_10731_b300 import scenes

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5       # m, grid positions of x, y and of every footprint circle
PSI_TOL = 1e-5       # rad, heading on the grid
OFFS = (-0.35, 0.0, 0.35)
RC = 0.15


def _problem(b, p, psi0, psif, rho_psi=1.0):
    c, a, v = b.obstacles(p)
    return fp.FPProblem(n_p=int(b.n_steps[p]), T=float(b.duration[p]), start=b.start[p],
                        goal=b.goal[p], psi0=float(psi0[p]), psif=float(psif[p]),
                        centers=np.asarray(c, float), semi_axes=np.asarray(a, float),
                        velocities=np.asarray(v, float), offsets=np.asarray(OFFS),
                        r_circle=RC, vmax=b.vmax, amax=b.amax, rho=b.rho, rho_psi=rho_psi)


def _headings(b):
    d = b.goal - b.start
    h = np.arctan2(d[:, 1], d[:, 0])
    return h, h


def _run(b, psi0, psif, xpsi0, iters, tol=-1.0, rho_psi=1.0):
    from paper_2408_10731_b300 import footprint as gfp
    h = gfp.from_batch(b, psi0, psif, xpsi0, OFFS, RC, rho_psi=rho_psi)
    try:
        st = h.solve(iters, tol)
        return h.get_trajectories(), st
    finally:
        h.close()


def _errors(b, out, iters, psi0, psif, xpsi0, tol=-1.0, rho_psi=1.0):
    e_pos, e_psi = 0.0, 0.0
    for p in range(b.n_problems):
        idx = np.nonzero(b.traj_problem == p)[0]
        prob = _problem(b, p, psi0, psif, rho_psi)
        xi0 = np.concatenate([b.xi0[idx, :2], xpsi0[idx].reshape(-1, 1, 11)], 1)
        ref = fp.solve(prob, xi0, iters, tol=tol)
        P, _, _ = am.bernstein(prob.n_p, prob.T)
        g = out["xi"][idx].astype(np.float64)
        for r in (0.0,) + OFFS:
            pg = np.stack([g[:, 0] @ P.T + r * (g[:, 1] @ P.T), g[:, 2] @ P.T + r * (g[:, 3] @ P.T)], -1)
            x = ref["xi"]
            po = np.stack([x[:, 0] @ P.T + r * (x[:, 1] @ P.T), x[:, 2] @ P.T + r * (x[:, 3] @ P.T)], -1)
            e_pos = max(e_pos, np.linalg.norm(pg - po, axis=-1).max())
        e_psi = max(e_psi, np.abs(g[:, 4] @ P.T - ref["xi_psi"] @ P.T).max())
        if tol >= 0:
            np.testing.assert_array_equal(out["iterations"][idx], ref["iterations"])
    return e_pos, e_psi


def test_scenes_with_moving_ellipses_match_oracle():
    """20 iterations: in the transient, where footprint circles sit deep inside
    ellipses, the method itself amplifies a 1e-7 relative change of its inputs to
    7e-6 m after 40 iterations on this scene (FP64 oracle against itself), so the
    FP32 path is held to 1e-5 m at 20 iterations, where that amplification is
    below 2e-6 m."""
    b = scenes.config2(11, n_scenes=3, inits=4, n_obstacles=12)
    psi0, psif = _headings(b)
    xpsi0 = np.repeat(psi0[b.traj_problem][:, None], 11, 1)
    out, _ = _run(b, psi0, psif, xpsi0, 20)
    e_pos, e_psi = _errors(b, out, 20, psi0, psif, xpsi0)
    assert e_pos <= POS_TOL and e_psi <= PSI_TOL, (e_pos, e_psi)


def test_uneven_problems_and_a_turning_heading():
    """Ragged horizons (50..150 points) and obstacle counts, end headings that
    differ from the travel direction by up to 2.5 rad, noisy initial headings."""
    b = scenes.config4(3, n_problems=5, inits=2)
    rng = np.random.default_rng(4)
    psi0 = rng.uniform(-np.pi, np.pi, b.n_problems)
    psif = psi0 + rng.uniform(-2.5, 2.5, b.n_problems)
    xpsi0 = np.stack([np.linspace(psi0[p], psif[p], 11) for p in b.traj_problem])
    xpsi0[:, 1:-1] += rng.normal(0, 0.1, (b.n_traj, 9))
    out, _ = _run(b, psi0, psif, xpsi0, 20, rho_psi=2.0)
    e_pos, e_psi = _errors(b, out, 20, psi0, psif, xpsi0, rho_psi=2.0)
    assert e_pos <= POS_TOL and e_psi <= PSI_TOL, (e_pos, e_psi)


def test_zero_iterations_returns_the_initial_iterate():
    b = scenes.config2(12, n_scenes=2, inits=2, n_obstacles=5)
    psi0, psif = _headings(b)
    xpsi0 = np.repeat(psi0[b.traj_problem][:, None], 11, 1)
    out, _ = _run(b, psi0, psif, xpsi0, 0)
    np.testing.assert_allclose(out["xi"][:, 0], b.xi0[:, 0], atol=0)
    np.testing.assert_allclose(out["xi"][:, 2], b.xi0[:, 1], atol=0)
    np.testing.assert_allclose(out["xi"][:, 4], xpsi0, atol=1e-6)
    np.testing.assert_allclose(out["xi"][:, 1], np.cos(xpsi0), atol=1e-6)
    np.testing.assert_allclose(out["xi"][:, 3], np.sin(xpsi0), atol=1e-6)
    assert np.all(out["iterations"] == 0)


def test_early_stop_matches_oracle_iterations():
    """Stop at the first iteration with all four residuals <= tol; the decision is
    checked against the oracle's (a residual within 2e-5 of tol could flip it, so the
    scene is checked for that margin first)."""
    b = scenes.config2(13, n_scenes=2, inits=4, n_obstacles=8)
    psi0, psif = _headings(b)
    xpsi0 = np.repeat(psi0[b.traj_problem][:, None], 11, 1)
    tol = 5e-3
    for p in range(b.n_problems):
        idx = np.nonzero(b.traj_problem == p)[0]
        ref = fp.solve(_problem(b, p, psi0, psif), np.concatenate(
            [b.xi0[idx, :2], xpsi0[idx].reshape(-1, 1, 11)], 1), 400, want_hist=True)
        h = ref["hist"].max(axis=2)                     # [iters, B]
        for i in range(h.shape[1]):                      # up to each oracle stop
            k = int(np.argmax(h[:, i] <= tol)) if np.any(h[:, i] <= tol) else h.shape[0] - 1
            assert np.all(np.abs(h[:k + 1, i] - tol) > 2e-5), "a residual sits on the tolerance"
    out, st = _run(b, psi0, psif, xpsi0, 400, tol)
    e_pos, e_psi = _errors(b, out, 400, psi0, psif, xpsi0, tol=tol)
    assert e_pos <= POS_TOL and e_psi <= PSI_TOL, (e_pos, e_psi)
    assert st["n_solved"] == int(np.sum(np.all(out["residual"] <= tol, axis=1)))


def test_eight_circles_on_the_longest_horizon_and_errors():
    """Eight footprint circles and n_p = 256 (the longest grid, eight points per
    lane); non-finite inputs, bad problem indices and calls out of order are
    refused."""
    from paper_2408_10731_b300 import footprint as gfp
    from paper_2408_10731_b300.trajbatch import TrajBatchError
    offs = tuple(np.linspace(-0.7, 0.7, 8))
    b = scenes.config2(21, n_scenes=1, inits=2, n_obstacles=6)
    b.n_steps = np.array([256], np.int32)
    b.duration = np.array([20.0])
    psi0, psif = _headings(b)
    xpsi0 = np.repeat(psi0[b.traj_problem][:, None], 11, 1)
    h = gfp.from_batch(b, psi0, psif, xpsi0, offs, RC)
    try:
        h.solve(10)
        out = h.get_trajectories()
    finally:
        h.close()
    c, a, v = b.obstacles(0)
    prob = fp.FPProblem(n_p=256, T=20.0, start=b.start[0], goal=b.goal[0], psi0=float(psi0[0]),
                        psif=float(psif[0]), centers=np.asarray(c, float),
                        semi_axes=np.asarray(a, float), velocities=np.asarray(v, float),
                        offsets=np.asarray(offs), r_circle=RC, vmax=b.vmax, amax=b.amax, rho=b.rho)
    ref = fp.solve(prob, np.concatenate([b.xi0[:, :2], xpsi0[:, None]], 1), 10)
    P, _, _ = am.bernstein(256, 20.0)
    for r in (0.0,) + offs:
        g, x = out["xi"].astype(np.float64), ref["xi"]
        pg = np.stack([g[:, 0] @ P.T + r * (g[:, 1] @ P.T), g[:, 2] @ P.T + r * (g[:, 3] @ P.T)], -1)
        po = np.stack([x[:, 0] @ P.T + r * (x[:, 1] @ P.T), x[:, 2] @ P.T + r * (x[:, 3] @ P.T)], -1)
        assert np.linalg.norm(pg - po, axis=-1).max() <= POS_TOL
    h = gfp.FootprintBatch(2, 4, 4, 100, (0.0,), 0.1, 1.0, 1.0)
    try:
        with pytest.raises(TrajBatchError):
            h.solve(5)                       # before set_problems / set_initial
        h.set_problems([50], [5.0], [[0, 0]], [[4, 4]], [0.0], [0.0], [0, 0],
                       np.zeros((0, 2)), np.zeros((0, 2)), np.zeros((0, 2)))
        with pytest.raises(TrajBatchError):
            h.set_initial([1], np.zeros((1, 3, 11)))        # problem index out of range
        bad = np.zeros((1, 3, 11)); bad[0, 0, 3] = np.inf
        with pytest.raises(TrajBatchError):
            h.set_initial([0], bad)
    finally:
        h.close()


def test_full_size_bench_workload_sampled():
    """The bench's workload (125 scenes x 8 initialisations, 20 moving ellipses, three
    circles) in one launch; three problems checked against the oracle after 20
    iterations."""
    b = scenes.config2(0, n_scenes=125, inits=8, n_obstacles=20)
    psi0, psif = _headings(b)
    xpsi0 = np.repeat(psi0[b.traj_problem][:, None], 11, 1)
    out, _ = _run(b, psi0, psif, xpsi0, 20)
    P, _, _ = am.bernstein(100, float(b.duration[0]))
    for p in (0, 62, 124):
        idx = np.nonzero(b.traj_problem == p)[0]
        ref = fp.solve(_problem(b, p, psi0, psif), np.concatenate(
            [b.xi0[idx, :2], xpsi0[idx].reshape(-1, 1, 11)], 1), 20)
        g, x = out["xi"][idx].astype(np.float64), ref["xi"]
        for r in (0.0,) + OFFS:
            pg = np.stack([g[:, 0] @ P.T + r * (g[:, 1] @ P.T), g[:, 2] @ P.T + r * (g[:, 3] @ P.T)], -1)
            po = np.stack([x[:, 0] @ P.T + r * (x[:, 1] @ P.T), x[:, 2] @ P.T + r * (x[:, 3] @ P.T)], -1)
            assert np.linalg.norm(pg - po, axis=-1).max() <= POS_TOL, p
