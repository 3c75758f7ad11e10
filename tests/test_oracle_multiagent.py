"""Pins of the multi-agent oracle (Algorithm 5) against special cases, brute force
and the properties the method must deliver."""
import numpy as np
import pytest

from oracle import am, multiagent as ma
from tests.test_oracle_am import _qp_bruteforce, _tables


def _prob(start, goal, r=0.3, h=0.0, n_p=50, T=5.0, obs=None, obs_r=None, **kw):
    start, goal = np.asarray(start, float), np.asarray(goal, float)
    return ma.MAProblem(dim=start.shape[1], n_p=n_p, T=T, start=start, goal=goal, radius=r,
                        height=h, obs_centers=None if obs is None else np.asarray(obs, float),
                        obs_radii=None if obs_r is None else np.asarray(obs_r, float), **kw)


def _brute_free(prob):
    """Each agent's min 1/2 sum_t ||p''||^2 s.t. the boundary rows, by the null-space
    method on BPoly tables (an independent basis)."""
    P, Pd, Pdd = _tables(prob.n_p, prob.T)
    A = np.stack([P[0], Pd[0], Pdd[0], P[-1], Pd[-1], Pdd[-1]])
    out = np.zeros((prob.n_agents, prob.dim, 11))
    for i in range(prob.n_agents):
        for a in range(prob.dim):
            b = np.array([prob.start[i, a], 0, 0, prob.goal[i, a], 0, 0])
            out[i, a] = _qp_bruteforce(Pdd.T @ Pdd, np.zeros(11), A, b)
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_agents_that_never_meet_stay_at_their_free_optima(dim):
    """Parallel lanes 4 m apart with r = 0.3: every d >= 1 is inactive, targets
    equal the current differences, lambda stays 0 and the x-step's fixed point is
    each agent's own QP optimum (a wrong pair sign, factor or KKT block moves it)."""
    start = [[0.0, 4.0 * i] + ([1.0] if dim == 3 else []) for i in range(3)]
    goal = [[10.0, 4.0 * i + 0.5] + ([2.0] if dim == 3 else []) for i in range(3)]
    prob = _prob(start, goal, h=0.3 if dim == 3 else 0.0, rho=2.0)
    out = ma.solve(prob, 8)
    np.testing.assert_allclose(out["xi"], _brute_free(prob), atol=1e-9)
    assert out["residual"] < 1e-12
    assert np.abs(out["lam_ag"]).max() < 1e-10


def test_d_step_is_the_dense_grid_minimiser_with_the_bound():
    rng = np.random.default_rng(0)
    for _ in range(30):
        e = rng.normal(size=3)
        delta = rng.normal(size=3) * 2
        lam = rng.normal(size=3)
        rho = rng.uniform(0.5, 3)
        grid = np.linspace(1.0, 30.0, 290001)
        f = ((delta[None] - grid[:, None] * e[None] + lam[None] / rho) ** 2).sum(1)
        d = ma.d_step(e[None], delta[None], lam[None], rho)[0]
        assert abs(d - grid[np.argmin(f)]) < 2e-4


def test_direction_lies_on_the_spheroid_along_delta():
    rng = np.random.default_rng(1)
    a, b = 0.8, 1.3
    delta = rng.normal(size=(200, 3)) * 3
    e = ma.direction(delta, a, b, 3)
    np.testing.assert_allclose((e[:, :2] ** 2).sum(1) / a ** 2 + e[:, 2] ** 2 / b ** 2, 1.0,
                               atol=1e-12)
    np.testing.assert_allclose(np.cross(e, delta), 0.0, atol=1e-11)
    assert np.all((e * delta).sum(1) > 0)
    e2 = ma.direction(delta[:, :2], a, b, 2)
    np.testing.assert_allclose(np.linalg.norm(e2, axis=1), a, atol=1e-12)
    np.testing.assert_allclose(e2[:, 0] * delta[:, 1] - e2[:, 1] * delta[:, 0], 0.0, atol=1e-11)
    # reading M2: delta = 0 gives alpha = beta = 0
    np.testing.assert_allclose(ma.direction(np.zeros((1, 3)), a, b, 3)[0], [0, 0, b])
    np.testing.assert_allclose(ma.direction(np.zeros((1, 2)), a, b, 2)[0], [a, 0])


def test_x_step_is_the_stacked_least_squares_optimum():
    """One x-step with arbitrary targets equals the brute-force minimiser of
    1/2 sum_i xi_i^T Pdd^T Pdd xi_i + rho/2 ||A_fo xi - b||^2 s.t. the boundary rows,
    with A_fo built here from BPoly tables, one dense block row per ordered pair
    and per (agent, obstacle)."""
    rng = np.random.default_rng(2)
    N, n_o, n_p, T, rho = 3, 2, 20, 4.0, 1.7
    start = rng.uniform(0, 5, (N, 2)); goal = rng.uniform(0, 5, (N, 2))
    prob = _prob(start, goal, n_p=n_p, T=T, obs=rng.uniform(0, 5, (n_o, 2)),
                 obs_r=[0.3, 0.4], rho=rho)
    P, Pd, Pdd = am.bernstein(n_p, T)
    Kinv = ma.kkt_inverse(Pdd.T @ Pdd, ma.build_A_fo(P, N, n_o), ma.boundary_rows(P, Pd, Pdd),
                          rho, N)
    ag, ob = ma.pair_lists(N, n_o)
    t_ag = rng.normal(size=(len(ag), n_p, 2)); t_ob = rng.normal(size=(len(ob), n_p, 2))
    e_bd = ma.boundary_values(start, goal)
    xi = ma.x_step(Kinv, ma.build_A_fo(P, N, n_o), rho, [t_ag, t_ob], e_bd, N)

    Pb, Pdb, Pddb = _tables(n_p, T)
    rows = []
    for (i, j) in ag:
        blk = np.zeros((n_p, N * 11)); blk[:, i * 11:(i + 1) * 11] = Pb; blk[:, j * 11:(j + 1) * 11] = -Pb
        rows.append(blk)
    for (i, o) in ob:
        blk = np.zeros((n_p, N * 11)); blk[:, i * 11:(i + 1) * 11] = Pb
        rows.append(blk)
    F = np.vstack(rows)
    Q = np.kron(np.eye(N), Pddb.T @ Pddb) + rho * F.T @ F
    A1 = np.stack([Pb[0], Pdb[0], Pddb[0], Pb[-1], Pdb[-1], Pddb[-1]])
    A = np.kron(np.eye(N), A1)
    for a in range(2):
        b = np.concatenate([t_ag[..., a].reshape(-1), t_ob[..., a].reshape(-1)])
        ref = _qp_bruteforce(Q, -rho * F.T @ b, A, e_bd[:, a, :].reshape(-1))
        np.testing.assert_allclose(xi[:, a, :].reshape(-1), ref, atol=1e-8)


def _min_pair_distance(prob, xi):
    pos = ma.positions(prob, xi)
    N = prob.n_agents
    return min(np.linalg.norm(pos[i] - pos[j], axis=1).min()
               for i in range(N) for j in range(i + 1, N))


def test_swap_separates_agents_and_keeps_its_symmetry():
    """Two agents exchange places nearly head-on (offset 0.1 m). The free optima
    collide; Algorithm 5 drives the residual down and separates them to >= 2r up to
    that residual, and the point symmetry p -> -p that exchanges the agents holds
    at every iterate."""
    start = np.array([[-4.0, 0.05], [4.0, -0.05]])
    goal = -start
    prob = _prob(start, goal, r=0.4, n_p=60, T=8.0, rho=2.0, rho_levels=10, rho_growth=1.5,
                 rho_every=40)
    free = ma.free_init(prob)
    assert _min_pair_distance(prob, free) < 0.3
    out = ma.solve(prob, 600, tol=1e-4, want_hist=True)
    assert out["residual"] <= 1e-4, out["residual"]
    assert _min_pair_distance(prob, out["xi"]) >= 0.8 - 2e-4
    np.testing.assert_allclose(out["xis"][:, 0], -out["xis"][:, 1], atol=1e-9)


def test_three_dimensional_crossing_with_a_static_obstacle():
    """Four agents cross through a shared centre region that also holds a static
    sphere; the method reaches residual 1e-3 and every pair and agent-obstacle
    spheroid constraint holds up to it."""
    start = np.array([[-3, 0, 1], [3, 0.2, 1.1], [0.1, -3, 0.9], [-0.2, 3, 1.0]], float)
    goal = -start * np.array([1, 1, 0]) + np.array([0, 0, 1.0])
    prob = _prob(start, goal, r=0.3, h=0.4, n_p=60, T=8.0, obs=[[0.1, 0.1, 1.2]], obs_r=[0.5],
                 rho=2.0, rho_levels=10, rho_growth=1.5, rho_every=40)
    out = ma.solve(prob, 800, tol=1e-3)
    assert out["residual"] <= 1e-3, out["residual"]
    pos = ma.positions(prob, out["xi"])
    for i in range(4):
        for j in range(i + 1, 4):
            d = pos[i] - pos[j]
            s = (d[:, :2] ** 2).sum(1) / 0.6 ** 2 + d[:, 2] ** 2 / 0.8 ** 2
            assert np.sqrt(s).min() >= 1 - 2e-3
        d = pos[i] - np.array([0.1, 0.1, 1.2])
        s = (d[:, :2] ** 2).sum(1) / 0.8 ** 2 + d[:, 2] ** 2 / 0.9 ** 2
        assert np.sqrt(s).min() >= 1 - 2e-3
    free = ma.positions(prob, ma.free_init(prob))
    d = free - np.array([0.1, 0.1, 1.2])
    assert (np.sqrt((d[..., :2] ** 2).sum(-1) / 0.8 ** 2 + d[..., 2] ** 2 / 0.9 ** 2)).min() < 0.5


def test_penalty_ladder_of_growth_one_is_the_fixed_penalty():
    start = np.array([[-4.0, 0.3], [4.0, -0.3], [0.2, -4.0]])
    goal = -start
    p1 = _prob(start, goal, n_p=40, rho=1.5)
    p2 = _prob(start, goal, n_p=40, rho=1.5, rho_levels=10, rho_growth=1.0, rho_every=3)
    a, b = ma.solve(p1, 30), ma.solve(p2, 30)
    np.testing.assert_array_equal(a["xi"], b["xi"])
    p3 = _prob(start, goal, n_p=40, rho=1.5, rho_levels=4, rho_growth=2.0, rho_every=10)
    c = ma.solve(p3, 30)
    assert np.abs(c["xi"] - a["xi"]).max() > 1e-6


def test_coincident_agents_are_pushed_apart():
    """Reading M2 at delta = 0: the pair (i, j), i < j, gets e = (0, 0, b) and (j, i)
    the opposite, so that every multiplier stays odd in the pair and two agents
    that start on top of each other separate (3D: vertically)."""
    e = ma.direction(np.zeros((2, 3)), 0.6, 0.8, 3, np.array([1.0, -1.0]))
    np.testing.assert_allclose(e, [[0, 0, 0.8], [0, 0, -0.8]])
    start = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    goal = np.array([[5.0, 0.0, 1.0], [5.0, 0.0, 1.0]])
    prob = _prob(start, goal, r=0.3, h=0.3, n_p=40, T=5.0, rho=2.0)
    out = ma.solve(prob, 60)
    pos = ma.positions(prob, out["xi"])
    mid = pos[:, 20]
    assert mid[0, 2] - mid[1, 2] > 0.1          # agent 0 above agent 1 mid-way
    np.testing.assert_allclose(pos[0, :, 2] + pos[1, :, 2], 2.0, atol=1e-9)
    np.testing.assert_allclose(out["lam_ag"][0], -out["lam_ag"][1], atol=1e-12)
