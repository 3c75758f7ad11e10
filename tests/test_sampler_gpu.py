"""GPU parity of the projection-guided sampler (Algorithm 3) against the oracle.

Every stage of every outer iteration is compared with the oracle run on the
GPU's own inputs to that stage, so that a discrete decision (which samples are
elites) is always taken on the same FP32 keys on both sides.
"""
import math

import numpy as np
import pytest

from oracle import am, priest
from paper_2408_10731_b300 import scenes
from tests.gpu_helpers import POS_TOL, position_error

pytestmark = pytest.mark.gpu


def _handle(B, seed=0):
    from paper_2408_10731_b300 import trajbatch as tb
    c3 = scenes.config3(seed, n_traj=B)
    b = c3["batch"]
    return c3, b, tb.from_batch(b, cost_mode="project")


def _cuda(x, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype or torch.float32, device="cuda")


def test_philox_box_muller_draws_match_oracle():
    import torch
    c3, b, h = _handle(64)
    try:
        D = 33
        mu, sigma, best = _cuda(np.zeros(D)), _cuda(np.eye(D)), _cuda(np.zeros(D + 1))
        samples = torch.zeros(64, D, device="cuda")
        cfg = dict(n_inner=0, n_proj=64, n_elite=8, gamma=1.0, sigma_lr=0.5, eps=0.0, seed=1234)
        h.sampler_step(cfg, 3, mu, sigma, best, trace=dict(samples=samples))
        z = priest.philox_normals(64, D, 1234, 3)
        np.testing.assert_allclose(samples.cpu().numpy(), z, atol=2e-5, rtol=2e-6)
    finally:
        h.close()


def test_sampler_steps_match_oracle_stagewise():
    import torch
    B = 256
    c3, b, h = _handle(B)
    D = 33
    cfg = dict(n_inner=20, n_proj=math.ceil(0.73 * B), n_elite=math.ceil(0.10 * B), gamma=1.0,
               sigma_lr=0.5, eps=1e-6, w_res=1.0, seed=0)
    mu, sigma, best = _cuda(c3["mu0"]), _cuda(c3["sigma0"]), _cuda(np.zeros(D + 1))
    try:
        for it in range(3):
            z = scenes.normal_draws(100 + it, (B, D))
            mu_in = mu.cpu().numpy().astype(np.float64)
            sig_in = sigma.cpu().numpy().astype(np.float64)
            tr = dict(samples=torch.zeros(B, D, device="cuda"),
                      projected=torch.zeros(B, D, device="cuda"),
                      residual=torch.zeros(B, device="cuda"), cost_aug=torch.zeros(B, device="cuda"),
                      proj_idx=torch.zeros(cfg["n_proj"], dtype=torch.int32, device="cuda"),
                      elite_idx=torch.zeros(cfg["n_elite"], dtype=torch.int32, device="cuda"))
            h.sampler_step(cfg, it, mu, sigma, best, z=_cuda(z), trace=tr)
            g = {k: v.cpu().numpy() for k, v in tr.items()}
            # draw
            ref = priest.sample(mu_in, sig_in, z, cfg["eps"])
            np.testing.assert_allclose(g["samples"], ref, atol=5e-5, rtol=1e-5)
            # projection (Algorithm 2 in projection mode) from the GPU's samples
            xs = g["samples"].astype(np.float64).reshape(B, 3, 11)
            o = am.solve(b, cfg["n_inner"], tol=-1.0, cost_mode=1, xi0=xs)
            err = position_error(b, g["projected"].reshape(B, 3, 11), o["xi"])
            assert err.max() <= POS_TOL, err.max()
            # residuals and costs of the GPU's projected trajectories
            r_o, c_o = priest.costs(b, g["projected"].astype(np.float64), o["residual"])
            np.testing.assert_allclose(g["residual"], r_o, atol=2e-5, rtol=1e-4)
            np.testing.assert_allclose(g["cost_aug"], c_o, atol=1e-4, rtol=2e-5)
            # selections on the GPU's own FP32 keys: exact
            p_o, e_o = priest.select(g["residual"], g["cost_aug"], cfg["n_proj"], cfg["n_elite"])
            np.testing.assert_array_equal(g["proj_idx"], p_o)
            np.testing.assert_array_equal(g["elite_idx"], e_o)
            # mean / covariance update from the GPU's elites
            m_o, s_o, best_o, bc_o = priest.refit(g["projected"].astype(np.float64),
                                                  g["cost_aug"].astype(np.float64), e_o, mu_in,
                                                  sig_in, cfg["gamma"], cfg["sigma_lr"])
            np.testing.assert_allclose(mu.cpu().numpy(), m_o, rtol=1e-4, atol=1e-4)
            np.testing.assert_allclose(sigma.cpu().numpy(), s_o, rtol=1e-3, atol=1e-4)
            np.testing.assert_array_equal(best.cpu().numpy()[:D], g["projected"][e_o[0]])
    finally:
        h.close()


def test_refit_weights_follow_the_cost_gap_closed_form():
    """Two elites whose augmented costs differ by gamma ln 3 weigh 1 and 1/3 (the
    cheaper one heavier), so with sigma_lr = 1 the device refit must give the mean
    (3 x1 + x2) / 4 and the covariance 3/16 d d^T, d = x1 - x2 (Algorithm 3's mean and
    covariance update). The first step reads the GPU's two elites and their costs;
    gamma is then set to their gap / ln 3 and the same step (same draws, so the same
    projected samples and costs) is repeated."""
    import torch
    B = 64
    c3, b, h = _handle(B, seed=3)
    D = 33
    z = _cuda(scenes.normal_draws(77, (B, D)))
    cfg = dict(n_inner=10, n_proj=32, n_elite=2, gamma=1.0, sigma_lr=1.0, eps=1e-6, w_res=1.0,
               seed=0)
    try:
        def run(gamma):
            mu, sigma, best = _cuda(c3["mu0"]), _cuda(c3["sigma0"]), _cuda(np.zeros(D + 1))
            tr = dict(projected=torch.zeros(B, D, device="cuda"),
                      cost_aug=torch.zeros(B, device="cuda"),
                      elite_idx=torch.zeros(2, dtype=torch.int32, device="cuda"))
            h.sampler_step(dict(cfg, gamma=gamma), 0, mu, sigma, best, z=z, trace=tr)
            return mu.cpu().numpy().astype(np.float64), sigma.cpu().numpy().astype(np.float64), \
                {k: v.cpu().numpy() for k, v in tr.items()}
        _, _, g = run(1.0)
        e = g["elite_idx"]
        c1, c2 = float(g["cost_aug"][e[0]]), float(g["cost_aug"][e[1]])
        assert c2 > c1
        gamma = (c2 - c1) / math.log(3.0)
        mu, sigma, g2 = run(gamma)
        np.testing.assert_array_equal(g2["elite_idx"], e)
        np.testing.assert_array_equal(g2["cost_aug"], g["cost_aug"])
        x1 = g2["projected"][e[0]].astype(np.float64)
        x2 = g2["projected"][e[1]].astype(np.float64)
        d = x1 - x2
        scale = np.abs(x1).max()
        np.testing.assert_allclose(mu, (3 * x1 + x2) / 4, atol=2e-6 * scale)
        np.testing.assert_allclose(sigma, 3.0 / 16.0 * np.outer(d, d),
                                   atol=2e-5 * max(1.0, np.abs(d).max() ** 2))
        # the opposite sign of the exponent would put the mean at (x1 + 3 x2) / 4
        assert np.abs(mu - (x1 + 3 * x2) / 4).max() > 100 * 2e-6 * scale
    finally:
        h.close()


def test_full_size_sampler_run_invariants():
    """The 3D workload at full size: 4096 samples, 10 outer x 20 inner iterations,
    on-device Philox draws."""
    import torch
    B = 4096
    c3, b, h = _handle(B)
    D = 33
    cfg = dict(n_inner=c3["n_inner"], n_proj=c3["n_proj"], n_elite=c3["n_elite"], gamma=1.0,
               sigma_lr=0.5, eps=1e-6, w_res=1.0, seed=7)
    mu, sigma, best = _cuda(c3["mu0"]), _cuda(c3["sigma0"]), _cuda(np.zeros(D + 1))
    caug = torch.zeros(B, device="cuda")
    elite = torch.zeros(cfg["n_elite"], dtype=torch.int32, device="cuda")
    try:
        for it in range(c3["n_outer"]):
            h.sampler_step(cfg, it, mu, sigma, best, trace=dict(cost_aug=caug, elite_idx=elite))
        torch.cuda.synchronize()
        S = sigma.cpu().numpy(); e = elite.cpu().numpy(); c = caug.cpu().numpy()
        assert np.all(np.isfinite(S)) and np.all(np.isfinite(mu.cpu().numpy()))
        np.testing.assert_allclose(S, S.T, rtol=1e-5, atol=1e-6)
        assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > -1e-4
        assert len(set(e.tolist())) == len(e) and e.min() >= 0 and e.max() < B
        assert np.all(np.diff(c[e]) >= 0)
        assert best.cpu().numpy()[D] == c[e[0]]
        # the best elite is a projected trajectory: boundary rows hold
        P, Pd, Pdd = am.bernstein(100, 20.0)
        xb = best.cpu().numpy()[:D].reshape(3, 11).astype(np.float64)
        np.testing.assert_allclose(xb @ P[0], b.start[0], atol=1e-3)
        np.testing.assert_allclose(xb @ P[-1], b.goal[0], atol=1e-3)
    finally:
        h.close()


def test_decentralised_sampler_with_barn_cost_matches_oracle_stagewise():
    """D-PRIEST: four distributions over groups of 64 samples, on-device Philox
    draws, the cost with curvature and path-distance terms. Every stage is checked
    against the oracle on the GPU's own inputs to it; the selections exactly.
    c_aug tolerance: c_kappa ~ ||p'||^-4 near the rest start, where p' is an
    11-term FP32 sum of O(10) products (absolute error ~1e-5 m/s at speeds
    ~0.2 m/s), so its relative error is ~4 x 5e-5; 1e-3 leaves a margin of 5."""
    import torch
    B, n_dist, D = 256, 4, 33
    Bg = B // n_dist
    c3, b, h = _handle(B)
    cfg = dict(n_inner=20, n_proj=math.ceil(0.73 * Bg), n_elite=math.ceil(0.10 * Bg), gamma=1.0,
               sigma_lr=0.5, eps=1e-6, w_res=1.0, seed=11, w_curv=0.05, w_path=0.5)
    rng = np.random.default_rng(3)
    mus = np.stack([c3["mu0"] + (g > 0) * rng.normal(0.0, 1.0, D) for g in range(n_dist)])
    sigmas = np.stack([c3["sigma0"] * (0.5 + 0.5 * g) for g in range(n_dist)])
    mu, sigma = _cuda(mus), _cuda(sigmas)
    best = _cuda(np.zeros((n_dist, D + 1)))
    try:
        for it in range(2):
            mu_in = mu.cpu().numpy().astype(np.float64)
            sig_in = sigma.cpu().numpy().astype(np.float64)
            tr = dict(samples=torch.zeros(B, D, device="cuda"),
                      projected=torch.zeros(B, D, device="cuda"),
                      residual=torch.zeros(B, device="cuda"), cost_aug=torch.zeros(B, device="cuda"),
                      proj_idx=torch.zeros(n_dist, cfg["n_proj"], dtype=torch.int32, device="cuda"),
                      elite_idx=torch.zeros(n_dist, cfg["n_elite"], dtype=torch.int32,
                                            device="cuda"))
            h.sampler_step(cfg, it, mu, sigma, best, trace=tr, n_dist=n_dist)
            g_ = {k: v.cpu().numpy() for k, v in tr.items()}
            z = priest.philox_normals(B, D, cfg["seed"], it)
            for g in range(n_dist):
                sl = slice(g * Bg, (g + 1) * Bg)
                ref = priest.sample(mu_in[g], sig_in[g], z[sl], cfg["eps"])
                np.testing.assert_allclose(g_["samples"][sl], ref, atol=2e-4, rtol=2e-5)
            xs = g_["samples"].astype(np.float64).reshape(B, 3, 11)
            o = am.solve(b, cfg["n_inner"], tol=-1.0, cost_mode=1, xi0=xs)
            err = position_error(b, g_["projected"].reshape(B, 3, 11), o["xi"])
            assert err.max() <= POS_TOL, err.max()
            r_o, c_o = priest.costs(b, g_["projected"].astype(np.float64), o["residual"],
                                    cfg["w_res"], w_curv=cfg["w_curv"], w_path=cfg["w_path"])
            _, c_plain = priest.costs(b, g_["projected"].astype(np.float64), o["residual"])
            assert np.all(c_o > c_plain)                    # the extra terms are live
            np.testing.assert_allclose(g_["residual"], r_o, atol=2e-5, rtol=1e-4)
            np.testing.assert_allclose(g_["cost_aug"], c_o, rtol=1e-3)
            B_ = best.cpu().numpy()
            for g in range(n_dist):
                sl = slice(g * Bg, (g + 1) * Bg)
                p_o, e_o = priest.select(g_["residual"][sl], g_["cost_aug"][sl], cfg["n_proj"],
                                         cfg["n_elite"])
                np.testing.assert_array_equal(g_["proj_idx"][g], p_o)
                np.testing.assert_array_equal(g_["elite_idx"][g], e_o)
                m_o, s_o, best_o, bc_o = priest.refit(g_["projected"][sl].astype(np.float64),
                                                      g_["cost_aug"][sl].astype(np.float64), e_o,
                                                      mu_in[g], sig_in[g], cfg["gamma"],
                                                      cfg["sigma_lr"])
                np.testing.assert_allclose(mu.cpu().numpy()[g], m_o, rtol=1e-4, atol=1e-4)
                np.testing.assert_allclose(sigma.cpu().numpy()[g], s_o, rtol=1e-3, atol=1e-4)
                np.testing.assert_array_equal(B_[g, :D], g_["projected"][sl][e_o[0]])
                assert B_[g, D] == g_["cost_aug"][sl][e_o[0]]
    finally:
        h.close()


def test_decentralised_sampler_with_one_distribution_is_the_plain_step():
    """n_dist = 1 through traj_sampler_step_multi gives bitwise the result of
    traj_sampler_step (same Philox draws, same kernels)."""
    import torch
    B, D = 128, 33
    outs = []
    for multi in (False, True):
        c3, b, h = _handle(B)
        cfg = dict(n_inner=10, n_proj=90, n_elite=13, gamma=1.0, sigma_lr=0.5, eps=1e-6,
                   seed=4, w_path=0.3)
        mu, sigma, best = _cuda(c3["mu0"]), _cuda(c3["sigma0"]), _cuda(np.zeros(D + 1))
        try:
            for it in range(2):
                if multi:
                    h.sampler_step(cfg, it, mu, sigma, best, n_dist=1)
                else:
                    h.sampler_step(cfg, it, mu, sigma, best)
            torch.cuda.synchronize()
            outs.append((mu.cpu().numpy(), sigma.cpu().numpy(), best.cpu().numpy()))
        finally:
            h.close()
    for a, c in zip(*outs):
        np.testing.assert_array_equal(a, c)


def test_selections_break_exact_ties_by_the_lower_index():
    """Every normal draw used twice (at random positions): the two copies project to
    bitwise the same trajectory, so every residual and cost ties with another sample's.
    ConstraintEliteSet and EliteSet must still equal the oracle's stable selection (the
    lower index first), including the ties that straddle N_proj and N_elite."""
    import torch
    B, D = 256, 33
    c3, b, h = _handle(B)
    cfg = dict(n_inner=20, n_proj=math.ceil(0.73 * B), n_elite=math.ceil(0.10 * B), gamma=1.0,
               sigma_lr=0.5, eps=1e-6, w_res=1.0, seed=0)
    mu, sigma, best = _cuda(c3["mu0"]), _cuda(c3["sigma0"]), _cuda(np.zeros(D + 1))
    half = scenes.normal_draws(321, (B // 2, D))
    order = np.random.default_rng(5).permutation(B)
    z = np.empty((B, D))
    z[order] = np.concatenate([half, half])
    try:
        tr = dict(residual=torch.zeros(B, device="cuda"), cost_aug=torch.zeros(B, device="cuda"),
                  proj_idx=torch.zeros(cfg["n_proj"], dtype=torch.int32, device="cuda"),
                  elite_idx=torch.zeros(cfg["n_elite"], dtype=torch.int32, device="cuda"))
        h.sampler_step(cfg, 0, mu, sigma, best, z=_cuda(z), trace=tr)
        g = {k: v.cpu().numpy() for k, v in tr.items()}
        twin = np.empty(B, dtype=np.int64)
        twin[order[:B // 2]] = order[B // 2:]
        twin[order[B // 2:]] = order[:B // 2]
        assert np.array_equal(g["residual"], g["residual"][twin])
        assert np.array_equal(g["cost_aug"], g["cost_aug"][twin])
        p_o, e_o = priest.select(g["residual"], g["cost_aug"], cfg["n_proj"], cfg["n_elite"])
        np.testing.assert_array_equal(g["proj_idx"], p_o)
        np.testing.assert_array_equal(g["elite_idx"], e_o)
    finally:
        h.close()


@pytest.mark.parametrize("n_elite", [900, 1500])
def test_refit_paths_for_large_elite_sets_match_the_oracle(n_elite):
    """The refit reads the elites from shared memory while they fit: the covariance up
    to 775 elites of 33 coefficients (weighted and centred copies), the mean up to
    1241. Beyond, it reads them from global memory; 900 elites take the covariance's
    global path, 1500 both. The selections are checked exactly and the mean,
    covariance and best elite against the oracle's refit on the GPU's own keys."""
    import torch
    B, D = 4096, 33
    c3, b, h = _handle(B)
    cfg = dict(n_inner=5, n_proj=3000, n_elite=n_elite, gamma=1.0, sigma_lr=0.5, eps=1e-6,
               w_res=1.0, seed=3)
    mu, sigma, best = _cuda(c3["mu0"]), _cuda(c3["sigma0"]), _cuda(np.zeros(D + 1))
    mu_in = c3["mu0"].astype(np.float64)
    sig_in = c3["sigma0"].astype(np.float64)
    try:
        tr = dict(projected=torch.zeros(B, D, device="cuda"),
                  residual=torch.zeros(B, device="cuda"), cost_aug=torch.zeros(B, device="cuda"),
                  proj_idx=torch.zeros(cfg["n_proj"], dtype=torch.int32, device="cuda"),
                  elite_idx=torch.zeros(n_elite, dtype=torch.int32, device="cuda"))
        h.sampler_step(cfg, 0, mu, sigma, best, trace=tr)
        g = {k: v.cpu().numpy() for k, v in tr.items()}
        p_o, e_o = priest.select(g["residual"], g["cost_aug"], cfg["n_proj"], n_elite)
        np.testing.assert_array_equal(g["proj_idx"], p_o)
        np.testing.assert_array_equal(g["elite_idx"], e_o)
        m_o, s_o, best_o, bc_o = priest.refit(g["projected"].astype(np.float64),
                                              g["cost_aug"].astype(np.float64), e_o, mu_in,
                                              sig_in, cfg["gamma"], cfg["sigma_lr"])
        np.testing.assert_allclose(mu.cpu().numpy(), m_o, rtol=1e-4, atol=1e-4)
        np.testing.assert_allclose(sigma.cpu().numpy(), s_o, rtol=1e-3, atol=1e-4)
        np.testing.assert_array_equal(best.cpu().numpy()[:D], g["projected"][e_o[0]])
        assert best.cpu().numpy()[D] == g["cost_aug"][e_o[0]]
    finally:
        h.close()


def test_two_dimensional_sampler_step_matches_oracle_stagewise():
    """The sampler on a 2D projection-mode handle (22 coefficients per sample: the
    Cholesky's D = 22 form): draws, projection, costs, selections and refit of one
    outer iteration against the oracle on the GPU's inputs to each stage."""
    import torch
    from paper_2408_10731_b300 import trajbatch as tb
    B, D = 128, 22
    b = scenes.config2(21, n_scenes=1, inits=B)
    h = tb.from_batch(b, cost_mode="project")
    mu0 = scenes.straight_line_coeffs(b.start[0], b.goal[0]).reshape(-1).astype(np.float64)
    sig0 = 0.5 * np.eye(D) + 0.05 * np.ones((D, D))
    cfg = dict(n_inner=10, n_proj=math.ceil(0.73 * B), n_elite=math.ceil(0.10 * B), gamma=1.0,
               sigma_lr=0.5, eps=1e-6, w_res=1.0, seed=0)
    mu, sigma, best = _cuda(mu0), _cuda(sig0), _cuda(np.zeros(D + 1))
    z = scenes.normal_draws(77, (B, D))
    try:
        tr = dict(samples=torch.zeros(B, D, device="cuda"),
                  projected=torch.zeros(B, D, device="cuda"),
                  residual=torch.zeros(B, device="cuda"), cost_aug=torch.zeros(B, device="cuda"),
                  proj_idx=torch.zeros(cfg["n_proj"], dtype=torch.int32, device="cuda"),
                  elite_idx=torch.zeros(cfg["n_elite"], dtype=torch.int32, device="cuda"))
        h.sampler_step(cfg, 0, mu, sigma, best, z=_cuda(z), trace=tr)
        g = {k: v.cpu().numpy() for k, v in tr.items()}
        ref = priest.sample(mu0, sig0.astype(np.float32).astype(np.float64), z, cfg["eps"])
        np.testing.assert_allclose(g["samples"], ref, atol=5e-5, rtol=1e-5)
        xs = g["samples"].astype(np.float64).reshape(B, 2, 11)
        o = am.solve(b, cfg["n_inner"], tol=-1.0, cost_mode=1, xi0=xs)
        err = position_error(b, g["projected"].reshape(B, 2, 11), o["xi"])
        assert err.max() <= POS_TOL, err.max()
        r_o, c_o = priest.costs(b, g["projected"].astype(np.float64), o["residual"])
        np.testing.assert_allclose(g["residual"], r_o, atol=2e-5, rtol=1e-4)
        np.testing.assert_allclose(g["cost_aug"], c_o, atol=1e-4, rtol=2e-5)
        p_o, e_o = priest.select(g["residual"], g["cost_aug"], cfg["n_proj"], cfg["n_elite"])
        np.testing.assert_array_equal(g["proj_idx"], p_o)
        np.testing.assert_array_equal(g["elite_idx"], e_o)
        m_o, s_o, _, _ = priest.refit(g["projected"].astype(np.float64),
                                      g["cost_aug"].astype(np.float64), e_o, mu0,
                                      sig0.astype(np.float32).astype(np.float64), cfg["gamma"],
                                      cfg["sigma_lr"])
        np.testing.assert_allclose(mu.cpu().numpy(), m_o, rtol=1e-4, atol=1e-4)
        np.testing.assert_allclose(sigma.cpu().numpy(), s_o, rtol=1e-3, atol=1e-4)
    finally:
        h.close()


@pytest.mark.parametrize("n_proj,n_elite", [(128, 1), (1, 1), (128, 128)])
def test_degenerate_selection_sizes_match_the_oracle(n_proj, n_elite):
    """Edge sizes of ConstraintEliteSet / EliteSet: every sample a candidate with one
    elite, a single candidate and elite, and every sample an elite. Selections exact,
    refit (a single elite: the mean moves toward it and the covariance takes its
    outer product) against the oracle on the GPU's own keys."""
    import torch
    B, D = 128, 33
    c3, b, h = _handle(B)
    cfg = dict(n_inner=5, n_proj=n_proj, n_elite=n_elite, gamma=1.0, sigma_lr=0.5, eps=1e-6,
               w_res=1.0, seed=9)
    mu, sigma, best = _cuda(c3["mu0"]), _cuda(c3["sigma0"]), _cuda(np.zeros(D + 1))
    try:
        tr = dict(projected=torch.zeros(B, D, device="cuda"),
                  residual=torch.zeros(B, device="cuda"), cost_aug=torch.zeros(B, device="cuda"),
                  proj_idx=torch.zeros(n_proj, dtype=torch.int32, device="cuda"),
                  elite_idx=torch.zeros(n_elite, dtype=torch.int32, device="cuda"))
        h.sampler_step(cfg, 0, mu, sigma, best, trace=tr)
        g = {k: v.cpu().numpy() for k, v in tr.items()}
        p_o, e_o = priest.select(g["residual"], g["cost_aug"], n_proj, n_elite)
        np.testing.assert_array_equal(g["proj_idx"], p_o)
        np.testing.assert_array_equal(g["elite_idx"], e_o)
        m_o, s_o, _, _ = priest.refit(g["projected"].astype(np.float64),
                                      g["cost_aug"].astype(np.float64), e_o,
                                      c3["mu0"].astype(np.float64),
                                      c3["sigma0"].astype(np.float64), cfg["gamma"],
                                      cfg["sigma_lr"])
        np.testing.assert_allclose(mu.cpu().numpy(), m_o, rtol=1e-4, atol=1e-4)
        np.testing.assert_allclose(sigma.cpu().numpy(), s_o, rtol=1e-3, atol=1e-4)
        assert best.cpu().numpy()[D] == g["cost_aug"][e_o[0]]
    finally:
        h.close()


def test_non_finite_samples_rank_last():
    """Two draws made NaN by the caller: their samples are NaN, the solve leaves them
    (non-finite input), their residual ranks as +inf and their cost is NaN, so both
    selections put them last, as the oracle's stable sort does, and the refit from
    the remaining elites stays finite."""
    import torch
    B, D = 128, 33
    c3, b, h = _handle(B)
    cfg = dict(n_inner=5, n_proj=100, n_elite=13, gamma=1.0, sigma_lr=0.5, eps=1e-6, w_res=1.0,
               seed=0)
    mu, sigma, best = _cuda(c3["mu0"]), _cuda(c3["sigma0"]), _cuda(np.zeros(D + 1))
    z = scenes.normal_draws(55, (B, D)).astype(np.float64)
    z[[17, 90]] = np.nan
    try:
        tr = dict(projected=torch.zeros(B, D, device="cuda"),
                  residual=torch.zeros(B, device="cuda"), cost_aug=torch.zeros(B, device="cuda"),
                  proj_idx=torch.zeros(cfg["n_proj"], dtype=torch.int32, device="cuda"),
                  elite_idx=torch.zeros(cfg["n_elite"], dtype=torch.int32, device="cuda"))
        h.sampler_step(cfg, 0, mu, sigma, best, z=_cuda(z), trace=tr)
        g = {k: v.cpu().numpy() for k, v in tr.items()}
        assert np.isinf(g["residual"][[17, 90]]).all()
        assert not np.isfinite(g["cost_aug"][[17, 90]]).any()
        p_o, e_o = priest.select(g["residual"], g["cost_aug"], cfg["n_proj"], cfg["n_elite"])
        np.testing.assert_array_equal(g["proj_idx"], p_o)
        np.testing.assert_array_equal(g["elite_idx"], e_o)
        assert 17 not in g["proj_idx"] and 90 not in g["proj_idx"]
        assert np.all(np.isfinite(mu.cpu().numpy())) and np.all(np.isfinite(sigma.cpu().numpy()))
        assert np.isfinite(best.cpu().numpy()).all()
    finally:
        h.close()
