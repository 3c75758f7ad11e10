"""Pins of the sampler oracle (Algorithm 3) against published vectors, library
routines and textbook special cases."""
import os

import numpy as np
from scipy import stats

from oracle import priest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_philox_known_answer_vectors():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        ctr, key, out = (tuple(int(w, 16) for w in part.split()) for part in line.split("|"))
        assert priest.philox4x32_10(ctr, key) == out
        n += 1
    assert n == 3


def test_box_muller_normals_pass_ks_against_scipy():
    z = priest.philox_normals(4000, 4, seed=123, iteration=0).ravel()
    res = stats.kstest(z, stats.norm.cdf)
    assert res.pvalue > 1e-3, res
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1.0) < 0.03


def test_sampling_has_the_requested_covariance():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(6, 6))
    sigma = A @ A.T + 0.5 * np.eye(6)
    mu = rng.normal(size=6)
    z = rng.standard_normal((200000, 6))
    x = priest.sample(mu, sigma, z, eps=0.0)
    np.testing.assert_allclose(x.mean(0), mu, atol=0.03)
    np.testing.assert_allclose(np.cov(x.T), sigma, rtol=0.05, atol=0.05)


def test_selection_matches_sorted_tuples_with_ties():
    rng = np.random.default_rng(1)
    r = rng.integers(0, 20, 500).astype(float)     # many ties
    caug = rng.integers(0, 30, 500).astype(float)
    proj, elite = priest.select(r, caug, 300, 40)
    ref_proj = [i for _, i in sorted((r[i], i) for i in range(500))][:300]
    ref_elite = [i for _, i in sorted((caug[i], i) for i in ref_proj)][:40]
    np.testing.assert_array_equal(proj, ref_proj)
    np.testing.assert_array_equal(elite, ref_elite)


def test_refit_uniform_weights_is_the_elite_sample_mean_and_covariance():
    # gamma -> infinity gives uniform weights; sigma_lr = 1 replaces the old moments (CEM)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(50, 7))
    caug = rng.uniform(0, 10, 50)
    elite = np.arange(10, 45)
    mu, sig, best, c = priest.refit(X, caug, elite, np.zeros(7), np.eye(7), gamma=1e30, sig=1.0)
    np.testing.assert_allclose(mu, X[elite].mean(0), atol=1e-12)
    np.testing.assert_allclose(sig, np.cov(X[elite].T, bias=True), atol=1e-12)
    # the learning rate mixes old and new moments
    mu2, sig2, _, _ = priest.refit(X, caug, elite, np.ones(7), 2 * np.eye(7), gamma=1e30, sig=0.25)
    np.testing.assert_allclose(mu2, 0.75 + 0.25 * X[elite].mean(0), atol=1e-12)
    # the covariance is taken about the NEW mean (eq. update_covariance): by the
    # parallel-axis identity that is the sample covariance plus the mean shift
    m = X[elite].mean(0)
    shift = np.outer(m - mu2, m - mu2)
    np.testing.assert_allclose(sig2, 1.5 * np.eye(7) + 0.25 * (np.cov(X[elite].T, bias=True) + shift),
                               atol=1e-12)
    np.testing.assert_array_equal(best, X[elite[0]])


def test_refit_weights_favour_the_cheaper_elite_by_exp_of_the_cost_gap():
    """Two elites whose augmented costs differ by gamma ln 3 carry weights 1 and 1/3
    (the cheaper one heavier: Algorithm 3's update concentrates on good samples). With
    sigma_lr = 1 the new mean is (3 x1 + x2) / 4 and, with d = x1 - x2, the new
    covariance about it is (3 (d/4)(d/4)^T + (3d/4)(3d/4)^T) / 4 = 3/16 d d^T. The
    printed exponent's sign would give (x1 + 3 x2) / 4 instead; this case tells the
    two apart, where uniform weights cannot."""
    rng = np.random.default_rng(5)
    for gamma in (1.0, 0.37, 12.0):
        X = rng.normal(size=(6, 5))
        x1, x2 = X[4], X[1]
        caug = rng.uniform(50, 60, 6)
        caug[4] = 3.25
        caug[1] = 3.25 + gamma * np.log(3.0)
        elite = np.array([4, 1])  # ascending c_aug, as select() returns them
        mu, sig, best, c = priest.refit(X, caug, elite, np.full(5, 9.0), 7 * np.eye(5),
                                        gamma=gamma, sig=1.0)
        d = x1 - x2
        np.testing.assert_allclose(mu, (3 * x1 + x2) / 4, atol=1e-12)
        np.testing.assert_allclose(sig, 3.0 / 16.0 * np.outer(d, d), atol=1e-12)
        np.testing.assert_array_equal(best, x1)
        assert c == 3.25
        # half a step: the old moments enter with weight 1/2, the covariance is about
        # the blended mean m, so each elite's deviation is x - m
        mu_h, sig_h, _, _ = priest.refit(X, caug, elite, np.full(5, 9.0), 7 * np.eye(5),
                                         gamma=gamma, sig=0.5)
        m = 0.5 * 9.0 + 0.5 * (3 * x1 + x2) / 4
        np.testing.assert_allclose(mu_h, m, atol=1e-12)
        cov = (3 * np.outer(x1 - m, x1 - m) + np.outer(x2 - m, x2 - m)) / 4
        np.testing.assert_allclose(sig_h, 3.5 * np.eye(5) + 0.5 * cov, atol=1e-12)


def _fit(n_p, T, pos):
    """Degree-10 Bernstein coefficients [dim][11] of a polynomial sampled at the grid."""
    from oracle import am
    P, _, _ = am.bernstein(n_p, T)
    return np.linalg.lstsq(P, pos, rcond=None)[0].T


def _batch(dim, n_p, T, start, goal):
    import types
    return types.SimpleNamespace(dim=dim, n_steps=np.array([n_p]), duration=np.array([T]),
                                 start=np.array([start], float), goal=np.array([goal], float))


def test_curvature_of_a_parabola_is_its_closed_form():
    """p(t) = (t, t^2): kappa = 2 / (1 + 4 t^2)^1.5, and ||p''||^2 = 4, so
    c_1 = sum_t (4 + w 4 / (1 + 4 t^2)^3); the same curve in a tilted 3D plane
    gives the same sum."""
    n_p, T = 60, 3.0
    t = np.linspace(0.0, T, n_p)
    closed = (4.0 + 0.7 * 4.0 / (1.0 + 4.0 * t ** 2) ** 3).sum()
    b2 = _batch(2, n_p, T, [0, 0], [1, 1])
    X = _fit(n_p, T, np.stack([t, t ** 2], 1))
    _, c = priest.costs(b2, X.reshape(1, -1), np.zeros((1, 3)), w_r=0.0, w_curv=0.7)
    np.testing.assert_allclose(c[0], closed, rtol=1e-9)
    e1 = np.array([2.0, 1.0, 2.0]) / 3.0
    e2 = np.array([1.0, -2.0, 0.0]) / np.sqrt(5.0)
    X3 = _fit(n_p, T, t[:, None] * e1 + (t ** 2)[:, None] * e2)
    b3 = _batch(3, n_p, T, [0, 0, 0], [1, 1, 1])
    _, c3 = priest.costs(b3, X3.reshape(1, -1), np.zeros((1, 3)), w_r=0.0, w_curv=0.7)
    np.testing.assert_allclose(c3[0], closed, rtol=1e-9)


def test_curvature_vanishes_on_a_straight_line_with_varying_speed():
    """p(t) = (t^2, 2 t^2): p' and p'' are parallel, so c_kappa = 0 and only
    ||p''||^2 = 4 + 16 remains; at t = 0 the speed is 0 and the term is 0."""
    n_p, T = 40, 2.0
    t = np.linspace(0.0, T, n_p)
    X = _fit(n_p, T, np.stack([t ** 2, 2 * t ** 2], 1))
    _, c = priest.costs(_batch(2, n_p, T, [0, 0], [1, 1]), X.reshape(1, -1), np.zeros((1, 3)),
                        w_r=0.0, w_curv=5.0)
    np.testing.assert_allclose(c[0], 20.0 * n_p, rtol=1e-9)


def test_path_distance_of_offset_and_overshooting_lines():
    """Path start (0, 0) -> goal (10, 0); p(t) = (-2 + 14 t / T, h): distance h over
    the segment, and the distance to the nearer end point beyond it."""
    n_p, T, h = 50, 5.0, 1.5
    t = np.linspace(0.0, T, n_p)
    x = -2.0 + 14.0 * t / T
    d = np.where(x < 0, np.hypot(x, h), np.where(x > 10, np.hypot(x - 10, h), h))
    X = _fit(n_p, T, np.stack([x, np.full(n_p, h)], 1))
    b = _batch(2, n_p, T, [0, 0], [10, 0])
    _, c0 = priest.costs(b, X.reshape(1, -1), np.zeros((1, 3)), w_r=0.0)
    _, c = priest.costs(b, X.reshape(1, -1), np.zeros((1, 3)), w_r=0.0, w_path=2.0)
    np.testing.assert_allclose(c0[0], 0.0, atol=1e-9)       # straight line, constant speed
    np.testing.assert_allclose(c[0] - c0[0], 2.0 * d.sum(), rtol=1e-9)
    # 3D: the same line lifted by a perpendicular offset in z adds in quadrature
    X3 = _fit(n_p, T, np.stack([x, np.full(n_p, h), np.full(n_p, 2.0)], 1))
    b3 = _batch(3, n_p, T, [0, 0, 0], [10, 0, 0])
    _, c3 = priest.costs(b3, X3.reshape(1, -1), np.zeros((1, 3)), w_r=0.0, w_path=1.0)
    d3 = np.where(x < 0, np.sqrt(x ** 2 + h ** 2 + 4), np.where(
        x > 10, np.sqrt((x - 10) ** 2 + h ** 2 + 4), np.hypot(h, 2.0)))
    np.testing.assert_allclose(c3[0], d3.sum(), rtol=1e-9)


def test_decentralised_step_is_independent_steps_per_group():
    """D-PRIEST with two distributions = two single-distribution steps, each on its
    own group of samples (draws given); n_dist = 1 reproduces step()."""
    from paper_2408_10731_b300 import scenes
    Bg, D = 6, 33
    c_full = scenes.config3(0, n_traj=2 * Bg)
    c_half = scenes.config3(0, n_traj=Bg)
    cfg = priest.SamplerConfig(n_inner=3, n_proj=4, n_elite=2, w_curv=0.5, w_path=0.2)
    z = scenes.normal_draws(5, (2 * Bg, D)).astype(np.float64)
    rng = np.random.default_rng(1)
    mus = np.stack([c_full["mu0"], c_full["mu0"] + rng.normal(size=D)]).astype(np.float64)
    sigmas = np.stack([np.eye(D) * 2.0, np.eye(D) * 0.5])
    m = priest.step_multi(c_full["batch"], cfg, 0, mus, sigmas, z=z)
    for g in range(2):
        s = priest.step(c_half["batch"], cfg, 0, mus[g], sigmas[g], z=z[g * Bg:(g + 1) * Bg])
        np.testing.assert_array_equal(m["elite_idx"][g], s["elite_idx"])
        np.testing.assert_array_equal(m["proj_idx"][g], s["proj_idx"])
        np.testing.assert_allclose(m["mu"][g], s["mu"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(m["sigma"][g], s["sigma"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(m["cost_aug"][g * Bg:(g + 1) * Bg], s["cost_aug"], rtol=1e-12)
    one = priest.step_multi(c_half["batch"], cfg, 0, mus[:1], sigmas[:1], z=z[:Bg])
    s0 = priest.step(c_half["batch"], cfg, 0, mus[0], sigmas[0], z=z[:Bg])
    np.testing.assert_array_equal(one["elite_idx"][0], s0["elite_idx"])
    np.testing.assert_allclose(one["best"][0], s0["best"], rtol=1e-12)
