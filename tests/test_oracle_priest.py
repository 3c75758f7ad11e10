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
