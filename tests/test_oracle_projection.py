"""Pins of the oracle's closed-form alpha/beta/d steps (Algorithm 2 lines 4-5).

Each projection subproblem is minimised independently by brute force on a
dense (alpha[, beta], d) grid refined around its best point; the oracle's
closed form must match it. Also: the closed form d = max(1, ||u||) (eq.
d_max), targets on or outside every ellipse, the v/a targets inside their
balls, and the atan2(0, 0) reading.
"""
import numpy as np
import pytest

from oracle import am


def _grid_min_2d(xt, ax, d_lo, d_hi, bound=1.0):
    """argmin over (alpha, d) of ||xt - d * bound * (a cos al, b sin al)||, coarse-to-fine."""
    al_c, al_w, d_c, d_w = 0.0, np.pi, 0.5 * (d_lo + d_hi), 0.5 * (d_hi - d_lo)
    for _ in range(7):
        al = al_c + np.linspace(-al_w, al_w, 801)
        d = np.clip(d_c + np.linspace(-d_w, d_w, 801), d_lo, d_hi)
        A, D = np.meshgrid(al, d, indexing="ij")
        gx = D * bound * ax[0] * np.cos(A); gy = D * bound * ax[1] * np.sin(A)
        f = (xt[0] - gx) ** 2 + (xt[1] - gy) ** 2
        k = np.unravel_index(np.argmin(f), f.shape)
        al_c, d_c = A[k], D[k]
        al_w *= 0.02; d_w *= 0.02
    return np.array([d_c * bound * ax[0] * np.cos(al_c), d_c * bound * ax[1] * np.sin(al_c)])


def _grid_min_3d(xt, ax, d_lo, d_hi, bound=1.0):
    al_c, al_w, be_c, be_w = 0.0, np.pi, 0.5 * np.pi, 0.5 * np.pi
    d_c, d_w = 0.5 * (d_lo + d_hi), 0.5 * (d_hi - d_lo)
    for _ in range(8):
        al = al_c + np.linspace(-al_w, al_w, 121)
        be = np.clip(be_c + np.linspace(-be_w, be_w, 121), 0.0, np.pi)
        d = np.clip(d_c + np.linspace(-d_w, d_w, 121), d_lo, d_hi)
        A, Bt, D = np.meshgrid(al, be, d, indexing="ij")
        g = np.stack([D * bound * ax[0] * np.cos(A) * np.sin(Bt),
                      D * bound * ax[1] * np.sin(A) * np.sin(Bt),
                      D * bound * ax[2] * np.cos(Bt)])
        f = ((xt[:, None, None, None] - g) ** 2).sum(0)
        k = np.unravel_index(np.argmin(f), f.shape)
        al_c, be_c, d_c = A[k], Bt[k], D[k]
        al_w *= 0.06; be_w *= 0.06; d_w *= 0.06
    return np.array([d_c * bound * ax[0] * np.cos(al_c) * np.sin(be_c),
                     d_c * bound * ax[1] * np.sin(al_c) * np.sin(be_c),
                     d_c * bound * ax[2] * np.cos(be_c)])


def test_obstacle_projection_2d_dense_grid():
    rng = np.random.default_rng(1)
    for _ in range(25):
        ax = rng.uniform(0.2, 0.8, 2)
        xt = rng.uniform(-1.2, 1.2, 2) * ax * 1.2
        g = am.project_obstacle(xt, ax)
        # the alternating alpha-then-d steps: in normalised coordinates u = x~/axes
        # they are the Euclidean projection onto {||u|| >= 1}
        u = xt / ax
        ref_u = u * max(1.0, 1.0 / np.linalg.norm(u))
        np.testing.assert_allclose(g / ax, ref_u, atol=1e-12)
        # brute force of the same subproblem in normalised coordinates
        gb = _grid_min_2d(u, np.ones(2), 1.0, 4.0)
        np.testing.assert_allclose(g / ax, gb, atol=2e-6)


def test_obstacle_projection_circle_is_nearest_boundary_point():
    # for circles the target is the exact nearest boundary point in metres
    rng = np.random.default_rng(2)
    for _ in range(20):
        r = rng.uniform(0.3, 0.6)
        xt = rng.uniform(-0.6, 0.6, 2)
        g = am.project_obstacle(xt, np.array([r, r]))
        gb = _grid_min_2d(xt, np.array([r, r]), 1.0, 4.0)
        np.testing.assert_allclose(g, gb, atol=2e-6)
        if np.linalg.norm(xt) < r:
            np.testing.assert_allclose(g, xt / np.linalg.norm(xt) * r, atol=1e-12)
        else:
            np.testing.assert_allclose(g, xt, atol=1e-12)


def test_obstacle_projection_3d_dense_grid():
    rng = np.random.default_rng(3)
    for _ in range(8):
        ax = rng.uniform(0.1, 0.6, 3)
        xt = rng.uniform(-1.0, 1.0, 3) * ax
        g = am.project_obstacle(xt, ax)
        u = xt / ax
        np.testing.assert_allclose(g / ax, u * max(1.0, 1.0 / np.linalg.norm(u)), atol=1e-12)
        gb = _grid_min_3d(u, np.ones(3), 1.0, 4.0)
        np.testing.assert_allclose(g / ax, gb, atol=5e-6)


def test_targets_on_or_outside_ellipse_and_d_max():
    rng = np.random.default_rng(4)
    for dim in (2, 3):
        for _ in range(200):
            ax = rng.uniform(0.1, 1.0, dim)
            xt = rng.normal(size=dim) * ax * rng.uniform(0.01, 3.0)
            g = am.project_obstacle(xt, ax)
            assert np.linalg.norm(g / ax) >= 1.0 - 1e-12
            # eq. d_max: d = max(1, ||x~ / axes||), g - o = d * unit direction
            d = max(1.0, np.linalg.norm(xt / ax))
            np.testing.assert_allclose(np.linalg.norm(g / ax), d, rtol=1e-12)


def test_atan2_zero_reading():
    # a point exactly at the centre: atan2(0, 0) = 0, pushed along +x by the semi-axis
    np.testing.assert_allclose(am.project_obstacle(np.zeros(2), np.array([0.3, 0.7])),
                               [0.3, 0.0], atol=0)
    np.testing.assert_allclose(am.project_obstacle(np.zeros(3), np.array([0.3, 0.7, 0.2])),
                               [0.0, 0.0, 0.2], atol=1e-17)


@pytest.mark.parametrize("dim", [2, 3])
def test_bound_projection_is_ball_projection(dim):
    rng = np.random.default_rng(5)
    for _ in range(30):
        w = rng.normal(size=dim) * rng.uniform(0.1, 3.0)
        vmax = 1.5
        g = am.project_bound(w, vmax)
        ref = w * min(1.0, vmax / np.linalg.norm(w))
        np.testing.assert_allclose(g, ref, atol=1e-12)
        assert np.linalg.norm(g) <= vmax * (1 + 1e-12)
    # brute force in 2D (alpha, d in [0, 1])
    for _ in range(10):
        w = rng.normal(size=2) * 2.0
        gb = _grid_min_2d(w, np.ones(2), 0.0, 1.0, bound=1.5)
        np.testing.assert_allclose(am.project_bound(w, 1.5), gb, atol=2e-6)
    np.testing.assert_array_equal(am.project_bound(np.zeros(dim), 1.5), np.zeros(dim))
