"""The seeded input generators (inputs only; none of the method's arithmetic): the
grazing scenes behind the cull tests and the held-out scenes of the default bench."""
import numpy as np

from paper_2408_10731_b300 import scenes


def _normalised_distances(b):
    """|u| = ||(p - c - v t) / a|| of the straight-line path's grid points, all problems."""
    out = []
    for p in range(b.n_problems):
        n_p, T = int(b.n_steps[p]), float(b.duration[p])
        t = np.arange(n_p) * T / (n_p - 1)
        path = b.start[p][None] + (t / T)[:, None] * (b.goal[p] - b.start[p])[None]
        c, a, v = (np.asarray(x, np.float64) for x in b.obstacles(p))
        if len(c) == 0:
            continue
        u = (path[:, None, :] - c[None] - v[None] * t[:, None, None]) / a[None]
        out.append(np.sqrt((u ** 2).sum(-1)).ravel())
    return np.concatenate(out)


def test_grazing_scenes_have_the_asked_counts_and_graze_the_path():
    counts, horizons = (1, 2, 7, 64, 65), (33, 100)
    for dim in (2, 3):
        b = scenes.grazing(3, n_obstacles=counts, n_steps=horizons, inits=2, dim=dim)
        assert b.dim == dim and b.n_problems == len(counts) * len(horizons)
        got = [(b.n_obstacles(p), int(b.n_steps[p])) for p in range(b.n_problems)]
        assert got == [(no, npt) for no in counts for npt in horizons]
        assert np.all(b.semi_axes >= 0.2 - 1e-6) and np.all(b.semi_axes <= 0.8 + 1e-6)
        assert np.all(np.linalg.norm(b.velocities, axis=1) <= 0.5 + 1e-6)
        # inputs are FP32-exact, so both sides of a parity test see the same numbers
        for x in (b.centers, b.semi_axes, b.velocities, b.xi0):
            assert np.array_equal(np.asarray(x, np.float64), np.asarray(x, np.float32).astype(np.float64))
        r = _normalised_distances(b)
        near = np.mean(np.abs(r - 1.0) < 0.05)
        assert 0.005 < near < 0.2, near  # many grid points sit close to an ellipse boundary
        assert np.mean(r < 1.0) > 0.0    # and some lie inside one


def test_grazing_scenes_are_seeded():
    a, b = scenes.grazing(5), scenes.grazing(5)
    assert np.array_equal(a.centers, b.centers) and np.array_equal(a.xi0, b.xi0)
    c = scenes.grazing(6)
    assert not np.array_equal(a.centers, c.centers)


def test_held_out_scenes_keep_start_and_goal_free():
    b = scenes.ellipse_scenes(99, 16, inits=8)
    assert b.n_problems == 16 and b.n_traj == 128 and np.all(b.n_steps == 100)
    T = float(b.duration[0])
    for p in range(b.n_problems):
        c, a, v = (np.asarray(x, np.float64) for x in b.obstacles(p))
        assert len(c) == 50
        assert np.all((((b.start[p] - c) / a) ** 2).sum(1) > 1.0)
        assert np.all((((b.goal[p] - (c + v * T)) / a) ** 2).sum(1) > 1.0)
