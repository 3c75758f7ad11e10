"""Pins of the warm-start oracle against library routines, finite differences and
special cases."""
import numpy as np
import torch

from oracle import mlp
from paper_2408_10731_b300 import scenes


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for name, shape in mlp.SHAPES:
        fan_in = shape[1] if len(shape) == 2 else 256
        out.append(rng.uniform(-1, 1, int(np.prod(shape))) * scale / np.sqrt(fan_in))
    return np.concatenate(out)


def test_gelu_matches_torch_tanh_form():
    z = np.linspace(-6, 6, 2001)
    ref = torch.nn.functional.gelu(torch.tensor(z, dtype=torch.float64), approximate="tanh")
    np.testing.assert_allclose(mlp.gelu(z), ref.numpy(), atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h),
                               atol=1e-8)


def test_backward_against_central_differences():
    rng = np.random.default_rng(3)
    params = _params(1)
    X = rng.normal(size=(6, mlp.IN))
    targets = rng.normal(size=(6, mlp.HEADS, mlp.D22))
    n_labels = np.array([1, 3, 0, 8, 2, 1])
    loss, g = mlp.backward(params, X, targets, n_labels)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    # make sure every tensor is probed
    o = 0
    for _, shape in mlp.SHAPES:
        idx = np.append(idx, o + rng.integers(0, int(np.prod(shape)), 3))
        o += int(np.prod(shape))
    h = 1e-6
    for i in idx:
        p1, p2 = params.copy(), params.copy()
        p1[i] += h; p2[i] -= h
        fd = (mlp.loss_wta(mlp.forward(p1, X)["Y"], targets, n_labels)[0]
              - mlp.loss_wta(mlp.forward(p2, X)["Y"], targets, n_labels)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_adamw_matches_torch():
    rng = np.random.default_rng(4)
    params = _params(2)
    m = np.zeros_like(params); v = np.zeros_like(params)
    tp = [torch.tensor(mlp.unpack(params)[n].copy(), dtype=torch.float64, requires_grad=True)
          for n, _ in mlp.SHAPES]
    decay = [t for (n, _), t in zip(mlp.SHAPES, tp) if n.startswith("W")]
    keep = [t for (n, _), t in zip(mlp.SHAPES, tp) if n.startswith("b")]
    opt = torch.optim.AdamW([{"params": decay, "weight_decay": 0.01},
                             {"params": keep, "weight_decay": 0.0}], lr=3e-3,
                            betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 5):
        g = rng.normal(size=params.shape)
        params, m, v = mlp.adamw(params, g, m, v, t, lr=3e-3, wd=0.01)
        gd = mlp.unpack(g)
        for (n, _), ti in zip(mlp.SHAPES, tp):
            ti.grad = torch.tensor(gd[n], dtype=torch.float64)
        opt.step()
    ref = np.concatenate([ti.detach().numpy().ravel() for ti in tp])
    np.testing.assert_allclose(params, ref, rtol=1e-12, atol=1e-14)


def test_features_nearest_obstacles_and_padding():
    b = scenes.config2(0, n_scenes=3, inits=1)
    X, line = mlp.features(b)
    for p in range(3):
        c, a, v = b.obstacles(p)
        s, g = b.start[p], b.goal[p]
        # brute-force distance to the segment on a fine grid
        pts = s[None] + np.linspace(0, 1, 20001)[:, None] * (g - s)[None]
        brute = np.sqrt(((c[:, None, :] - pts[None]) ** 2).sum(-1)).min(1)
        d = mlp.segment_distance(c, s, g)
        np.testing.assert_allclose(d, brute, atol=1e-3)
        order = np.argsort(d, kind="stable")[:50]
        got_c = X[p, 4:4 + 6 * 50].reshape(50, 6)[:, :2] / 0.1 + s
        np.testing.assert_allclose(got_c, c[order], atol=1e-12)
        assert np.all(np.diff(d[order]) >= 0)
        np.testing.assert_array_equal(X[p, 4 + 6 * 50:], 0.0)  # 14 absent slots
        np.testing.assert_allclose(X[p, 2:4], 0.1 * (g - s))
        np.testing.assert_allclose(line[p].reshape(2, 11), scenes.straight_line_coeffs(s, g))


def test_wta_loss_special_cases():
    rng = np.random.default_rng(5)
    t = rng.normal(size=(2, mlp.HEADS, mlp.D22))
    # every head equal to the label: zero loss and gradient
    Y = np.tile(t[:, :1], (1, mlp.HEADS, 1)).reshape(2, mlp.OUT)
    loss, dY = mlp.loss_wta(Y, t, np.array([1, 1]))
    assert loss == 0 and np.all(dY == 0)
    # identical heads at distance e from one label: loss = (1 + 0.05) * |e|^2
    e = rng.normal(size=mlp.D22)
    Y = np.tile((t[0, 0] + e)[None], (mlp.HEADS, 1)).reshape(1, mlp.OUT)
    loss, _ = mlp.loss_wta(Y, t[:1], np.array([1]))
    np.testing.assert_allclose(loss, 1.05 * (e @ e), rtol=1e-12)
