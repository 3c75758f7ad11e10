"""Oracle of the learned warm start -- TEST INFRASTRUCTURE ONLY, FP64 numpy.

The thesis names learning-based methods as future work and prints no network;
this oracle restates the library's documented design (features, MLP
388-256-256-256-176 with tanh-form GELU, winner-takes-all loss, AdamW) as plain
array code, so that the GPU's BF16 kernels can be checked against it.

Parity status: gelu pinned against torch.nn.functional.gelu (tanh form);
backward pinned by central finite differences; adamw pinned against
torch.optim.AdamW; features pinned by a brute-force point-to-segment distance
and the stated ordering; loss_wta pinned by special cases.
"""
from __future__ import annotations

import numpy as np

IN, HID, OUT, HEADS, D22, NEAR = 388, 256, 176, 8, 22, 64
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, HID)), ("b3", (HID,)), ("W4", (OUT, HID)), ("b4", (OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[n], np.float64).ravel() for n, _ in SHAPES])


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(np.sqrt(2.0 / np.pi) * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    k0 = np.sqrt(2.0 / np.pi)
    t = np.tanh(k0 * (z + 0.044715 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * k0 * (1.0 + 3 * 0.044715 * z * z)


def segment_distance(c, s, g):
    """Distance of points c [n,2] to the segment s->g."""
    d = g - s
    L2 = float(d @ d)
    u = np.clip(((c - s) @ d) / L2, 0.0, 1.0) if L2 > 0 else np.zeros(len(c))
    return np.linalg.norm(c - (s + u[:, None] * d), axis=1)


def features(batch):
    """[n_problems, 388] features and [n_problems, 22] straight-line coefficients."""
    n = batch.n_problems
    X = np.zeros((n, IN))
    line = np.zeros((n, D22))
    for p in range(n):
        s, g = batch.start[p].astype(np.float64), batch.goal[p].astype(np.float64)
        c, a, v = batch.obstacles(p)
        X[p, 2:4] = 0.1 * (g - s)
        if len(c):
            dist = segment_distance(c, s, g)
            order = np.lexsort((np.arange(len(c)), dist))[:NEAR]
            for slot, j in enumerate(order):
                X[p, 4 + 6 * slot:4 + 6 * slot + 6] = [0.1 * (c[j, 0] - s[0]), 0.1 * (c[j, 1] - s[1]),
                                                       a[j, 0], a[j, 1], v[j, 0], v[j, 1]]
        i = np.arange(11) / 10.0
        line[p] = np.concatenate([s[0] + (g[0] - s[0]) * i, s[1] + (g[1] - s[1]) * i])
    return X, line


def forward(params, X):
    P = unpack(params)
    c = {"X": np.asarray(X, np.float64)}
    h = c["X"]
    for L in (1, 2, 3):
        z = h @ P[f"W{L}"].T + P[f"b{L}"]
        c[f"Z{L}"] = z
        h = gelu(z)
        c[f"H{L}"] = h
    c["Y"] = h @ P["W4"].T + P["b4"]
    return c


def loss_wta(Y, targets, n_labels):
    """Winner-takes-all loss over K = 8 heads and its gradient dL/dY."""
    Y = np.asarray(Y, np.float64)
    total = max(1, int(np.sum(n_labels)))
    dY = np.zeros_like(Y)
    loss = 0.0
    for s in range(Y.shape[0]):
        y = Y[s].reshape(HEADS, D22)
        for m in range(int(n_labels[s])):
            t = targets[s, m]
            d = ((y - t[None]) ** 2).sum(1)
            k = int(np.argmin(d))
            loss += d[k] + 0.05 * d.mean()
            coef = np.full(HEADS, 0.05 / HEADS)
            coef[k] += 1.0
            dY[s] += (2.0 * coef[:, None] * (y - t[None])).ravel() / total
    return loss / total, dY


def backward(params, X, targets, n_labels):
    P = unpack(params)
    c = forward(params, X)
    loss, dY = loss_wta(c["Y"], targets, n_labels)
    g = {"W4": dY.T @ c["H3"], "b4": dY.sum(0)}
    dH = dY @ P["W4"]
    for L in (3, 2, 1):
        dZ = dH * gelu_grad(c[f"Z{L}"])
        prev = c[f"H{L - 1}"] if L > 1 else c["X"]
        g[f"W{L}"] = dZ.T @ prev
        g[f"b{L}"] = dZ.sum(0)
        dH = dZ @ P[f"W{L}"]
    return loss, pack(g)


def adamw(params, grads, m, v, t, lr, wd, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW step; decoupled decay only on the weight matrices."""
    params, m, v = params.copy(), m.copy(), v.copy()
    decay = np.concatenate([np.full(int(np.prod(s)), 1.0 if n.startswith("W") else 0.0)
                            for n, s in SHAPES])
    params = params - lr * wd * decay * params
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    params = params - lr * mh / (np.sqrt(vh) + eps)
    return params, m, v
