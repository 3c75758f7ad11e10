"""GPU parity of the learned warm start (features, BF16 forward/backward on the
tcgen05 GEMMs, AdamW) against the FP64 oracle, and the gain of a trained
network over random initialisation on held-out scenes."""
import numpy as np
import pytest

from oracle import mlp
from paper_2408_10731_b300 import scenes

pytestmark = pytest.mark.gpu


def _bf16(x):
    import torch
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _cos(a, b):
    return float(a.ravel() @ b.ravel() / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))


def _setup(n_scenes=64, seed=0):
    import torch
    from paper_2408_10731_b300 import warmstart
    b = scenes.ellipse_scenes(seed, n_scenes)
    ws = warmstart.WarmStart(max_rows=256)
    params = _bf16(warmstart.init_params(3) * 4.0)  # larger last layer: non-trivial outputs
    ws.set_params(params)
    X, line = ws.features(b)
    return torch, warmstart, b, ws, params.astype(np.float64), X, line


def test_features_match_oracle():
    torch, warmstart, b, ws, params, X, line = _setup()
    Xg = X.float().cpu().numpy()
    Xo, lo = mlp.features(b)
    np.testing.assert_allclose(line.cpu().numpy(), lo, atol=1e-5)
    np.testing.assert_allclose(Xg[:, :4], _bf16(Xo[:, :4]), atol=0)
    for p in range(b.n_problems):
        c, a, v = b.obstacles(p)
        d = mlp.segment_distance(c, b.start[p], b.goal[p])
        # the GPU's slots: identify each slot's obstacle by its exact (bf16) feature values
        slots = Xg[p, 4:4 + 6 * 50].reshape(50, 6)
        ref = _bf16(np.column_stack([0.1 * (c - b.start[p]), a, v]))
        chosen = [int(np.nonzero(np.all(ref == s, axis=1))[0][0]) for s in slots]
        assert sorted(chosen) == list(range(50))            # every obstacle once (50 < 64)
        assert np.all(np.diff(d[chosen]) >= -1e-6)          # ascending distance
        np.testing.assert_array_equal(Xg[p, 4 + 6 * 50:], 0.0)
    ws.close()


def test_forward_matches_oracle_bf16():
    torch, warmstart, b, ws, params, X, line = _setup()
    prop = ws.forward(X, line).cpu().numpy().reshape(b.n_problems, -1)
    ws.sync()
    Xo = X.float().cpu().numpy().astype(np.float64)[:, :mlp.IN]
    Y = mlp.forward(params, Xo)["Y"] + np.tile(line.cpu().numpy(), (1, 8))
    assert _rel(prop, Y) <= 2e-2 and _cos(prop - np.tile(line.cpu().numpy(), (1, 8)),
                                          Y - np.tile(line.cpu().numpy(), (1, 8))) >= 0.999
    ws.close()


def test_gradients_and_adamw_match_oracle():
    torch, warmstart, b, ws, params, X, line = _setup()
    rng = np.random.default_rng(1)
    P = b.n_problems
    targets = rng.normal(0, 0.5, (P, 8, 22)).astype(np.float32)
    n_labels = rng.integers(0, 9, P).astype(np.int32)
    tt = torch.as_tensor(targets, device="cuda")
    nt = torch.as_tensor(n_labels, device="cuda")
    g, loss = ws.gradients(X, tt, nt)
    Xo = X.float().cpu().numpy().astype(np.float64)[:, :mlp.IN]
    lo, go = mlp.backward(params, Xo, targets.astype(np.float64), n_labels)
    assert abs(loss - lo) <= 2e-2 * abs(lo)
    gd, od = mlp.unpack(g.astype(np.float64)), mlp.unpack(go)
    for name, _ in mlp.SHAPES:
        assert _rel(gd[name], od[name]) <= 2e-2, (name, _rel(gd[name], od[name]))
        assert _cos(gd[name], od[name]) >= 0.999, (name, _cos(gd[name], od[name]))
    # one AdamW step on the GPU equals the oracle's step from the GPU's own gradients
    ws.set_params(params.astype(np.float32))
    ws.train_step(X, tt, nt, 1e-3, 1e-2)
    ws.sync()
    new = ws.get_params().astype(np.float64)
    ref, _, _ = mlp.adamw(params, g.astype(np.float64), np.zeros_like(params),
                          np.zeros_like(params), 1, 1e-3, 1e-2)
    np.testing.assert_allclose(new, ref, rtol=1e-5, atol=1e-7)
    ws.close()


def test_fp32_operand_gradients_match_oracle_to_1e4():
    """The debug instantiation with FP32 operands (CUDA-core GEMMs, FP32 activations):
    loss and every parameter tensor's gradient within 1e-4 relative of the FP64
    oracle, tight enough that a dropped term on part of a tensor (a bias gradient
    row, a GELU' factor) shows, where the BF16 check's 2e-2 could hide it."""
    torch, warmstart, b, ws, params, X, line = _setup()
    rng = np.random.default_rng(2)
    P = b.n_problems
    targets = rng.normal(0, 0.5, (P, 8, 22)).astype(np.float32)
    n_labels = rng.integers(0, 9, P).astype(np.int32)
    g, loss = ws.gradients_fp32(X, torch.as_tensor(targets, device="cuda"),
                                torch.as_tensor(n_labels, device="cuda"))
    Xo = X.float().cpu().numpy().astype(np.float64)[:, :mlp.IN]
    lo, go = mlp.backward(params, Xo, targets.astype(np.float64), n_labels)
    assert abs(loss - lo) <= 1e-5 * abs(lo), (loss, lo)
    gd, od = mlp.unpack(g.astype(np.float64)), mlp.unpack(go)
    for name, _ in mlp.SHAPES:
        assert _rel(gd[name], od[name]) <= 1e-4, (name, _rel(gd[name], od[name]))
        # per row as well: a wrong row of a matrix (one unit's gradient) cannot hide
        rows = np.atleast_2d(gd[name])
        orow = np.atleast_2d(od[name])
        scale = np.abs(orow).max()
        assert np.abs(rows - orow).max() <= 1e-4 * scale, (name, np.abs(rows - orow).max() / scale)
    ws.close()


def test_training_checkpoint_resumes_bitwise(tmp_path):
    """Train 3 AdamW steps, checkpoint (weights, moments, step) to a file, train 4
    more; a fresh handle that loads the file and trains the same 4 steps ends with
    bitwise the same weights and moments. The restored moments and step are the
    saved ones, and one more step from them equals the oracle's AdamW step."""
    torch, warmstart, b, ws, params, X, line = _setup()
    rng = np.random.default_rng(4)
    P = b.n_problems
    batches = [(torch.as_tensor(rng.normal(0, 0.5, (P, 8, 22)).astype(np.float32), device="cuda"),
                torch.as_tensor(rng.integers(1, 9, P).astype(np.int32), device="cuda"))
               for _ in range(7)]
    for tt, nt in batches[:3]:
        ws.train_step(X, tt, nt, 1e-3, 1e-2)
    ws.sync()
    path = tmp_path / "ws.ckpt"
    ws.save_checkpoint(path, lr=1e-3, weight_decay=1e-2, next_batch=3)
    saved = ws.get_state()
    assert saved[3] == 3 and np.any(saved[1] != 0) and np.all(saved[2] >= 0)
    for tt, nt in batches[3:]:
        ws.train_step(X, tt, nt, 1e-3, 1e-2)
    ws.sync()
    direct = ws.get_state()
    ws.close()

    ws2 = warmstart.WarmStart(max_rows=256)
    ws2.set_params(warmstart.init_params(9))  # unrelated weights, overwritten by the load
    meta = ws2.load_checkpoint(path)
    assert meta == {"lr": 1e-3, "weight_decay": 1e-2, "next_batch": 3}
    back = ws2.get_state()
    for a, c in zip(back[:3], saved[:3]):
        np.testing.assert_array_equal(a, c)
    assert back[3] == 3
    # the next step from the restored state is the oracle's AdamW step (t = 4)
    g, _ = ws2.gradients(X, *batches[3])
    ref, _, _ = mlp.adamw(back[0].astype(np.float64), g.astype(np.float64),
                          back[1].astype(np.float64), back[2].astype(np.float64), 4, 1e-3, 1e-2)
    for tt, nt in batches[3:]:
        ws2.train_step(X, tt, nt, 1e-3, 1e-2)
        if tt is batches[3][0]:
            ws2.sync()
            np.testing.assert_allclose(ws2.get_params().astype(np.float64), ref, rtol=1e-5, atol=1e-7)
    ws2.sync()
    resumed = ws2.get_state()
    for a, c in zip(resumed[:3], direct[:3]):
        np.testing.assert_array_equal(a, c)
    assert resumed[3] == direct[3] == 7
    ws2.close()


def test_device_propose_matches_host_path_and_flags_bad_offsets():
    """traj_warmstart_propose (device inputs, no synchronisation) gives bitwise the
    features and proposals of traj_warmstart_features + traj_warmstart_forward;
    offsets outside the obstacle range are reported by the next sync."""
    torch, warmstart, b, ws, params, X, line = _setup()
    prop = ws.forward(X, line).cpu().numpy()
    st = ws.stage(b)
    out = ws.propose(st)
    ws.sync()
    np.testing.assert_array_equal(st["X"].float().cpu().numpy(), X.float().cpu().numpy())
    np.testing.assert_array_equal(st["line"].cpu().numpy(), line.cpu().numpy())
    np.testing.assert_array_equal(out.cpu().numpy(), prop)
    bad = dict(st)
    bad["offsets"] = st["offsets"].clone()
    bad["offsets"][-1] = st["n_obs"] + 5
    ws.propose(bad)
    from paper_2408_10731_b300.trajbatch import TrajBatchError
    with pytest.raises(TrajBatchError):
        ws.sync()
    ws.sync()  # the flag is cleared once reported
    ws.close()


def test_homotopy_signature_tells_the_sides_apart():
    """One static obstacle on the straight path from (0, 0) to (8, 8): a trajectory
    bending through (5, 3) keeps it on its left (bit set), one through (3, 5) on its
    right (bit clear); an obstacle far off the path's left is on the left of both.
    Random trajectories against a host evaluation of the same definition."""
    import dataclasses
    from paper_2408_10731_b300 import trajbatch as tb
    start, goal = np.array([0.0, 0.0]), np.array([8.0, 8.0])
    line = scenes.straight_line_coeffs(start, goal)
    bump = np.sin(np.pi * np.arange(11) / 10.0)  # zero at both ends
    right = line + 1.5 * np.stack([bump, -bump])
    left = line + 1.5 * np.stack([-bump, bump])
    b = scenes.Batch(dim=2, n_steps=np.array([100], np.int32), duration=np.array([10.0]),
                     start=start[None], goal=goal[None], offsets=np.array([0, 2], np.int32),
                     centers=np.array([[4.0, 4.0], [1.0, 7.0]], np.float32),
                     semi_axes=np.full((2, 2), 0.5, np.float32),
                     velocities=np.zeros((2, 2), np.float32),
                     traj_problem=np.zeros(2, np.int32),
                     xi0=scenes.f32(np.stack([right, left])), vmax=1e6, amax=1e6, rho=1.0)
    h = tb.from_batch(b)
    try:
        h.solve(0, -1.0)  # the initial coefficients are projected, not moved: compare as given
        sig = h.homotopy_signature()
        xi = h.get_trajectories()["xi"].astype(np.float64)
    finally:
        h.close()
    assert int(sig[0]) & 1 == 1 and int(sig[1]) & 1 == 0, sig
    assert int(sig[0]) & 2 == 2 and int(sig[1]) & 2 == 2, sig
    # random scenes: the same definition evaluated on the host from the GPU's coefficients
    rb = scenes.config2(4, n_scenes=4, inits=8)
    h = tb.from_batch(rb)
    try:
        h.solve(30, -1.0)
        sig = h.homotopy_signature()
        xi = h.get_trajectories()["xi"].astype(np.float64)
    finally:
        h.close()
    from oracle import am
    P, Pd, _ = am.bernstein(100, 10.0)
    t = np.linspace(0.0, 10.0, 100)
    checked = 0
    for k in range(rb.n_traj):
        p_ = rb.traj_problem[k]
        c, a, v = (np.asarray(x, np.float64) for x in rb.obstacles(p_))
        pos, vel = xi[k] @ P.T, xi[k] @ Pd.T  # [2, n_p]
        for j in range(c.shape[0]):
            o = c[j][:, None] + v[j][:, None] * t[None]
            d2 = (((pos - o) / a[j][:, None]) ** 2).sum(0)
            order = np.argsort(d2)
            if d2[order[1]] - d2[order[0]] < 1e-4 * max(1.0, d2[order[0]]):
                continue  # a near tie of the closest grid point: FP32 may pick the other
            ts = order[0]
            d, r = pos[:, ts] - o[:, ts], vel[:, ts] - v[j]
            cr = d[0] * r[1] - d[1] * r[0]
            if abs(cr) < 1e-4 * (np.linalg.norm(d) * np.linalg.norm(r) + 1e-12):
                continue
            assert ((int(sig[k]) >> j) & 1) == (1 if cr > 0 else 0), (k, j, cr)
            checked += 1
    assert checked > 1000
