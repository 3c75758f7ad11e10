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
