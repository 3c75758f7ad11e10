"""Learned warm start for the batched optimizer (binding and training pipeline).

The network, its features and loss run in the library's CUDA kernels
(traj_warmstart_*: tcgen05 BF16 GEMMs, fused GELU epilogues, AdamW); this
module marshals arguments and orchestrates:

  make_labels  -- solve many scenes from random initialisations with the
                  optimizer itself and keep, per scene, up to 8 solved
                  trajectories: one per homotopy class first (in order of
                  acceleration cost), then the cheapest others;
  train        -- epochs of shuffled minibatches through traj_warmstart_train_step;
  proposals    -- features -> network -> K = 8 initial coefficient sets per scene.

Without a trained network the solver's straight-line / random initialisations
remain the fallback; the optimizer's residual judges every proposal.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import scenes, trajbatch as tb

IN, IN_PAD, OUT, HEADS, D22 = 388, 400, 176, 8, 22
_vp, _ci, _cf = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
_READY = False


def _lib():
    global _READY
    lib = tb.load_library()
    if not _READY:
        lib.traj_warmstart_num_params.restype = _ci
        lib.traj_warmstart_create.argtypes = [_ci, _vp, ctypes.POINTER(_vp)]
        lib.traj_warmstart_destroy.argtypes = [_vp]
        lib.traj_warmstart_set_params.argtypes = [_vp, _vp]
        lib.traj_warmstart_get_params.argtypes = [_vp, _vp]
        lib.traj_warmstart_features.argtypes = [_vp, _ci, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        lib.traj_warmstart_forward.argtypes = [_vp, _ci, _vp, _vp, _vp]
        lib.traj_warmstart_propose.argtypes = [_vp, _ci, _ci] + [_vp] * 9
        lib.traj_warmstart_gradients.argtypes = [_vp, _ci, _vp, _vp, _vp, _vp, _vp]
        lib.traj_warmstart_gradients_fp32.argtypes = [_vp, _ci, _vp, _vp, _vp, _vp, _vp]
        lib.traj_warmstart_train_step.argtypes = [_vp, _ci, _vp, _vp, _vp, _cf, _cf, _vp]
        lib.traj_warmstart_sync.argtypes = [_vp]
        lib.traj_warmstart_get_state.argtypes = [_vp, _vp, _vp, _vp, ctypes.POINTER(_ci)]
        lib.traj_warmstart_set_state.argtypes = [_vp, _vp, _vp, _vp, _ci]
        lib.traj_get_accel_cost.argtypes = [_vp, _vp]
        for n in ("traj_warmstart_create", "traj_warmstart_destroy", "traj_warmstart_set_params",
                  "traj_warmstart_get_params", "traj_warmstart_features", "traj_warmstart_forward",
                  "traj_warmstart_propose",
                  "traj_warmstart_gradients", "traj_warmstart_gradients_fp32",
                  "traj_warmstart_train_step", "traj_warmstart_sync",
                  "traj_warmstart_get_state", "traj_warmstart_set_state", "traj_get_accel_cost"):
            getattr(lib, n).restype = _ci
        _READY = True
    return lib


def num_params() -> int:
    return int(_lib().traj_warmstart_num_params())


CHECKPOINT_MAGIC = "trajbatch-warmstart-checkpoint"


def write_checkpoint(path, params, m, v, step, **meta):
    """Flat binary checkpoint: one JSON header line (magic, format version, parameter
    count, AdamW step, array names in file order, dtype, byte order, caller metadata
    such as the learning rate or the data cursor), then the arrays params, m and v as
    raw little-endian FP32 in that order. Written to a temporary name and renamed."""
    import json
    import os
    arrs = [np.ascontiguousarray(a, "<f4") for a in (params, m, v)]
    n = arrs[0].size
    if any(a.ndim != 1 or a.size != n for a in arrs):
        raise ValueError("params, m and v must be 1-D arrays of one length")
    head = {"magic": CHECKPOINT_MAGIC, "version": 1, "num_params": int(n), "step": int(step),
            "arrays": ["params", "adam_m", "adam_v"], "dtype": "float32",
            "byteorder": "little", "meta": meta}
    tmp = str(path) + ".tmp"
    with open(tmp, "wb") as f:
        f.write((json.dumps(head, sort_keys=True) + "\n").encode())
        for a in arrs:
            f.write(a.tobytes())
    os.replace(tmp, path)


def read_checkpoint(path):
    """(params, m, v, step, meta) from a write_checkpoint file; ValueError when the
    header or the payload size does not match."""
    import json
    with open(path, "rb") as f:
        line = f.readline()
        try:
            head = json.loads(line)
        except ValueError as e:
            raise ValueError(f"{path}: no checkpoint header") from e
        if head.get("magic") != CHECKPOINT_MAGIC or head.get("version") != 1:
            raise ValueError(f"{path}: not a version-1 warm-start checkpoint")
        n = int(head["num_params"])
        data = np.frombuffer(f.read(), "<f4")
    if data.size != 3 * n:
        raise ValueError(f"{path}: payload holds {data.size} values, expected {3 * n}")
    p, m, v = (data[i * n:(i + 1) * n].astype(np.float32) for i in range(3))
    return p, m, v, int(head["step"]), head.get("meta", {})


def init_params(seed: int = 0) -> np.ndarray:
    """Uniform(+-1/sqrt(fan_in)) weights and biases; the last layer scaled by 0.1 so an
    untrained network proposes (nearly) the straight line."""
    rng = np.random.default_rng(seed)
    shapes = [(256, IN), (256,), (256, 256), (256,), (256, 256), (256,), (OUT, 256), (OUT,)]
    fans = [IN, IN, 256, 256, 256, 256, 256, 256]
    out = []
    for k, (shape, fan) in enumerate(zip(shapes, fans)):
        w = rng.uniform(-1.0, 1.0, int(np.prod(shape))) / math.sqrt(fan)
        if k >= 6:
            w *= 0.1
        out.append(w)
    return np.concatenate(out).astype(np.float32)


def _check(rc, what):
    if rc != 0:
        raise tb.TrajBatchError(rc, f"{what}: {tb.load_library().traj_last_error(None).decode()}")


class WarmStart:
    """Handle of the network (C struct traj_warmstart)."""

    def __init__(self, max_rows: int = 4096, stream=None):
        import torch
        self.torch = torch
        self.max_rows = max_rows
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        h = _vp()
        _check(_lib().traj_warmstart_create(max_rows, self.stream, ctypes.byref(h)), "create")
        self._h = h
        self.loss = torch.zeros(1, device="cuda")

    def close(self):
        if getattr(self, "_h", None):
            _lib().traj_warmstart_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, np.float32)
        _check(_lib().traj_warmstart_set_params(self._h, p.ctypes.data), "set_params")

    def get_params(self) -> np.ndarray:
        p = np.zeros(num_params(), np.float32)
        _check(_lib().traj_warmstart_get_params(self._h, p.ctypes.data), "get_params")
        return p

    def get_state(self):
        """Training state: (params, AdamW m, AdamW v, step), FP32 arrays in the public order."""
        n = num_params()
        p, m, v = (np.zeros(n, np.float32) for _ in range(3))
        step = ctypes.c_int(0)
        _check(_lib().traj_warmstart_get_state(self._h, p.ctypes.data, m.ctypes.data,
                                               v.ctypes.data, ctypes.byref(step)), "get_state")
        return p, m, v, int(step.value)

    def set_state(self, params, m, v, step):
        """Restore a training state; the next train_step continues it bit for bit."""
        arrs = [np.ascontiguousarray(a, np.float32) for a in (params, m, v)]
        if any(a.shape != (num_params(),) for a in arrs):
            raise ValueError(f"each state array must hold {num_params()} FP32 values")
        _check(_lib().traj_warmstart_set_state(self._h, arrs[0].ctypes.data, arrs[1].ctypes.data,
                                               arrs[2].ctypes.data, int(step)), "set_state")

    def save_checkpoint(self, path, **meta):
        """Write the training state to `path` (see write_checkpoint)."""
        p, m, v, step = self.get_state()
        write_checkpoint(path, p, m, v, step, **meta)

    def load_checkpoint(self, path):
        """Restore the training state written by save_checkpoint; returns its metadata."""
        p, m, v, step, meta = read_checkpoint(path)
        self.set_state(p, m, v, step)
        return meta

    def features(self, batch, host=None):
        """BF16 features [P, 400] and straight-line coefficients [P, 22] (CUDA tensors).
        host: optional FP32 CPU tensors (pinned for asynchronous copies) holding the
        batch's "centers", "semi_axes" and "velocities", copied to the device on the
        current stream instead of the batch's numpy arrays."""
        torch = self.torch
        P = batch.n_problems
        dev = torch.device("cuda")
        if host is not None:  # copied on the handle's stream, ahead of the features kernel
            with torch.cuda.stream(torch.cuda.ExternalStream(self.stream)):
                cen, ax, vel = (host[k].to(dev, non_blocking=True)
                                for k in ("centers", "semi_axes", "velocities"))
        else:
            cen = torch.as_tensor(batch.centers, dtype=torch.float32, device=dev).contiguous()
            ax = torch.as_tensor(batch.semi_axes, dtype=torch.float32, device=dev).contiguous()
            vel = torch.as_tensor(batch.velocities, dtype=torch.float32, device=dev).contiguous()
        X = torch.zeros(P, IN_PAD, dtype=torch.bfloat16, device=dev)
        line = torch.zeros(P, D22, dtype=torch.float32, device=dev)
        st = np.ascontiguousarray(batch.start, np.float64)
        gl = np.ascontiguousarray(batch.goal, np.float64)
        off = np.ascontiguousarray(batch.offsets, np.int32)
        _check(_lib().traj_warmstart_features(self._h, P, st.ctypes.data, gl.ctypes.data,
                                              off.ctypes.data, cen.data_ptr(), ax.data_ptr(),
                                              vel.data_ptr(), X.data_ptr(), line.data_ptr()),
               "features")
        return X, line

    def forward(self, X, line):
        """Proposals [rows, 8, 2, 11] = line + network(X); rows padded to a multiple of 8."""
        torch = self.torch
        rows = X.shape[0]
        R = (rows + 7) // 8 * 8
        if R != rows:
            X = torch.cat([X, torch.zeros(R - rows, IN_PAD, dtype=X.dtype, device=X.device)])
            line = torch.cat([line, torch.zeros(R - rows, D22, dtype=line.dtype, device=line.device)])
        out = torch.empty(R, HEADS, 2, 11, dtype=torch.float32, device="cuda")
        for r0 in range(0, R, self.max_rows):
            r1 = min(R, r0 + self.max_rows)
            _check(_lib().traj_warmstart_forward(self._h, r1 - r0, X[r0:r1].data_ptr(),
                                                 line[r0:r1].contiguous().data_ptr(),
                                                 out[r0:r1].data_ptr()), "forward")
        return out[:rows]

    def stage(self, batch):
        """The scene arrays of a batch as device tensors plus feature/line/proposal
        buffers, for propose() (one host-to-device copy, done here)."""
        torch = self.torch
        dev = torch.device("cuda")
        P = batch.n_problems
        if P % 8 != 0 or P > self.max_rows:
            raise ValueError("propose() needs a multiple of 8 scenes, at most max_rows")
        f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev)
        return dict(P=P, n_obs=int(batch.offsets[-1]),
                    start=torch.as_tensor(np.ascontiguousarray(batch.start, np.float64), device=dev),
                    goal=torch.as_tensor(np.ascontiguousarray(batch.goal, np.float64), device=dev),
                    offsets=torch.as_tensor(np.ascontiguousarray(batch.offsets, np.int32), device=dev),
                    centers=f32(batch.centers), axes=f32(batch.semi_axes), vel=f32(batch.velocities),
                    X=torch.zeros(P, IN_PAD, dtype=torch.bfloat16, device=dev),
                    line=torch.zeros(P, D22, dtype=torch.float32, device=dev),
                    out=torch.empty(P, HEADS, 2, 11, dtype=torch.float32, device=dev))

    def propose(self, st):
        """Proposals [P, 8, 2, 11] for a staged scene set (asynchronous, device only)."""
        _check(_lib().traj_warmstart_propose(
            self._h, st["P"], st["n_obs"], st["start"].data_ptr(), st["goal"].data_ptr(),
            st["offsets"].data_ptr(), st["centers"].data_ptr(), st["axes"].data_ptr(),
            st["vel"].data_ptr(), st["X"].data_ptr(), st["line"].data_ptr(), st["out"].data_ptr()),
            "propose")
        return st["out"]

    def gradients(self, X, targets, n_labels):
        g = np.zeros(num_params(), np.float32)
        _check(_lib().traj_warmstart_gradients(self._h, X.shape[0], X.data_ptr(),
                                               targets.data_ptr(), n_labels.data_ptr(),
                                               g.ctypes.data, self.loss.data_ptr()), "gradients")
        self.sync()
        return g, float(self.loss.item())

    def gradients_fp32(self, X, targets, n_labels):
        """Loss and gradients of the FP32-operand debug instantiation (CUDA-core FP32
        GEMMs, FP32 activations)."""
        g = np.zeros(num_params(), np.float32)
        _check(_lib().traj_warmstart_gradients_fp32(self._h, X.shape[0], X.data_ptr(),
                                                    targets.data_ptr(), n_labels.data_ptr(),
                                                    g.ctypes.data, self.loss.data_ptr()),
               "gradients_fp32")
        self.sync()
        return g, float(self.loss.item())

    def train_step(self, X, targets, n_labels, lr, weight_decay):
        _check(_lib().traj_warmstart_train_step(self._h, X.shape[0], X.data_ptr(),
                                                targets.data_ptr(), n_labels.data_ptr(),
                                                float(lr), float(weight_decay),
                                                self.loss.data_ptr()), "train_step")
        return self.loss

    def sync(self):
        _check(_lib().traj_warmstart_sync(self._h), "sync")


def make_labels(batch, n_inits=32, cap=300, tol=1e-3, max_labels=HEADS, seed=0,
                chunk=2048, diverse=True):
    """Solve every scene of `batch` from n_inits random initialisations N(line, 0.5 m)
    and keep up to max_labels solved trajectories per scene as offsets from the
    straight line: (targets [P, 8, 22], n_labels [P]). With `diverse`, the labels cover
    the scene's homotopy classes first (traj_homotopy_signature: which side of every
    obstacle a solution passes): the cheapest solution of each class in order of
    acceleration cost, then the cheapest remaining ones; otherwise the cheapest
    solutions overall."""
    P = batch.n_problems
    rng = np.random.default_rng(seed)
    targets = np.zeros((P, HEADS, D22), np.float32)
    n_labels = np.zeros(P, np.int32)
    for p0 in range(0, P, chunk):
        probs = list(range(p0, min(P, p0 + chunk)))
        sub = batch.select_problems(probs)
        lines = np.stack([scenes.straight_line_coeffs(sub.start[k], sub.goal[k])
                          for k in range(sub.n_problems)])
        xi0 = scenes.f32(np.repeat(lines, n_inits, 0) +
                         rng.normal(0.0, 0.5, (sub.n_problems * n_inits, 2, 11)))
        tp = np.repeat(np.arange(sub.n_problems, dtype=np.int32), n_inits)
        import dataclasses
        sub = dataclasses.replace(sub, xi0=xi0, traj_problem=tp)
        h = tb.from_batch(sub)
        try:
            h.solve(cap, tol)
            out = h.get_trajectories()
            cost = np.zeros(sub.n_traj, np.float32)
            rc = _lib().traj_get_accel_cost(h._h, cost.ctypes.data)
            _check(rc, "accel cost")
            sig = h.homotopy_signature() if diverse else None
        finally:
            h.close()
        ok = out["status"] == tb.TRAJ_CONVERGED
        for k in range(sub.n_problems):
            idx = np.nonzero(ok[k * n_inits:(k + 1) * n_inits])[0] + k * n_inits
            if idx.size == 0:
                continue
            idx = idx[np.argsort(cost[idx], kind="stable")]
            if diverse:
                first, seen = [], set()
                for i in idx:
                    if int(sig[i]) not in seen:
                        seen.add(int(sig[i]))
                        first.append(i)
                rest = [i for i in idx if i not in set(first)]
                idx = np.array(first + rest, dtype=idx.dtype)
            idx = idx[:max_labels]
            targets[p0 + k, :idx.size] = (out["xi"][idx] - lines[k][None]).reshape(idx.size, D22)
            n_labels[p0 + k] = idx.size
    return targets, n_labels


def train(ws: WarmStart, X, targets, n_labels, epochs=40, batch_rows=4096, lr=1e-3,
          weight_decay=1e-4, seed=0):
    """Shuffled minibatch training on the GPU; returns the mean loss of every epoch."""
    torch = ws.torch
    keep = torch.nonzero(n_labels > 0).flatten()
    X, targets, n_labels = X[keep], targets[keep], n_labels[keep]
    n = X.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        tot, steps = 0.0, 0
        for r0 in range(0, n, batch_rows):
            idx = perm[r0:r0 + batch_rows]
            rows = idx.numel() // 8 * 8
            if rows < 8:
                continue
            idx = idx[:rows]
            loss = ws.train_step(X[idx].contiguous(), targets[idx].contiguous(),
                                 n_labels[idx].contiguous(), lr, weight_decay)
            tot += float(loss.item())
            steps += 1
        losses.append(tot / max(1, steps))
    ws.sync()
    return losses


def proposals(ws: WarmStart, batch):
    """K = 8 initial coefficient sets per scene: (xi0 [P*8, 2, 11] CUDA, traj_problem)."""
    X, line = ws.features(batch)
    prop = ws.forward(X, line)
    P = batch.n_problems
    return prop.reshape(P * HEADS, 2, 11), np.repeat(np.arange(P, dtype=np.int32), HEADS)


def trained(seed=1000, n_scenes=200000, epochs=20, lr=1e-3, weight_decay=1e-4, cache=None,
            max_rows=4096, diverse=True):
    """A WarmStart trained on n_scenes config-2-style scenes labelled by the optimizer
    (labels covering homotopy classes first when `diverse`), cached as .npy parameters
    (keyed by the training settings)."""
    import os
    if cache is None:
        tag = "_div" if diverse else ""
        cache = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib",
                             f"warmstart_{seed}_{n_scenes}_{epochs}_{lr:g}_{weight_decay:g}{tag}.npy")
    ws = WarmStart(max_rows)
    if os.path.exists(cache):
        ws.set_params(np.load(cache))
        return ws, None
    import torch
    tr = scenes.ellipse_scenes(seed, n_scenes)
    targets, n_labels = make_labels(tr, seed=seed + 1, diverse=diverse)
    ws.set_params(init_params(seed))
    X, _ = ws.features(tr)
    losses = train(ws, X, torch.as_tensor(targets, device="cuda"),
                   torch.as_tensor(n_labels, device="cuda"), epochs=epochs, lr=lr,
                   weight_decay=weight_decay, seed=seed)
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    np.save(cache, ws.get_params())
    return ws, dict(losses=losses, labelled=int((n_labels > 0).sum()), labels=int(n_labels.sum()))
