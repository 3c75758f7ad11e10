"""Cached launch-shape tuning: traj_autotune's choice per (GPU, batch shape) in JSON.

The tuner itself runs in the library (traj_autotune times each candidate CTA
shape on the handle's own batch); this module only remembers its answers so a
later process with the same GPU and batch shape skips the search.
"""
import json
import os

import numpy as np

CACHE = os.environ.get("TRAJBATCH_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib",
                                    "tune_cache.json"))


def batch_key(batch, precision="fp32", gpu_name=None):
    if gpu_name is None:
        import torch
        gpu_name = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    n_o = np.diff(batch.offsets)
    bucket = lambda x: int(2 ** round(np.log2(max(1.0, float(x)))))
    return (f"{gpu_name}|dim{batch.dim}|np{int(batch.n_steps.max())}|"
            f"traj{bucket(batch.n_traj)}|obs{bucket(n_o.mean() if n_o.size else 1)}|{precision}")


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned(handle, batch, precision="fp32", iters=20):
    """Apply the cached shape for this batch, or tune, store and apply it."""
    key = batch_key(batch, precision)
    cache = _load()
    if key in cache:
        e = cache[key]
        handle.set_launch_shape(e["warps_per_block"], e["blocks_per_sm"],
                                e.get("warps_per_trajectory", 1), e.get("occupancy", 0))
        return dict(e, cached=True)
    e = handle.autotune(iters)
    cache = _load()
    cache[key] = e
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)
    return dict(e, cached=False)
