"""The warm-start training checkpoint file (host logic, no GPU): a JSON header line
followed by params, AdamW m and AdamW v as raw little-endian FP32."""
import json

import numpy as np
import pytest

from paper_2408_10731_b300 import warmstart


def _state(n=1000, seed=0):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32),
            rng.random(n).astype(np.float32))


def test_round_trip_is_bitwise(tmp_path):
    p, m, v = _state()
    path = tmp_path / "a.ckpt"
    warmstart.write_checkpoint(path, p, m, v, 17, lr=1e-3, epoch=2)
    p2, m2, v2, step, meta = warmstart.read_checkpoint(path)
    for a, b in ((p, p2), (m, m2), (v, v2)):
        np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    assert step == 17 and meta == {"lr": 1e-3, "epoch": 2}


def test_layout_is_header_then_three_fp32_arrays(tmp_path):
    p, m, v = _state(10)
    path = tmp_path / "b.ckpt"
    warmstart.write_checkpoint(path, p, m, v, 3)
    raw = path.read_bytes()
    line, payload = raw.split(b"\n", 1)
    head = json.loads(line)
    assert head["magic"] == warmstart.CHECKPOINT_MAGIC and head["num_params"] == 10
    assert head["arrays"] == ["params", "adam_m", "adam_v"] and head["step"] == 3
    assert payload == p.astype("<f4").tobytes() + m.astype("<f4").tobytes() + v.astype("<f4").tobytes()


def test_bad_files_are_refused(tmp_path):
    p, m, v = _state(10)
    good = tmp_path / "c.ckpt"
    warmstart.write_checkpoint(good, p, m, v, 1)
    raw = good.read_bytes()
    trunc = tmp_path / "trunc.ckpt"
    trunc.write_bytes(raw[:-4])
    with pytest.raises(ValueError):
        warmstart.read_checkpoint(trunc)
    other = tmp_path / "other.ckpt"
    other.write_bytes(raw.replace(warmstart.CHECKPOINT_MAGIC.encode(), b"x" * len(warmstart.CHECKPOINT_MAGIC)))
    with pytest.raises(ValueError):
        warmstart.read_checkpoint(other)
    with pytest.raises(ValueError):
        warmstart.write_checkpoint(tmp_path / "d.ckpt", p, m[:5], v, 1)
