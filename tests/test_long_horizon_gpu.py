"""GPU parity of the long-horizon solve (more than 256 grid points per problem)
against the FP64 oracle.

Paper I plans over n_p = 1000 grid points with 10 obstacles. Above 256 grid
points the FP32 form runs one warp per trajectory that streams its grid points
in chunks (256 in 2D, 128 in 3D) every iteration, accumulating the contraction F^T r and the
residual maxima over the chunks; the FP64 set-up stages the basis 256 rows at a
time. The bar is that of every FP32 parity test: max coefficient-evaluated
position error <= 1e-5 m after a fixed iteration count, residuals to FP32
rounding.
"""
import dataclasses

import numpy as np
import pytest

from oracle import am
from paper_2408_10731_b300 import scenes
from tests.gpu_helpers import POS_TOL, gpu_solve, position_error

pytestmark = pytest.mark.gpu


def _parity(batch, iters):
    g = gpu_solve(batch, iters)
    o = am.solve(batch, iters, tol=-1.0)
    err = position_error(batch, g["xi"], o["xi"])
    assert err.max() <= POS_TOL, (err.max(), np.argmax(err))
    np.testing.assert_allclose(g["residual"], o["residual"], atol=2e-5, rtol=1e-4)
    assert np.all(g["iters"] == iters)
    return g, o


@pytest.mark.parametrize("dim,n_p", [(2, 257), (2, 300), (2, 1000), (3, 640), (3, 1000)])
def test_long_horizon_parity(dim, n_p):
    """One chunk plus a single grid point (257), a ragged last chunk (300), five full
    chunks (640) and Paper I's n_p = 1000, moving obstacles, 2D and 3D."""
    _parity(scenes.long_horizon(seed=n_p + dim, n_scenes=2, inits=3, n_steps=n_p, dim=dim), 20)


def test_long_horizon_static_obstacles_parity():
    """Paper I's 2D static setting: 10 fixed ellipses, n_p = 1000."""
    _parity(scenes.long_horizon(seed=5, n_scenes=2, inits=4, n_steps=1000, moving=False), 30)


@pytest.mark.parametrize("n_steps", [[50, 1000, 50, 1000], [50, 256, 400, 257]])
def test_mixed_horizons_in_one_launch(n_steps):
    """Short and long problems in one batch: the chunked kernel takes them all (the
    basis tables of the distinct horizons stay within 160 KB)."""
    b = scenes.long_horizon(seed=8, n_scenes=4, inits=2, n_steps=n_steps)
    _parity(b, 20)


def test_basis_tables_beyond_160_kb_are_refused():
    """Distinct horizons 50, 256, 400 and 1000 need 245 KB of basis tables."""
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.long_horizon(seed=8, n_scenes=4, inits=2, n_steps=[50, 256, 400, 1000])
    with pytest.raises(tb.TrajBatchError) as e:
        tb.from_batch(b)
    assert e.value.code == -4 and "160 KB" in str(e.value)


def test_long_horizon_solves_to_tolerance():
    """Solving to 1e-3 m: every trajectory reported solved meets the tolerance when its
    coefficients are evaluated in FP64 (the oracle's residuals of the returned
    coefficients), and the reported FP32 residuals agree with those."""
    b = scenes.long_horizon(seed=3, n_scenes=4, inits=4, n_steps=1000)
    tol = 1e-3
    g = gpu_solve(b, 500, tol=tol)
    ok = np.nonzero(g["status"] == 0)[0]
    assert ok.size > 0
    sub = b.subset(ok)
    r = am.solve(dataclasses.replace(sub, xi0=g["xi"][ok].astype(np.float64)), 0,
                 tol=-1.0)["residual"]
    assert np.all(r <= tol * (1 + 1e-3) + 2e-6), r.max()
    np.testing.assert_allclose(g["residual"][ok], r, atol=5e-6)


def test_long_horizon_refusals():
    """The tensor-core form and teams of warps stop at 256 grid points; a handle
    takes at most 1024."""
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.long_horizon(seed=1, n_scenes=1, inits=2, n_steps=300)
    h = tb.from_batch(b, precision="mixed")
    try:
        with pytest.raises(tb.TrajBatchError) as e:
            h.solve(5, -1.0)
        assert e.value.code == -4  # TRAJ_ESHAPE
    finally:
        h.close()
    h = tb.from_batch(b)
    try:
        h.set_launch_shape(4, 0, 2)
        with pytest.raises(tb.TrajBatchError) as e:
            h.solve(5, -1.0)
        assert e.value.code == -4
        h.set_launch_shape(4, 0, 1)
        h.solve(5, -1.0)
    finally:
        h.close()
    with pytest.raises(tb.TrajBatchError):
        tb.TrajBatch(2, 1, 2, 10, 1025, 1.5, 2.0, 1.0, 1.0, 1.0, "fp32", "smooth_track", None)


def test_long_horizon_launch_shapes_agree_bitwise():
    """One warp per trajectory whatever the CTA shape: the spread default, fixed
    shapes, a replayed graph and the autotuned shape give bitwise the same result."""
    from paper_2408_10731_b300 import trajbatch as tb
    b = scenes.long_horizon(seed=12, n_scenes=3, inits=3, n_steps=[257, 640, 100])
    h = tb.from_batch(b)
    try:
        ref = None
        for w, bps in ((0, 0), (8, 0), (2, 0), (8, 1), (1, 1)):
            h.set_launch_shape(w, bps, 1)
            for _ in range(2):  # capture, then replay
                h.solve(15, tol=-1.0)
                out = h.get_trajectories()
                ref = out if ref is None else ref
                np.testing.assert_array_equal(out["xi"], ref["xi"])
        choice = h.autotune(5)
        assert choice["warps_per_trajectory"] == 1
        assert tb.load_library().traj_last_error(h._h).decode() == ""
        h.solve(15, tol=-1.0)
        np.testing.assert_array_equal(h.get_trajectories()["xi"], ref["xi"])
    finally:
        h.close()
    o = am.solve(b, 15, tol=-1.0)
    assert position_error(b, ref["xi"], o["xi"]).max() <= POS_TOL
