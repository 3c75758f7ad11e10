"""The tensor-core form (TRAJ_PREC_MIXED): BF16 contraction on tcgen05 with FP32
accumulation and one FP32 refinement pass. Its error against the FP64 oracle is
reported, not gated at the FP32 tolerance; what is gated: the error stays
within the BF16 contraction's reach, and every trajectory it reports solved has
FP64-evaluated residuals within the tolerance."""
import dataclasses

import numpy as np
import pytest

from oracle import am
from paper_2408_10731_b300 import scenes
from tests.gpu_helpers import gpu_solve, position_error

pytestmark = pytest.mark.gpu


def _oracle_residual(batch, xi):
    """Residuals of given coefficients (zero iterations: the initial projection)."""
    return am.solve(dataclasses.replace(batch, xi0=xi.astype(np.float64)), 0, tol=-1.0)["residual"]


@pytest.mark.parametrize("make", [lambda: scenes.config2(1, n_scenes=8, inits=8),
                                  lambda: scenes.config1(feasible=True)])
def test_mixed_error_against_fp64_is_small_and_reported(make, capsys):
    b = make()
    g = gpu_solve(b, 20, precision="mixed")
    o = am.solve(b, 20, tol=-1.0)
    err = position_error(b, g["xi"], o["xi"])
    with capsys.disabled():
        print(f"\nmixed vs FP64 after 20 iterations ({b.name}): max {err.max():.2e} m, "
              f"p99 {np.percentile(err, 99):.2e} m, median {np.median(err):.2e} m")
    assert err.max() <= 5e-2 and np.median(err) <= 5e-3
    assert np.all(g["iters"] == 20)


def test_mixed_solved_trajectories_meet_the_tolerance_in_fp64():
    b = scenes.config2(0, n_scenes=16, inits=8)
    tol = 1e-3
    g = gpu_solve(b, 500, tol=tol, precision="mixed")
    ok = g["status"] == 0
    assert ok.sum() > 0
    r = _oracle_residual(b.subset(np.nonzero(ok)[0]), g["xi"][ok])
    assert np.all(r <= tol * (1 + 1e-3) + 2e-6), r.max()
    np.testing.assert_allclose(g["residual"][ok], r, atol=5e-6)
    # the FP32 form on the same inputs solves a comparable number
    f = gpu_solve(b, 500, tol=tol)
    assert ok.sum() >= 0.8 * (f["status"] == 0).sum()


def test_mixed_3d_projection_mode_and_launch_errors():
    c3 = scenes.config3(0, n_traj=64)
    z = scenes.normal_draws(9, (64, 33))
    L = np.linalg.cholesky(c3["sigma0"])
    xi0 = scenes.f32((c3["mu0"][None] + z @ L.T).reshape(64, 3, 11))
    b = dataclasses.replace(c3["batch"], xi0=xi0)
    g = gpu_solve(b, 20, precision="mixed", cost_mode="project")
    o = am.solve(b, 20, tol=-1.0, cost_mode=1)
    assert position_error(b, g["xi"], o["xi"]).max() <= 5e-2
    # uneven horizons are rejected by the tensor-core form (one horizon per batch)
    from paper_2408_10731_b300 import trajbatch as tb
    from tests.gpu_helpers import reduced_config4
    u = reduced_config4(8, seed=1)
    h = tb.from_batch(u, precision="mixed")
    try:
        with pytest.raises(tb.TrajBatchError) as e:
            h.solve(5, -1.0)
        assert e.value.code == -4
    finally:
        h.close()


def test_mixed_full_size_sampled_error(capsys):
    """The bench workload at full size in the tensor-core form (1024 trajectories,
    the default launch): 24 sampled trajectories against the oracle after 20
    iterations, error reported and bounded as above."""
    b = scenes.config2(0)
    g = gpu_solve(b, 20, precision="mixed")
    pick = np.random.default_rng(5).choice(b.n_traj, 24, replace=False)
    sub = b.subset(pick)
    o = am.solve(sub, 20, tol=-1.0)
    err = position_error(sub, g["xi"][pick], o["xi"])
    with capsys.disabled():
        print(f"\nmixed vs FP64, full-size launch, 24 sampled: max {err.max():.2e} m, "
              f"median {np.median(err):.2e} m")
    assert err.max() <= 5e-2 and np.median(err) <= 5e-3
    assert np.all(np.isfinite(g["xi"])) and np.all(g["iters"] == 20)


@pytest.mark.parametrize("n_steps", [17, 37, 75, 150, 256])
def test_mixed_every_contraction_length(n_steps, capsys):
    """Horizons whose padded contraction length K = n_p rounded up to 16 spans one
    to four 64-wide tiles, with a ragged last tile and odd n_p (the time-reversed
    residual that stands in for the last d2B column pairs t with n_p - 1 - t)."""
    b = scenes.config2(3, n_scenes=4, inits=4, n_obstacles=20, n_steps=n_steps)
    g = gpu_solve(b, 20, precision="mixed")
    o = am.solve(b, 20, tol=-1.0)
    err = position_error(b, g["xi"], o["xi"])
    with capsys.disabled():
        print(f"\nmixed vs FP64 after 20 iterations, n_p = {n_steps}: max {err.max():.2e} m, "
              f"median {np.median(err):.2e} m")
    assert err.max() <= 5e-2 and np.median(err) <= 5e-3
    assert np.all(g["iters"] == 20)
