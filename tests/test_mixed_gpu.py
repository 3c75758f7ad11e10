"""The tensor-core forms: BF16 contraction on tcgen05 with FP32 accumulation and one
FP32 refinement pass (TRAJ_PREC_MIXED), and the same with both operands split into
BF16 hi/lo pairs (TRAJ_PREC_MIXED_SPLIT). Their error against the FP64 oracle is
reported, not gated at the FP32 tolerance; what is gated: the error stays within
the reach of the operands' precision, and every trajectory a form reports solved
has FP64-evaluated residuals within the tolerance."""
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


# error bars of each form after 20 fixed iterations: (max, median), metres
BOUND = {"mixed": (5e-2, 5e-3), "mixed_split": (1e-3, 1e-4)}


def _report(capsys, what, prec, err):
    with capsys.disabled():
        print(f"\n{prec} vs FP64 after 20 iterations ({what}): max {err.max():.2e} m, "
              f"p99 {np.percentile(err, 99):.2e} m, median {np.median(err):.2e} m")


@pytest.mark.parametrize("prec", ["mixed", "mixed_split"])
@pytest.mark.parametrize("make", [lambda: scenes.config2(1, n_scenes=8, inits=8),
                                  lambda: scenes.config1(feasible=True)])
def test_mixed_error_against_fp64_is_small_and_reported(make, prec, capsys):
    b = make()
    g = gpu_solve(b, 20, precision=prec)
    o = am.solve(b, 20, tol=-1.0)
    err = position_error(b, g["xi"], o["xi"])
    _report(capsys, b.name, prec, err)
    assert err.max() <= BOUND[prec][0] and np.median(err) <= BOUND[prec][1]
    assert np.all(g["iters"] == 20)


@pytest.mark.parametrize("prec", ["mixed", "mixed_split"])
def test_mixed_uneven_batch_in_one_launch(prec, capsys):
    """The uneven batch (every horizon 50/75/100/150 and obstacle counts 4-256) in the
    tensor-core forms: one launch, each trajectory's MMAs on its own horizon's basis
    operand and its own contraction length."""
    from tests.gpu_helpers import reduced_config4
    b = reduced_config4(12, seed=2)
    assert set(int(n) for n in b.n_steps) == {50, 75, 100, 150}
    if prec == "mixed_split":
        # hi and lo basis operands of all four horizons (256 KB) exceed a CTA's shared
        # memory: refused; three horizons fit
        from paper_2408_10731_b300 import trajbatch as tb
        h = tb.from_batch(b, precision=prec)
        try:
            with pytest.raises(tb.TrajBatchError) as e:
                h.solve(5, -1.0)
            assert e.value.code == -4
        finally:
            h.close()
        b = b.select_problems([p for p in range(b.n_problems) if int(b.n_steps[p]) != 150])
    g = gpu_solve(b, 20, precision=prec)
    o = am.solve(b, 20, tol=-1.0)
    err = position_error(b, g["xi"], o["xi"])
    _report(capsys, "uneven batch", prec, err)
    assert err.max() <= BOUND[prec][0] and np.median(err) <= BOUND[prec][1]
    assert np.all(g["iters"] == 20)
    # per horizon: no horizon reads another's operand (errors of one size everywhere)
    for n_p in sorted(set(int(n) for n in b.n_steps)):
        sel = b.n_steps[b.traj_problem] == n_p
        assert err[sel].max() <= BOUND[prec][0], (n_p, err[sel].max())


@pytest.mark.parametrize("prec", ["mixed", "mixed_split"])
def test_mixed_solved_trajectories_meet_the_tolerance_in_fp64(prec):
    b = scenes.config2(0, n_scenes=16, inits=8)
    tol = 1e-3
    g = gpu_solve(b, 500, tol=tol, precision=prec)
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
    gs = gpu_solve(b, 20, precision="mixed_split", cost_mode="project")
    assert position_error(b, gs["xi"], o["xi"]).max() <= BOUND["mixed_split"][0]
    # more distinct horizons than the form holds basis operands for: refused
    from paper_2408_10731_b300 import trajbatch as tb
    many = scenes.config2(2, n_scenes=17, inits=1, n_obstacles=2)
    many = dataclasses.replace(many, n_steps=np.arange(20, 37, dtype=np.int32),
                               duration=0.1 * np.arange(20, 37))
    h = tb.from_batch(many, precision="mixed")
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


@pytest.mark.parametrize("prec", ["mixed", "mixed_split"])
@pytest.mark.parametrize("n_steps", [17, 37, 75, 150, 256])
def test_mixed_every_contraction_length(n_steps, prec, capsys):
    """Horizons whose padded contraction length K = n_p rounded up to 16 spans one
    to four 64-wide tiles, with a ragged last tile and odd n_p (the time-reversed
    residual that stands in for the last d2B column pairs t with n_p - 1 - t)."""
    b = scenes.config2(3, n_scenes=4, inits=4, n_obstacles=20, n_steps=n_steps)
    g = gpu_solve(b, 20, precision=prec)
    o = am.solve(b, 20, tol=-1.0)
    err = position_error(b, g["xi"], o["xi"])
    _report(capsys, f"n_p = {n_steps}", prec, err)
    assert err.max() <= BOUND[prec][0] and np.median(err) <= BOUND[prec][1]
    assert np.all(g["iters"] == 20)
