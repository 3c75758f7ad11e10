"""The exact cull of the obstacle tests against the dense loop and the oracle.

Grazing scenes (`scenes.grazing`) put obstacles about one semi-axis from the path,
so that many grid points sit near an ellipse boundary, with obstacle counts around
the cull's 32-record chunks (63, 64, 65 and 130 obstacles, an odd count's sentinel
half) and horizons that leave the last 32-point slot partly filled (33, 65, 100).

The one-warp-per-trajectory kernels run the culled pair loop; the two-warp team
kernel runs the dense loop (every record at every grid point). The two differ only
in the contraction's summation order, so a record the cull dropped while it held a
point would move the result by a whole projection (centimetres), far beyond the
1e-5 m they are held to here. Both forms, the tensor-core split form and the
footprint solver (whose circle tests are culled the same way) are also checked
against the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import am, footprint as fp
from paper_2408_10731_b300 import scenes
from tests.gpu_helpers import POS_TOL, position_error

pytestmark = pytest.mark.gpu

ITERS = 20


def _solve(batch, shape, precision="fp32"):
    from paper_2408_10731_b300 import trajbatch as tb
    h = tb.from_batch(batch, precision=precision)
    try:
        h.set_launch_shape(*shape)
        h.solve(ITERS, -1.0)
        out = h.get_trajectories()
        out["info"] = h.launch_info()
        return out
    finally:
        h.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_culled_single_warp_matches_the_dense_team(dim):
    b = scenes.grazing(7, dim=dim)
    culled = _solve(b, (4, 0, 1, 0))
    dense = _solve(b, (4, 0, 2, 0))
    assert culled["info"]["warps_per_trajectory"] == 1 and dense["info"]["warps_per_trajectory"] == 2
    err = position_error(b, culled["xi"], dense["xi"])
    assert err.max() <= POS_TOL, err.max()
    o = am.solve(b, ITERS, tol=-1.0)
    for out in (culled, dense):
        e = position_error(b, out["xi"], o["xi"])
        assert e.max() <= POS_TOL, e.max()


def test_culled_capped_build_is_bitwise_the_default_build():
    """The register-capped build runs the same culled loop in the same order."""
    b = scenes.grazing(8, n_steps=(33, 100, 150))
    a = _solve(b, (4, 0, 1, 0))
    c = _solve(b, (4, 0, 1, 1))
    assert c["info"]["occupancy"] == 1
    np.testing.assert_array_equal(a["xi"], c["xi"])
    np.testing.assert_array_equal(a["residual"], c["residual"])


def test_culled_tensor_core_split_form_matches_the_oracle():
    """Split hi/lo BF16 operands: the same bar as the split form's other parity cases."""
    b = scenes.grazing(9, n_obstacles=(1, 24, 65), n_steps=(33, 65, 100))
    g = _solve(b, (0, 0, 1, 0), precision="mixed_split")
    o = am.solve(b, ITERS, tol=-1.0)
    err = position_error(b, g["xi"], o["xi"])
    assert err.max() <= 1e-4, err.max()


def test_culled_footprint_matches_the_oracle():
    """Three circles of radius 0.15 m at -0.35, 0, 0.35 m along the heading."""
    from paper_2408_10731_b300 import footprint as gfp
    offs, rc = (-0.35, 0.0, 0.35), 0.15
    b = scenes.grazing(10, n_obstacles=(2, 33, 65), n_steps=(33, 100), inits=2)
    d = b.goal - b.start
    psi = np.arctan2(d[:, 1], d[:, 0])
    xpsi0 = np.repeat(psi[b.traj_problem][:, None], 11, 1)
    h = gfp.from_batch(b, psi, psi, xpsi0, offs, rc)
    try:
        h.solve(ITERS, -1.0)
        out = h.get_trajectories()
    finally:
        h.close()
    e_pos = 0.0
    for p in range(b.n_problems):
        idx = np.nonzero(b.traj_problem == p)[0]
        c, a, v = b.obstacles(p)
        prob = fp.FPProblem(n_p=int(b.n_steps[p]), T=float(b.duration[p]), start=b.start[p],
                            goal=b.goal[p], psi0=float(psi[p]), psif=float(psi[p]),
                            centers=np.asarray(c, float), semi_axes=np.asarray(a, float),
                            velocities=np.asarray(v, float), offsets=np.asarray(offs),
                            r_circle=rc, vmax=b.vmax, amax=b.amax, rho=b.rho, rho_psi=1.0)
        xi0 = np.concatenate([b.xi0[idx, :2], xpsi0[idx].reshape(-1, 1, 11)], 1)
        ref = fp.solve(prob, xi0, ITERS)
        P, _, _ = am.bernstein(prob.n_p, prob.T)
        g = out["xi"][idx].astype(np.float64)
        x = ref["xi"]
        for r in (0.0,) + offs:
            pg = np.stack([g[:, 0] @ P.T + r * (g[:, 1] @ P.T), g[:, 2] @ P.T + r * (g[:, 3] @ P.T)], -1)
            po = np.stack([x[:, 0] @ P.T + r * (x[:, 1] @ P.T), x[:, 2] @ P.T + r * (x[:, 3] @ P.T)], -1)
            e_pos = max(e_pos, float(np.linalg.norm(pg - po, axis=-1).max()))
    assert e_pos <= POS_TOL, e_pos
