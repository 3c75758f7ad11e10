"""The bench's roofline arithmetic (CPU): the algorithmic operation counts per
trajectory-iteration, and the rule that a measured DRAM traffic figure is reported only
for the kernel sources it was captured on."""
import numpy as np

import bench
from paper_2408_10731_b300 import scenes


def test_lane_op_count_per_iteration_on_the_config2_scene():
    # one 2D problem, n_o = 50, n_p = 100: per evaluate / project / contract pass
    # 50 x 100 pairs x 13 + 200 bound rows x 10 + 2 x 300 x 11 x 2, per QP step 2 x 121 x 2
    b = scenes.config2(0, n_scenes=2, inits=3)
    assert np.all(np.diff(b.offsets) == 50) and np.all(b.n_steps == 100) and b.dim == 2
    per_pass = 50 * 100 * 13 + 2 * 100 * 10 + 2 * 3 * 100 * 11 * 2
    assert per_pass + 484 == 80684
    for k in (0, 1, 7):
        want = b.n_traj * ((k + 1) * per_pass + k * 484)
        assert bench.algorithmic_ops(b, np.full(b.n_traj, k)) == want
    # one iteration more costs one pass and one QP step per trajectory
    assert (bench.algorithmic_ops(b, np.full(b.n_traj, 5)) -
            bench.algorithmic_ops(b, np.full(b.n_traj, 4))) == b.n_traj * 80684


def test_rsqrt_count_per_pass():
    b = scenes.config2(0, n_scenes=2, inits=3)
    assert bench.algorithmic_mufu(b, np.zeros(b.n_traj)) == b.n_traj * (50 * 100 + 200)
    assert bench.algorithmic_mufu(b, np.full(b.n_traj, 9)) == 10 * b.n_traj * 5200


def test_the_3d_pair_weighs_17_and_ragged_batches_add_per_trajectory():
    b3 = scenes.grazing(1, n_obstacles=(4,), n_steps=(33,), inits=2, dim=3)
    per_pass = 4 * 33 * 17 + 2 * 33 * 10 + 2 * 3 * 33 * 11 * 3
    assert bench.algorithmic_ops(b3, np.zeros(b3.n_traj)) == b3.n_traj * per_pass
    u = scenes.grazing(2, n_obstacles=(1, 64), n_steps=(33, 100), inits=1)
    iters = np.arange(u.n_traj)
    want = 0
    for k in range(u.n_traj):
        p = u.traj_problem[k]
        n_o, n_p = u.n_obstacles(p), int(u.n_steps[p])
        want += (iters[k] + 1) * (n_o * n_p * 13 + 2 * n_p * 10 + 2 * 3 * n_p * 11 * 2) + iters[k] * 484
    assert bench.algorithmic_ops(u, iters) == want


def test_measured_traffic_holds_only_for_the_captured_sources(monkeypatch):
    for kernel in ("k_am_fp32", "k_am_mixed"):
        d = bench.source_digest(kernel)
        assert d == bench.source_digest(kernel) and len(d) == 16
        monkeypatch.setitem(bench.MEASURED_TRAFFIC, (kernel, "config5"), (1234, d))
        assert bench.measured_traffic(kernel, "config5") == 1234
        assert bench.measured_traffic(kernel + " (split operands)", "config5") == 1234
        monkeypatch.setitem(bench.MEASURED_TRAFFIC, (kernel, "config5"), (1234, "0" * 16))
        assert bench.measured_traffic(kernel, "config5") is None
    assert bench.measured_traffic("k_am_fp32", "no such workload") is None


def test_single_thread_baseline_spans_every_scene_of_the_all_core_sample():
    """The one-thread oracle run takes every 4th trajectory of the all-core sample's
    scenes, so that it covers the same scenes (two trajectories each of eight)."""
    b = scenes.config2(0, n_scenes=4, inits=8)
    one = bench.cpu_baseline(workload=b, scenes_idx=range(4), n_threads=1, traj_stride=4,
                             max_iters=3)
    assert one["cores"] == 1 and one["kind"] == "oracle"
    assert one["sample"].startswith("8 trajectories (scenes 0..3 of the workload, every 4th "
                                    "trajectory)")
    assert 0 <= one["solved"] <= 8 and one["trajectory_iterations_per_s"] > 0
    sub = b.select_problems(range(4)).subset(range(0, 32, 4))
    assert sorted(set(sub.traj_problem.tolist())) == [0, 1, 2, 3]
    allc = bench.cpu_baseline(workload=b, scenes_idx=range(4), max_iters=3)
    assert allc["sample"].startswith("32 trajectories (scenes 0..3 of the workload, all "
                                     "initialisations)")
