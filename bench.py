#!/usr/bin/env python
"""Benchmark: solved trajectories/sec at residual <= 1e-3 m of the batched optimizer.

Default workload (config5): the learned warm start on 4096 held-out 2D moving-ellipse
scenes (n_p = 100 over 10 s, 50 constant-velocity ellipses) x 8 trajectories =
32 768, iteration cap 500, one batch solve per step (proposals included); beside it
the plain FP32 form from random and straight-line initialisations on the same scenes.
Other workloads: config2 (128 scenes x 8), uneven, long, priest, multiagent,
footprint, mpc, gemm.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|mixed_split]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Prints one JSON line (rank 0). Under torchrun each rank solves its own seeded
batch (independent problems, no data-path collective: weak scaling); the
barrier and the max over ranks are the only cross-rank steps.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("solved trajectories/sec at residual ≤1e-3 m; ms per batch solve vs plain FP32 GPU")
UNIT = "solved trajectories/s"
WORKLOAD = ("2D moving ellipses: n_p=100 over T=10 s, 50 constant-velocity axis-aligned "
            "ellipses (semi-axes U(0.2,0.8) m, speed U(0,1) m/s), start (0,0) goal (8,8), "
            "128 scenes x 8 initialisations N(straight line, 0.5 m) = 1024 trajectories, "
            "vmax 1.5 m/s, amax 2 m/s^2, rho 1, cap 500 iterations, tol 1e-3")
WORKLOAD_CONFIG5 = ("learned warm start on held-out scenes: {n} config-2-style 2D scenes (seed 99: "
                    "n_p=100 over T=10 s, 50 constant-velocity axis-aligned ellipses, semi-axes "
                    "U(0.2,0.8) m, speed U(0,1) m/s, start (0,0) goal (8,8)), K=8 trajectories per "
                    "scene = {b}: the network's 8 proposals (headline) vs 8 random N(straight line, "
                    "0.5 m) and 8 straight-line initialisations; vmax 1.5 m/s, amax 2 m/s^2, rho 1, "
                    "cap 500 iterations, tol 1e-3")
WORKLOAD_UNEVEN = ("uneven 2D batch: 2048 problems, obstacle counts log-uniform 4-256, horizons "
                   "n_p in {50,75,100,150} over T=0.1 n_p s, goal 0.55 vmax T away, 8 "
                   "initialisations each = 16384 trajectories in one persistent launch "
                   "(CUDA graph, autotuned CTA shape), cap 500 iterations, tol 1e-3")
WORKLOAD_LONG = ("long-horizon 2D batch (Paper I's n_o = 10, n_p = 1000): 128 scenes, n_p=1000 "
                 "over T=10 s, 10 constant-velocity axis-aligned ellipses (semi-axes U(0.2,0.8) m, "
                 "speed U(0,1) m/s), start (0,0), goal 0.55 vmax T along the diagonal, 8 "
                 "initialisations N(straight line, 0.5 m) = 1024 trajectories, grid points "
                 "streamed in chunks of 256, vmax 1.5 m/s, amax 2 m/s^2, rho 1, cap 500 "
                 "iterations, tol 1e-3")


# DRAM bytes (read + write) per launch of each solve kernel on its bench workload,
# from one ncu capture each (profiles/), valid only for the kernel sources they were
# taken on: (kernel, workload) -> (bytes, source digest of KERNEL_SOURCES). A changed
# source reports null until the kernel is captured again. The config5 entries were
# captured on 512 of the 4096 held-out scenes (4096 trajectories: the full launch is
# too long for a many-pass capture) and scaled by 8: the bytes are the problems'
# constants, obstacle records and the coefficients, all proportional to the batch.
KERNEL_SOURCES = {
    "k_am_fp32": ("am_solve.cu", "am_device.cuh", "internal.cuh"),
    "k_am_team": ("am_solve.cu", "am_device.cuh", "internal.cuh"),
    "k_am_long": ("am_solve.cu", "am_device.cuh", "internal.cuh"),
    "k_am_mixed": ("am_mixed.cu", "am_device.cuh", "internal.cuh", "tcgen05.cuh"),
}
MEASURED_TRAFFIC = {
    ("k_am_fp32", "config5"): (8 * 2865664, "0b4f1a0787df6ca5"),
    ("k_am_mixed", "config5"): (8 * 2802432, "96366f47fb100bee"),
}


def source_digest(kernel):
    """SHA-256 (first 16 hex digits) over the sources that build a solve kernel."""
    kernel = kernel.split(" ")[0]
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_2408_10731_b300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload="config2"):
    kernel = kernel.split(" ")[0]
    entry = MEASURED_TRAFFIC.get((kernel, workload))
    return entry[0] if entry and entry[1] == source_digest(kernel) else None


def combine_ranks(dist, world, total_ms, n_solved, e2e_rate, device="cpu"):
    """Whole-job figures over the ranks (weak scaling, one independent batch per rank):
    the slowest rank's timed total, the solved trajectories of all ranks, and the sum
    of the ranks' end-to-end rates. One all_gather; no collective touches the data path."""
    if world <= 1 or dist is None:
        return float(total_ms), float(n_solved), float(e2e_rate)
    import torch
    t = torch.tensor([total_ms, n_solved, e2e_rate], device=device, dtype=torch.float64)
    gathered = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(gathered, t)
    g = torch.stack(gathered).cpu().numpy()
    return float(g[:, 0].max()), float(g[:, 1].sum()), float(g[:, 2].sum())


def kernel_name(precision, shape, max_np=100):
    """The solve kernel a handle of this precision and launch shape runs."""
    if precision in ("mixed", "mixed_split"):
        return "k_am_mixed" if precision == "mixed" else "k_am_mixed (split operands)"
    if max_np > 256:
        return "k_am_long"
    return "k_am_team" if shape and shape.get("warps_per_trajectory", 1) > 1 else "k_am_fp32"


def algorithmic_ops(batch, iters):
    """FP32 lane operations the method must execute for the given iteration counts,
    counted per trajectory-iteration (the dense count of the method's definition):
      every obstacle-timestep pair (the dense test, every pair every iteration):
        13 in 2D, 17 in 3D (Delta = p - (c + v t), u = Delta / a, |u|^2, the
        compare, and the projection's share: 1 / |u| - 1, the scale and the sum);
      every velocity and acceleration bound row: 10 (norm, compare, projection);
      the contractions P xi, Pd xi, Pdd xi (evaluation) and F^T r: 2 x 3 n_p x 11 x dim;
      the QP step: 2 x 11 x 11 x dim.
    On the 2D workload (n_o = 50, n_p = 100) that is 5000 x 13 + 200 x 10 + 13 200 +
    484 = 80 684 per trajectory-iteration. The initial projection counts as one more
    evaluate / project / contract pass."""
    dim = batch.dim
    pair = 13 if dim == 2 else 17
    n_o = np.diff(batch.offsets)[batch.traj_problem]
    n_p = batch.n_steps[batch.traj_problem]
    proj = n_o * n_p * pair + 2 * n_p * 10 + 2 * 3 * n_p * 11 * dim
    qp = 2 * 11 * 11 * dim
    it = np.asarray(iters, np.int64)
    return float(np.sum((it + 1) * proj + it * qp))


def algorithmic_mufu(batch, iters):
    """MUFU operations (rsqrtf) per the same count: one per obstacle-timestep pair and
    one per velocity and acceleration bound row, every pass."""
    n_o = np.diff(batch.offsets)[batch.traj_problem]
    n_p = batch.n_steps[batch.traj_problem]
    it = np.asarray(iters, np.int64)
    return float(np.sum((it + 1) * (n_o * n_p + 2 * n_p)))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every interval_ms (200 ms; shorter
    for a timed region of well under a second); mark() brackets the timed region so
    that only the samples taken inside it are summarised."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id, interval_ms=200):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.marks = []
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_id}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", str(interval_ms)],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
            return
        t0 = time.time()
        while time.time() - t0 < 10 and self._lines() == 0 and self.p.poll() is None:
            time.sleep(0.05)

    def _lines(self):
        with open(self.f.name) as fh:
            return sum(1 for _ in fh)

    def mark(self):
        self.marks.append(self._lines())

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        with open(self.f.name) as fh:
            lines = fh.read().splitlines()
        os.unlink(self.f.name)
        lo, hi = (self.marks + [0, len(lines)])[:2] if len(self.marks) >= 2 else (0, len(lines))
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines[lo:hi]:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _pci_id(torch, dev):
    p = torch.cuda.get_device_properties(dev)
    try:
        return f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
    except AttributeError:
        return str(dev)


def cpu_baseline(seed=0, scenes_idx=range(16), max_iters=500, tol=1e-3, workload=None,
                 n_threads=None, traj_stride=1):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload: the
    listed scenes of the seeded batch with every traj_stride-th of their trajectories;
    n_threads None uses every host core (OpenMP over trajectories)."""
    from oracle import am
    from paper_2408_10731_b300 import scenes
    full = workload if workload is not None else scenes.config2(seed)
    idx = list(scenes_idx)
    b = full.select_problems(idx)
    if traj_stride > 1:
        b = b.subset(range(0, b.n_traj, traj_stride))
    which = "all initialisations" if traj_stride == 1 else f"every {traj_stride}th trajectory"
    cores = n_threads or (os.cpu_count() or 1)
    t0 = time.perf_counter()
    out = am.solve(b, max_iters, tol=tol, n_threads=cores)
    dt = time.perf_counter() - t0
    solved = int(np.sum(np.all(out["residual"] <= tol, axis=1) & (out["iters"] < max_iters + 1)))
    return {"value": solved / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{b.n_traj} trajectories (scenes {idx[0]}..{idx[-1]} of the workload, "
                      f"{which}), full solve (cap {max_iters}, tol {tol}), FP64, "
                      f"{'one thread' if cores == 1 else 'OpenMP over trajectories'}; "
                      f"{solved} solved in {dt:.2f} s",
            "seconds": dt, "solved": solved,
            "trajectory_iterations_per_s": float(np.sum(out["iters"])) / dt}


def cpu_baseline_both(batch, wl):
    """The oracle on the host: all cores on 32 scenes (256 trajectories; 4 scenes of the
    long horizon), and one thread on every 4th trajectory of the same scenes (64; 8 of
    the long horizon). On the held-out scenes only about one trajectory in seven
    converges and the converging ones gather in some scenes, so both samples span all
    32 scenes; trajectory-iterations/s is reported beside."""
    n_all = 4 if wl == "long" else 32
    allc = cpu_baseline(workload=batch, scenes_idx=range(n_all))
    one = cpu_baseline(workload=batch, scenes_idx=range(n_all), n_threads=1, traj_stride=4)
    for d in (allc, one):
        d.pop("seconds", None); d.pop("solved", None)
    allc["single_thread"] = one
    return allc


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle timed on the host cores (rank 0 only), on the same
    workload as the default run. Step i solves scenes 8i .. 8i + 7 (mod the scene count)
    with all their initialisations (64 trajectories: a quarter of the held-out scenes
    have a solution at all, so a smaller step often solves none), and successive steps
    sweep the batch; the value is the total solved over the total time of the timed
    steps."""
    if rank != 0:
        return
    from paper_2408_10731_b300 import scenes
    if args.workload == "config5":
        full = heldout_scenes(0, args.scenes)
        workload = WORKLOAD_CONFIG5.format(n=full.n_problems, b=full.n_traj)
    else:
        full = scenes.config2(args.seed)
        workload = WORKLOAD
    P = full.n_problems

    per_step = 8

    def step(i):
        return cpu_baseline(args.seed, tuple((per_step * i + j) % P for j in range(per_step)),
                            workload=full)

    for i in range(args.warmup):
        step(i)
    solved, secs = 0, []
    for i in range(args.steps):
        r = step(i)
        solved += r["solved"]; secs.append(r["seconds"])
    value = solved / float(np.sum(secs))
    sample = (f"64 trajectories per step (scenes 8i .. 8i+7 of the workload, all 8 random "
              f"initialisations), full FP64 solve; {solved} solved in {np.sum(secs):.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_priest(args, torch):
    """The 3D projection-guided sampler: 4096 samples, 10 outer x 20 inner iterations,
    256 sphere obstacles; one step = one full sampler run from (mu0, Sigma0)."""
    from paper_2408_10731_b300 import scenes, trajbatch
    c3 = scenes.config3(args.seed, n_traj=4096)
    b = c3["batch"]
    h = trajbatch.from_batch(b, cost_mode="project")
    D = 33
    cfg = dict(n_inner=c3["n_inner"], n_proj=c3["n_proj"], n_elite=c3["n_elite"], gamma=1.0,
               sigma_lr=0.5, eps=1e-6, w_res=1.0, seed=args.seed)
    dev = torch.device("cuda")
    mu0 = torch.as_tensor(c3["mu0"], dtype=torch.float32, device=dev)
    s0 = torch.as_tensor(c3["sigma0"], dtype=torch.float32, device=dev)
    mu, sigma, best = mu0.clone(), s0.clone(), torch.zeros(D + 1, device=dev)
    stream = torch.cuda.current_stream()

    def run():
        mu.copy_(mu0); sigma.copy_(s0)
        for it in range(c3["n_outer"]):
            h.sampler_step(cfg, it, mu, sigma, best)

    # launch shape of the projection solve: tuned on the sampler's own first samples
    h.sampler_step(cfg, 0, mu, sigma, best)
    if args.shape:
        w, bps, team = (int(x) for x in args.shape.split(","))
        h.set_launch_shape(w, bps, team)
        shape = {"warps_per_block": w, "blocks_per_sm": bps, "warps_per_trajectory": team,
                 "fixed": True}
    else:
        from paper_2408_10731_b300 import autotune
        shape = autotune.tuned(h, b, "fp32-project", iters=c3["n_inner"])
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    ms = []
    clk = ClockSampler(_pci_id(torch, 0), interval_ms=20)
    clk.mark()
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream); run(); e1.record(stream); e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk.mark()
    clocks = clk.stop()
    # D-PRIEST: 4 distributions of 1024 samples each refined in parallel, with the BARN
    # cost terms (curvature, distance to the straight path); same solve and launch shape
    nd = 4
    cfg_d = dict(cfg, n_proj=int(np.ceil(0.73 * 1024)), n_elite=int(np.ceil(0.10 * 1024)),
                 w_curv=0.05, w_path=0.5)
    mus0 = mu0.repeat(nd, 1)
    mus0[1:] += torch.randn(nd - 1, D, generator=torch.Generator(device=dev).manual_seed(args.seed),
                            device=dev)
    sig0 = s0.repeat(nd, 1, 1)
    mus, sigs, bests = mus0.clone(), sig0.clone(), torch.zeros(nd, D + 1, device=dev)

    def run_d():
        mus.copy_(mus0); sigs.copy_(sig0)
        for it in range(c3["n_outer"]):
            h.sampler_step(cfg_d, it, mus, sigs, bests, n_dist=nd)

    for _ in range(args.warmup):
        run_d()
    torch.cuda.synchronize()
    msd = []
    for _ in range(max(3, args.steps // 2)):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream); run_d(); e1.record(stream); e1.synchronize()
        msd.append(e0.elapsed_time(e1))
    dpriest = {"ms_per_run": float(np.mean(msd)), "distributions": nd, "samples_per_distribution": 1024,
               "best_cost_aug": [float(x) for x in bests[:, D].cpu()],
               "cost": "sum_t ||p''||^2 + 0.05 curvature^2 + 0.5 path distance + residual",
               "launches_per_run": c3["n_outer"] * 8}
    # PRIEST's workspace bounds (the 20 x 20 x 5 m box of the scene) as extra rows of F
    h.set_workspace([[0.0, 0.0, 0.0]], [[20.0, 20.0, 5.0]])
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    msw = []
    for _ in range(max(3, args.steps // 2)):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream); run(); e1.record(stream); e1.synchronize()
        msw.append(e0.elapsed_time(e1))
    wsb = {"ms_per_run": float(np.mean(msw)), "box_lo": [0.0, 0.0, 0.0], "box_hi": [20.0, 20.0, 5.0],
           "best_cost_aug": float(best[D].item())}
    h.set_workspace(None, None)
    # residual of the returned trajectory (one more projection-free evaluation on the host
    # is not needed: the sampler's best is a projected sample; report its c_aug)
    bc = float(best[D].item())
    # ALU roofline of the run: every outer iteration projects all samples for n_inner
    # fixed iterations (the refit, sampling and sorts are < 1 % of the run)
    fp32_peak = trajbatch.measure_fp32_peak(5)
    ops = c3["n_outer"] * algorithmic_ops(b, np.full(b.n_traj, c3["n_inner"]))
    achieved = ops / (float(np.mean(ms)) * 1e-3)
    line = {"metric": "ms per projection-guided sampler run (3D, 4096 samples, 10 outer x 20 "
                      "inner)", "value": float(np.mean(ms)), "unit": "ms", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ms)),
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "3D: 256 spheres r~U(0.1,0.3) on 12 box surfaces in 20x20x5 m, "
                                   "n_p=100 over 20 s, B=4096, N_proj=2991, N_elite=410, gamma 1, "
                                   "sigma_lr 0.5", "launch_shape": shape},
            "best_cost_aug": bc, "gpu_launches_per_step": c3["n_outer"] * 8, "clocks": clocks,
            "forms": {"d_priest_barn": dpriest, "workspace_bounds": wsb},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fp32_peak / 2e12,
                         "unit": "Top/s", "frac": achieved / (fp32_peak / 2.0), "traffic": None,
                         "kernel": kernel_name("fp32", shape) + " (3D, projection mode; whole run timed)",
                         "count": "the method's dense count: every sample x sphere x grid point "
                                  "test, including those the kernel's exact cull skips (their "
                                  "projections are zero)",
                         "peak_source": "measured FFMA microbenchmark (traj_measure_fp32_peak), "
                                        "FP32 lane-ops/s",
                         "algorithmic_ops_per_run": ops}}
    print(json.dumps(line), flush=True)
    h.close()


def multiagent_ops(N, dim, n_p, n_o, iters):
    """FP32 lane operations Algorithm 5 must execute per scene for `iters` iterations
    (+ the initial pass). Per unordered agent pair or agent-obstacle pair and grid
    point (the pair pass): delta [dim], spheroid norm and e [3 dim + 4], d [2 dim + 2],
    r and ||r|| [2 dim + 1], multiplier update [dim] -> 2D 23, 3D 31. Per agent,
    axis and grid point: the multiplier sums [N - 1 + n_o + 2] and the positions
    [11 FMA]. Per agent, axis and coefficient: u = P^T w [n_p FMA] and the x-step
    [2 x 11 + 2 FMA]."""
    pair = 8 * dim + 7
    per_pt = (N - 1 + n_o + 2) + 11
    per_c = n_p + 24
    per_it = (N * (N - 1) // 2 + N * n_o) * n_p * pair + N * dim * n_p * per_pt + N * dim * 11 * per_c
    return float(per_it) * (np.asarray(iters, np.float64) + 1.0)


def run_multiagent(args, torch):
    """Joint multi-agent optimizer (Paper IV, Algorithm 5): a batch of random-benchmark
    scenes, each with N agents solved jointly to residual <= 0.01; one step = one
    batch solve."""
    from paper_2408_10731_b300 import scenes, multiagent as gma, trajbatch
    N, S = args.ma_agents, args.ma_scenes
    sc = scenes.ma_random(args.seed, n_scenes=S, n_agents=N, dim=3, room=8.0,
                          radius=args.ma_radius, n_steps=100, T=10.0)
    rho = dict(rho=2.0, rho_levels=10, rho_growth=1.5, rho_every=20)
    tol, cap = 1e-2, 500
    h = gma.from_scenes(sc, **rho)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        h.solve(cap, tol, stats=False)
    torch.cuda.synchronize()
    ms, conv = [], []
    clk = ClockSampler(_pci_id(torch, 0), interval_ms=20)
    clk.mark()
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream); h.solve(cap, tol, stats=False); e1.record(stream); e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk.mark()
    clocks = clk.stop()
    out = h.get_trajectories()
    n_conv = int(np.sum(out["residual"] <= tol))
    step_ms = float(np.mean(ms))
    # end to end through the public API: host inputs -> set_problems (copies + FP64 set-up)
    # -> solve -> coefficients back to the host
    e2e = []
    for _ in range(max(1, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.set_problems(sc)
        h.solve(cap, tol, stats=False)
        r = h.get_trajectories()
        e2e.append(time.perf_counter() - t0)
    h2d = sc.duration.nbytes + 2 * sc.start.nbytes + sc.radius.nbytes * 2 + sc.obs_offsets.nbytes
    d2h = r["xi"].nbytes + r["residual"].nbytes + r["iterations"].nbytes
    it = out["iterations"].astype(np.float64)
    ops = float(np.sum(multiagent_ops(N, 3, 100, 0, it)))
    fp32_peak = trajbatch.measure_fp32_peak(5)
    achieved = ops / (step_ms * 1e-3)
    line = {"metric": f"multi-agent scenes solved/s ({N} agents jointly, residual <= 0.01 m)",
            "value": n_conv / (step_ms * 1e-3), "unit": "scenes/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"random benchmark: {S} scenes x {N} agents (3D spheres r "
                                   f"{args.ma_radius} m, starts and goals uniform in an 8 x 8 m "
                                   f"room at z in [0.5, 1.5] m, separation >= 2r + 0.2 m), n_p=100 "
                                   f"over 10 s, rho 2 x 1.5^l (10 levels, every 20), cap {cap}",
                       "l2": "the working set (pair multipliers) is rewritten every iteration"},
            "scenes_converged": n_conv, "scenes": S,
            "iters_median": float(np.median(it)), "iters_max": int(it.max()),
            "ms_per_scene_latency": step_ms,
            "e2e": {"value": n_conv / float(np.mean(e2e)), "unit": "scenes/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": 1,
            "clocks": clocks,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fp32_peak / 2e12,
                         "unit": "Top/s", "frac": achieved / (fp32_peak / 2.0), "traffic": None,
                         "kernel": "k_ma_solve<3>",
                         "peak_source": "measured FFMA microbenchmark (traj_measure_fp32_peak), "
                                        "FP32 lane-ops/s",
                         "algorithmic_ops_per_launch": ops},
            "context": "Paper IV: 32 agents in 0.7 s on an RTX 2080 (JAX/CuPy), another machine "
                       "and benchmark instance"}
    if not args.no_cpu_baseline:
        from oracle import multiagent as ma
        p0 = ma.MAProblem(dim=3, n_p=100, T=10.0, start=sc.start[0], goal=sc.goal[0],
                          radius=float(sc.radius[0]), height=float(sc.height[0]), **rho)
        n_cpu = 40
        t0 = time.perf_counter()
        ma.solve(p0, n_cpu)
        t_it = (time.perf_counter() - t0) / n_cpu
        mean_it = float(np.mean(it[out["residual"] <= tol])) if n_conv else float(cap)
        line["cpu_baseline"] = {"value": 1.0 / (t_it * mean_it), "unit": "scenes/s",
                                "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"scene 0, {n_cpu} iterations timed ({t_it:.3f} s per "
                                          f"iteration), scaled by the GPU's mean iteration "
                                          f"count per converged scene ({mean_it:.0f})"}
    print(json.dumps(line), flush=True)
    h.close()


def footprint_ops(n_p, n_o, n_c, iters):
    """FP32 lane operations per trajectory for `iters` iterations of the footprint
    method (+ the initial pass). Per grid point: the containment test of each
    circle against each ellipse [footprint offset 2 FMA + the 9 of the point test],
    the evaluations of x, y (value, speed, acceleration), c, s and psi [9 x 11 FMA]
    and of c, s, psi for the heading step [3 x 11], the speed and acceleration
    tests [8], the contractions F^T r [88] and P^T (psi^ - psi) [11]. Per
    trajectory: the xi-step [44 x 44 FMA] and the heading step [11 x 11]."""
    per_t = n_c * n_o * 11 + 99 + 33 + 8 + 88 + 11
    return (n_p * per_t + 44 * 44 + 11 * 11) * (np.asarray(iters, np.float64) + 1.0)


def run_footprint(args, torch):
    """Paper II's batch optimizer for a rectangular robot (3 circles, heading):
    1000 trajectories (125 scenes x 8 initialisations, 20 moving ellipses each),
    a fixed number of iterations; one step = one batch solve."""
    from paper_2408_10731_b300 import scenes, footprint as gfp, trajbatch
    b = scenes.config2(args.seed, n_scenes=125, inits=8, n_obstacles=20)
    d = b.goal - b.start
    head = np.arctan2(d[:, 1], d[:, 0])
    xpsi0 = np.repeat(head[b.traj_problem][:, None], 11, 1)
    offs, rc, iters = (-0.35, 0.0, 0.35), 0.15, 100
    h = gfp.from_batch(b, head, head, xpsi0, offs, rc)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        h.solve(iters, -1.0, stats=False)
    torch.cuda.synchronize()
    clk = ClockSampler(_pci_id(torch, 0), interval_ms=20)
    clk.mark()
    ms = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream); h.solve(iters, -1.0, stats=False); e1.record(stream); e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk.mark()
    clocks = clk.stop()
    step_ms = float(np.mean(ms))
    out = h.get_trajectories()
    e2e = []
    xi0 = np.concatenate([b.xi0[:, :2], xpsi0[:, None, :]], 1)
    for _ in range(max(1, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.set_initial(b.traj_problem, xi0)
        h.solve(iters, -1.0, stats=False)
        r = h.get_trajectories()
        e2e.append(time.perf_counter() - t0)
    ops = float(b.n_traj * footprint_ops(100, 20, len(offs), iters))
    fp32_peak = trajbatch.measure_fp32_peak(5)
    achieved = ops / (step_ms * 1e-3)
    line = {"metric": "ms per iteration, batch of 1000 trajectories (3-circle footprint with "
                      "heading, 20 moving ellipses)", "value": step_ms / iters, "unit": "ms",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "125 scenes x 8 initialisations N(straight line, 0.5 m), 2D, "
                                   "n_p=100 over 10 s, 20 constant-velocity ellipses (semi-axes "
                                   "U(0.2,0.8) m), footprint circles at -0.35/0/0.35 m of radius "
                                   f"0.15 m, heading fixed at both ends, {iters} fixed iterations",
                       "l2": "inputs and state stay on chip; one launch per step"},
            "residual_median": [float(np.median(out["residual"][:, k])) for k in range(4)],
            "e2e": {"value": float(np.mean(e2e)) * 1e3 / iters, "unit": "ms",
                    "h2d_bytes_per_step": int(xi0.astype(np.float32).nbytes + b.traj_problem.nbytes),
                    "d2h_bytes_per_step": int(r["xi"].nbytes + r["residual"].nbytes + r["iterations"].nbytes)},
            "gpu_launches": 1, "clocks": clocks,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fp32_peak / 2e12,
                         "unit": "Top/s", "frac": achieved / (fp32_peak / 2.0), "traffic": None,
                         "kernel": "k_fp_solve<4>",
                         "peak_source": "measured FFMA microbenchmark (traj_measure_fp32_peak), "
                                        "FP32 lane-ops/s",
                         "algorithmic_ops_per_launch": ops},
            "context": "Paper II reports 4.5 ms per iteration at a batch of 1000 on its (unnamed) GPU"}
    if not args.no_cpu_baseline:
        from oracle import footprint as fp
        c, a, v = b.obstacles(0)
        prob = fp.FPProblem(n_p=100, T=float(b.duration[0]), start=b.start[0], goal=b.goal[0],
                            psi0=float(head[0]), psif=float(head[0]), centers=np.asarray(c, float),
                            semi_axes=np.asarray(a, float), velocities=np.asarray(v, float),
                            offsets=np.asarray(offs), r_circle=rc, vmax=b.vmax, amax=b.amax,
                            rho=b.rho)
        idx = np.nonzero(b.traj_problem == 0)[0]
        t0 = time.perf_counter()
        fp.solve(prob, xi0[idx], 20)
        t_it = (time.perf_counter() - t0) / 20
        line["cpu_baseline"] = {"value": t_it * 1e3 * b.n_traj / len(idx), "unit": "ms",
                                "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"scene 0 ({len(idx)} trajectories), 20 iterations, "
                                          "scaled to 1000 trajectories per iteration"}
    print(json.dumps(line), flush=True)
    h.close()


def run_mpc(args, torch):
    """Paper II's MPC use of the batch optimizer: 125 scenes x 8 plans (B = 1000), each
    control step shifts the horizon by 0.1 s (the robot follows each scene's best plan,
    the obstacles move on, the multipliers carry over) and runs 10 warm-started
    iterations. One bench step = one control step; episodes of 10 control steps start
    from a converged plan (the episode set-up is outside the timed region)."""
    from paper_2408_10731_b300 import scenes, trajbatch
    b = scenes.config2(args.seed, n_scenes=125, inits=8)
    h = trajbatch.from_batch(b)
    iters, delta, episode = 10, 0.1, 10
    stream = torch.cuda.current_stream()
    res = torch.empty(b.n_traj, 3).pin_memory()
    coeffs = torch.empty(b.n_traj, 2, 11).pin_memory()

    def start_episode():
        h.set_problems(b.n_steps, b.duration, b.start, b.goal)
        h.set_obstacles(b.offsets, b.centers, b.semi_axes, b.velocities)
        h.set_initial(b.traj_problem, b.xi0)
        h.solve(500, 1e-3)

    def control_step():  # one CUDA graph: shift, boundary update, solve
        h.mpc_step(delta, iters, 1e-3)

    def control_step_calls():  # the same step as two calls
        h.shift_horizon(delta)
        h.solve(iters, 1e-3, stats=False)

    def shape_of(w, bps, team):
        return {"warps_per_block": w, "blocks_per_sm": bps, "warps_per_trajectory": team}

    # launch shape of the solve: the caller's, else the one whose control steps ran
    # fastest over a short trial of each candidate (outside the timed region)
    if args.shape:
        w, bps, team = (int(x) for x in args.shape.split(","))
        h.set_launch_shape(w, bps, team)
        shape = dict(shape_of(w, bps, team), fixed=True)
    else:
        trial = {}
        for w, bps, team in ((0, 0, 1), (1, 0, 1), (2, 0, 1), (8, 0, 1), (2, 0, 2), (4, 0, 2)):
            h.set_launch_shape(w, bps, team)
            start_episode()
            for _ in range(3):
                control_step()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                control_step()
            e1.record(stream); e1.synchronize()
            trial[(w, bps, team)] = e0.elapsed_time(e1) / 5
        best = min(trial, key=trial.get)
        h.set_launch_shape(*best)
        shape = dict(shape_of(*best), tuned_on="5 control steps per candidate",
                     trial_ms={f"{w},{bps},{t}": round(v, 4) for (w, bps, t), v in trial.items()})

    def episodes(step_fn, clk=None):
        start_episode()
        for _ in range(args.warmup):
            step_fn()
        ms, solved_frac, e2e = [], [], []
        if clk:
            clk.mark()
        k = 0
        while len(ms) < args.steps:
            if k % episode == 0:
                start_episode()
            k += 1
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(stream)
            step_fn()
            e1.record(stream)
            # end to end: the plans and residuals back to the host every control step
            h.get_trajectories(coeffs, res, None, None)
            e2e.append(time.perf_counter() - t0)
            ms.append(e0.elapsed_time(e1))
            worst = res.numpy().max(axis=1).reshape(b.n_problems, 8)
            solved_frac.append(float((worst.min(axis=1) <= 1e-3).mean()))
        if clk:
            clk.mark()
        return ms, solved_frac, e2e

    clk = ClockSampler(_pci_id(torch, 0), interval_ms=20)
    ms, solved_frac, e2e = episodes(control_step, clk)
    clocks = clk.stop()
    ms_calls, _, e2e_calls = episodes(control_step_calls)
    step_ms = float(np.mean(ms))
    line = {"metric": "ms per MPC control step (horizon shift + 10 warm-started iterations), "
                      "B = 1000", "value": step_ms, "unit": "ms", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "125 scenes x 8 plans of the 2D moving-ellipse workload (n_p=100 "
                                   "over 10 s, 50 ellipses), shift 0.1 s per control step onto "
                                   "each scene's smallest-residual plan, obstacles moved by their "
                                   "velocity, multipliers carried, 10 iterations (tol 1e-3); "
                                   "episodes of 10 control steps from a converged plan",
                       "l2": "state and inputs stay on the device; each control step is one "
                             "CUDA graph launch (traj_mpc_step: shift kernels, obstacle "
                             "packing, boundary update, solve)",
                       "launch_shape": shape},
            "scenes_with_a_solved_plan": float(np.mean(solved_frac)),
            "e2e": {"value": 1e3 * float(np.mean(e2e)), "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(coeffs.numel() * 4 + res.numel() * 4)},
            "gpu_launches": 6,  # 3 shift kernels, obstacle packing, boundary update, solve
            "clocks": clocks,
            "forms": {"separate_calls": {
                "ms_per_step": float(np.mean(ms_calls)), "e2e_ms": 1e3 * float(np.mean(e2e_calls)),
                "calls": "traj_shift_horizon then traj_solve, the kernels launched one by one"}},
            "context": "Paper II: 10 iterations at a batch of 1000 within its 0.04 s MPC budget "
                       "(JAX, unnamed GPU)"}
    print(json.dumps(line), flush=True)
    h.close()


def run_gemm(args, torch):
    """The warm-start network's tcgen05 BF16 GEMM (C = A B^T, FP32 accumulate): the
    training shapes of the network (4096 rows: 400 -> 256, 256 -> 256, 256 -> 176)
    and a square 8192^3 problem for the tensor roofline."""
    from paper_2408_10731_b300 import trajbatch
    dev = torch.device("cuda")
    g = torch.Generator(device=dev).manual_seed(args.seed)
    stream = torch.cuda.current_stream()
    peak = None
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks):
        with open(peaks) as fh:
            peak = json.load(fh).get("bf16_tflops")
    shapes = [(4096, 256, 400), (4096, 256, 256), (4096, 176, 256), (8192, 8192, 8192)]
    out = {}
    for M, N, K in shapes:
        A = torch.randn(M, K, generator=g, device=dev).to(torch.bfloat16)
        B = torch.randn(N, K, generator=g, device=dev).to(torch.bfloat16)
        C = torch.empty(M, N, device=dev)
        err = torch.zeros(1, dtype=torch.int32, device=dev)
        for _ in range(args.warmup):
            trajbatch.gemm_bf16(A, B, C, err)
        torch.cuda.synchronize()
        ms = []
        big_shape = (M, N, K) == (8192, 8192, 8192)
        if big_shape:
            clk = ClockSampler(_pci_id(torch, 0), interval_ms=20)
            clk.mark()
        for _ in range(max(5, args.steps)):
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream); trajbatch.gemm_bf16(A, B, C, err); e1.record(stream); e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        if big_shape:
            clk.mark()
            clocks = clk.stop()
        t = float(np.median(ms))
        ref = (A[:64].float() @ B.float().T)
        rel = float((C[:64] - ref).abs().max() / ref.abs().max())
        assert int(err.item()) == 0 and rel < 1e-2, (M, N, K, rel)
        out[f"{M}x{N}x{K}"] = {"ms": t, "tflops": 2.0 * M * N * K / (t * 1e-3) / 1e12}
    big = out["8192x8192x8192"]
    line = {"metric": "BF16 GEMM TFLOP/s (tcgen05, 128x128 tiles, FP32 accumulate), 8192^3",
            "value": big["tflops"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": big["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "C = A B^T with A [M, K], B [N, K] normal draws in BF16, C in FP32",
                       "l2": "the 8192^3 operands (256 MB) exceed L2"},
            "shapes": out, "gpu_launches": 1, "clocks": clocks,
            "roofline": {"bound": "tensor", "achieved": big["tflops"], "peak": peak,
                         "unit": "TFLOP/s", "frac": big["tflops"] / peak if peak else None,
                         "traffic": None, "kernel": "k_gemm_bf16<0, 128>",
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)"}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_split"],
                    help="tensor-core form of the headline (and of the plain_<precision> form)")
    ap.add_argument("--scenes", type=int, default=4096,
                    help="held-out scenes of the config5 workload (8 trajectories each)")
    ap.add_argument("--max-iters", type=int, default=500)
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workload", default="config5",
                    choices=["config5", "config2", "uneven", "long", "priest", "multiagent",
                             "footprint", "gemm", "mpc"])
    ap.add_argument("--ma-agents", type=int, default=32)
    ap.add_argument("--ma-scenes", type=int, default=148)
    ap.add_argument("--ma-radius", type=float, default=0.4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-warmstart", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--ws-scenes", type=int, default=200000)
    ap.add_argument("--rho-ladder", default="10,1.3,30",
                    help="penalty continuation of the extra *_rho_ladder forms: levels,growth,every")
    ap.add_argument("--no-rho-ladder", action="store_true")
    ap.add_argument("--shape", default=None,
                    help="FP32 launch shape W,B,T (warps per block, blocks per SM, warps per "
                         "trajectory) instead of the autotuned one")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_2408_10731_b300 import build as cuda_build, scenes, trajbatch

    cuda_build.build()
    if args.workload == "priest":
        return run_priest(args, torch)
    if args.workload == "multiagent":
        return run_multiagent(args, torch)
    if args.workload == "footprint":
        return run_footprint(args, torch)
    if args.workload == "gemm":
        return run_gemm(args, torch)
    if args.workload == "mpc":
        return run_mpc(args, torch)
    return run_solve(args, torch, dist, world, rank, local)


def heldout_scenes(rank=0, n_scenes=4096):
    """The learned warm start's held-out set: config-2-style scenes (seed 99 + rank),
    8 random initialisations N(straight line, 0.5 m) each."""
    from paper_2408_10731_b300 import scenes
    return scenes.ellipse_scenes(99 + rank, n_scenes, inits=8)


def run_solve(args, torch, dist, world, rank, local):
    """The batch solve workloads (config5 = default, config2, uneven, long): one step is
    one batch solve of the form, initialisation included (the learned warm start's
    features and network run inside the timed step)."""
    import dataclasses
    from paper_2408_10731_b300 import autotune, scenes, trajbatch
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    wl = args.workload
    if wl == "config5":
        batch = heldout_scenes(rank, args.scenes)
    elif wl == "uneven":
        batch = scenes.config4(args.seed + rank)
    elif wl == "long":
        batch = scenes.long_horizon(args.seed + rank, n_scenes=128, inits=8, n_steps=1000)
    else:
        batch = scenes.config2(args.seed + rank)
    tc = args.precision  # the tensor-core form of the headline
    use_tc = not args.no_mixed and wl != "long"
    use_ws = not args.no_warmstart and wl in ("config5", "config2")
    ladder = None if args.no_rho_ladder or wl not in ("config5", "config2") else \
        tuple(f(x) for f, x in zip((int, float, int), args.rho_ladder.split(",")))

    def tuned_handle(prec, ladder_on=False):
        hh = trajbatch.from_batch(batch, precision=prec)
        if ladder_on:
            hh.set_rho_schedule(*ladder)
        if args.shape and prec == "fp32":
            w, bps, team = (int(x) for x in args.shape.split(","))
            hh.set_launch_shape(w, bps, team)
            return hh, {"warps_per_block": w, "blocks_per_sm": bps, "warps_per_trajectory": team,
                        "fixed": True}
        return hh, autotune.tuned(hh, batch, prec, iters=100)

    handles, shapes = {}, {}
    handles["fp32"], shapes["fp32"] = tuned_handle("fp32")
    if use_tc:
        handles[tc], shapes[tc] = tuned_handle(tc)
        # the other tensor-core form, reported beside (split hi/lo BF16 operands: error
        # against FP64 near the FP32 form's; or the single BF16 operands)
        other = "mixed_split" if tc == "mixed" else "mixed"
        if not (other == "mixed_split" and wl == "uneven"):  # four horizons' hi/lo operands
            handles[other], shapes[other] = tuned_handle(other)  # exceed a CTA's shared memory
    if ladder:
        handles["fp32_ladder"], shapes["fp32_ladder"] = tuned_handle("fp32", True)
        if use_tc:
            handles[tc + "_ladder"], shapes[tc + "_ladder"] = tuned_handle(tc, True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sampler = ClockSampler(_pci_id(torch, local))
    fp32_peak = trajbatch.measure_fp32_peak(5) if rank == 0 else None
    mufu_peak = trajbatch.measure_mufu_peak(5) if rank == 0 else None

    xi0_rand = torch.as_tensor(batch.xi0, dtype=torch.float32, device="cuda")
    line = np.stack([scenes.straight_line_coeffs(batch.start[p], batch.goal[p])
                     for p in range(batch.n_problems)])[batch.traj_problem]
    xi0_line = torch.as_tensor(scenes.f32(line), dtype=torch.float32, device="cuda")
    forms = {"plain_fp32": ("fp32", xi0_rand)}
    if wl == "config5":
        forms["plain_fp32_straight"] = ("fp32", xi0_line)
    if use_tc:
        forms[f"plain_{tc}"] = (tc, xi0_rand)
        for k in handles:
            if k in ("mixed", "mixed_split") and k != tc:
                forms[f"plain_{k}"] = (k, xi0_rand)
    if ladder:
        forms["plain_fp32_rho_ladder"] = ("fp32_ladder", xi0_rand)
    ws = None
    if use_ws:
        from paper_2408_10731_b300 import warmstart
        ws, ws_info = warmstart.trained(seed=1000, n_scenes=args.ws_scenes, epochs=20,
                                        max_rows=max(4096, batch.n_problems))
        staged = ws.stage(batch)  # the scenes resident on the device before the timed steps

        def ws_init(hh):
            prop = ws.propose(staged).reshape(batch.n_traj, 2, 11)
            hh.set_initial(None, prop)
        forms["warmstart_fp32"] = ("fp32", ws_init)
        if use_tc:
            forms[f"warmstart_{tc}"] = (tc, ws_init)
            if ladder:
                forms[f"warmstart_{tc}_rho_ladder"] = (tc + "_ladder", ws_init)

    def run_form(form, steps):
        key, init = form
        hh = handles[key]
        if not callable(init):
            hh.set_initial(None, init)
        step_ms, kern_ms, solved = [], [], []
        for _ in range(steps):
            flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if callable(init):
                init(hh)
            hh.solve(args.max_iters, args.tol, stats=False)
            e1.record(stream)
            e1.synchronize()
            # outside the events: the solve's own kernel time and the solved count
            st = hh.last_stats()
            step_ms.append(e0.elapsed_time(e1)); kern_ms.append(st["gpu_ms"]); solved.append(st["n_solved"])
        return step_ms, kern_ms, solved, hh.get_trajectories()

    results = {}
    barrier()
    sampler.mark()
    for name, form in forms.items():
        run_form(form, args.warmup)
        barrier()
        results[name] = run_form(form, args.steps)
    barrier()
    sampler.mark()
    clocks = sampler.stop()
    headline = next(f for f in (f"warmstart_{tc}", f"plain_{tc}", "plain_fp32") if f in results)
    h_step_ms, h_kern_ms, h_solved, h_out = results[headline]
    hkey = forms[headline][0]
    hh = handles[hkey]

    # end to end through the public API with pinned host buffers (headline form)
    tp_h = batch.traj_problem.astype(np.int32)
    xi0_h = torch.from_numpy(batch.xi0.astype(np.float32)).pin_memory()
    res = {k: torch.empty(s, dtype=d).pin_memory() for k, s, d in (
        ("coeffs", (batch.n_traj, batch.dim, 11), torch.float32),
        ("residual", (batch.n_traj, 3), torch.float32), ("iters", (batch.n_traj,), torch.int32),
        ("status", (batch.n_traj,), torch.int8))}
    # the scene's obstacle arrays held in pinned host memory, as a serving process would
    scene_h = {k: torch.from_numpy(np.ascontiguousarray(getattr(batch, k), np.float32)).pin_memory()
               for k in ("centers", "semi_axes", "velocities")}
    e2e_s, e2e_solved = [], []
    for _ in range(max(3, min(20, args.steps // 2))):
        flush.fill_(1.0); torch.cuda.synchronize()
        t0 = time.perf_counter()
        if headline.startswith("warmstart"):
            # features copy the scene (obstacles, start, goal, offsets) host -> device
            Xw, lw = ws.features(batch, host=scene_h)
            prop = ws.forward(Xw, lw).reshape(batch.n_traj, 2, 11)
            hh.set_initial(None, prop)
        else:
            hh.set_initial(tp_h, xi0_h)
        hh.solve(args.max_iters, args.tol, stats=False)
        hh.get_trajectories(res["coeffs"], res["residual"], res["iters"], res["status"])
        e2e_s.append(time.perf_counter() - t0)
        e2e_solved.append(int((res["status"].numpy() == 0).sum()))
    scene_bytes = 3 * batch.centers.size * 4 + batch.start.nbytes + batch.goal.nbytes + \
        batch.offsets.astype(np.int32).nbytes
    h2d = scene_bytes if headline.startswith("warmstart") else xi0_h.numel() * 4 + tp_h.nbytes
    d2h = sum(t.numel() * t.element_size() for t in res.values())

    total_ms = float(np.sum(h_step_ms))
    n_solved = float(np.sum(h_solved))
    e2e_val = float(np.mean(e2e_solved)) / float(np.mean(e2e_s))
    total_ms_max, n_solved_all, e2e_all = combine_ranks(
        dist if world > 1 else None, world, total_ms, n_solved, e2e_val, device="cuda")
    value = n_solved_all / (total_ms_max * 1e-3)

    def kern_of(key):
        prec = key.split("_ladder")[0]
        return kernel_name(prec, shapes.get(key), int(batch.n_steps.max()))

    form_summary = {}
    for name, (sm, km, sv, o) in results.items():
        ok = o["status"] == 0
        key = forms[name][0]
        ops = algorithmic_ops(batch, o["iters"])
        form_summary[name] = {"kernel": kern_of(key), "launch_shape": shapes.get(key),
                              "solved_per_s": float(np.sum(sv)) / (float(np.sum(sm)) * 1e-3),
                              "ms_per_batch_solve": float(np.mean(sm)),
                              "solve_kernel_ms": float(np.mean(km)),
                              "solved_per_step": float(np.mean(sv)),
                              "scenes_with_a_solution": float(ok.reshape(batch.n_problems, -1).any(1).mean()),
                              "iters_median_solved": float(np.median(o["iters"][ok])) if ok.any() else None,
                              "iters_p90_solved": float(np.percentile(o["iters"][ok], 90)) if ok.any() else None,
                              "solve_roofline_frac": (ops / (float(np.mean(km)) * 1e-3) / (fp32_peak / 2.0))
                              if fp32_peak else None}

    if rank == 0:
        # roofline of the headline step's dominant kernel (the solve): FP32 lane operations
        # against the measured FFMA rate, and MUFU operations against the measured rsqrtf rate
        ops = algorithmic_ops(batch, h_out["iters"])
        mufu = algorithmic_mufu(batch, h_out["iters"])
        kern_s = float(np.mean(h_kern_ms)) * 1e-3
        achieved = ops / kern_s
        peak_ops = fp32_peak / 2.0  # FFMA rate in lane-operations/s (2 FLOP per FMA)
        kern = kern_of(hkey)
        wl_key = {"config5": "config5", "config2": "config2", "uneven": "uneven", "long": "long"}[wl]
        traffic = measured_traffic(kern, wl_key)
        workload = {"config5": WORKLOAD_CONFIG5.format(n=batch.n_problems, b=batch.n_traj),
                    "config2": WORKLOAD, "uneven": WORKLOAD_UNEVEN, "long": WORKLOAD_LONG}[wl]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+bf16" if hkey != "fp32" else "f32",
            "data": "synthetic",
            "config": {"workload": workload, "precision": hkey, "launch_shape": shapes.get(hkey),
                       "l2": "flushed between timed steps (256 MB write, outside the events)",
                       "per_rank_batch": "seed + rank",
                       "rho_ladder_forms": (None if not ladder else
                                            {"levels": ladder[0], "growth": ladder[1],
                                             "every": ladder[2], "rho0": batch.rho})},
            "ms_per_batch_solve": float(np.mean(h_step_ms)),
            "ms_per_batch_solve_plain_fp32": float(np.mean(results["plain_fp32"][0])),
            "solved_per_s_plain_fp32": form_summary["plain_fp32"]["solved_per_s"],
            "solved_per_step": float(np.mean(h_solved)), "trajectories_per_step": batch.n_traj,
            "iters": {"min": int(h_out["iters"].min()), "median": int(np.median(h_out["iters"])),
                      "max": int(h_out["iters"].max())},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": "Top/s", "frac": achieved / peak_ops, "traffic": traffic,
                         "kernel": kern,
                         "peak_source": "measured FFMA microbenchmark "
                         "(traj_measure_fp32_peak), FP32 lane-ops/s",
                         "algorithmic_ops_per_launch": ops,
                         "count": "the method's dense count: every trajectory x obstacle x grid "
                                  "point test, including those the kernel's exact cull skips "
                                  "(their projections are zero); ncu's FMA-pipe activity is the "
                                  "executed share (profiles/)",
                         "mufu": {"achieved": mufu / kern_s / 1e12, "peak": mufu_peak / 1e12,
                                  "unit": "T rsqrt/s", "frac": mufu / kern_s / mufu_peak,
                                  "algorithmic_per_launch": mufu,
                                  "peak_source": "measured rsqrtf microbenchmark "
                                                 "(traj_measure_mufu_peak)"}},
            "e2e": {"value": e2e_all, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": args.steps * (7 if headline.startswith("warmstart") else 1),
            "clocks": clocks,
            "headline_form": headline, "forms": form_summary,
            "source_digest": {k: source_digest(k) for k in KERNEL_SOURCES},
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_both(batch, wl)
        print(json.dumps(line), flush=True)
    for hx in handles.values():
        hx.close()
    if ws is not None:
        ws.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
