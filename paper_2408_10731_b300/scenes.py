"""Seeded synthetic scenes for the batched trajectory optimizer.

This module only draws inputs: problem descriptions (horizon, duration, start,
goal), obstacle sets and initial coefficient sets. It holds none of the
method's arithmetic, and both the CUDA path and the CPU oracle consume what it
returns. Every floating-point array that the GPU receives in FP32 is rounded
through float32 here, so that the FP64 oracle sees bit-identical inputs.

The paper's benchmarks (crowd simulator scenes, the BARN dataset, Gazebo
worlds) are not available; these generators stand in for them with the
shapes the thesis describes: a holonomic point robot, Bernstein degree-10
coefficients per axis, moving axis-aligned elliptical obstacles (Paper II
problem statement) and sphere obstacles on box surfaces that emulate the
down-sampled point clouds of the PRIEST experiments.

Data layout of a ``Batch`` (all numpy):
  dim            2 or 3
  n_steps[P]     int32, horizon n_p of each problem
  duration[P]    float64, horizon length T in seconds
  start[P,dim]   float64, goal[P,dim] float64
  offsets[P+1]   int32, CSR offsets of each problem's obstacles
  centers[N,dim], semi_axes[N,dim], velocities[N,dim]   float32-exact float64
  traj_problem[B] int32, problem index of each trajectory
  xi0[B,dim,11]  float32-exact float64, initial coefficients
  vmax, amax, rho  scalars
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_COEFF = 11  # Bernstein degree 10


def f32(x):
    """Round through float32 and return float64 (bit-identical inputs)."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@dataclasses.dataclass
class Batch:
    dim: int
    n_steps: np.ndarray
    duration: np.ndarray
    start: np.ndarray
    goal: np.ndarray
    offsets: np.ndarray
    centers: np.ndarray
    semi_axes: np.ndarray
    velocities: np.ndarray
    traj_problem: np.ndarray
    xi0: np.ndarray
    vmax: float
    amax: float
    rho: float = 1.0
    name: str = ""

    @property
    def n_problems(self) -> int:
        return int(self.n_steps.shape[0])

    @property
    def n_traj(self) -> int:
        return int(self.traj_problem.shape[0])

    def n_obstacles(self, p: int) -> int:
        return int(self.offsets[p + 1] - self.offsets[p])

    def obstacles(self, p: int):
        s, e = int(self.offsets[p]), int(self.offsets[p + 1])
        return self.centers[s:e], self.semi_axes[s:e], self.velocities[s:e]

    def subset(self, traj_idx) -> "Batch":
        """Same problems, a subset of the trajectories (in the given order)."""
        traj_idx = np.asarray(traj_idx, dtype=np.int64)
        return dataclasses.replace(self, traj_problem=self.traj_problem[traj_idx].copy(),
                                   xi0=self.xi0[traj_idx].copy())

    def select_problems(self, probs) -> "Batch":
        """Keep only the listed problems and their trajectories (re-indexed)."""
        probs = [int(p) for p in probs]
        remap = {p: k for k, p in enumerate(probs)}
        cen, ax, vel, offs = [], [], [], [0]
        for p in probs:
            c, a, v = self.obstacles(p)
            cen.append(c); ax.append(a); vel.append(v); offs.append(offs[-1] + c.shape[0])
        keep = np.array([k for k in range(self.n_traj) if int(self.traj_problem[k]) in remap],
                        dtype=np.int64)
        tp = np.array([remap[int(self.traj_problem[k])] for k in keep], dtype=np.int32)
        d = self.dim
        return dataclasses.replace(
            self, n_steps=self.n_steps[probs].copy(), duration=self.duration[probs].copy(),
            start=self.start[probs].copy(), goal=self.goal[probs].copy(),
            offsets=np.array(offs, dtype=np.int32),
            centers=np.concatenate(cen) if cen else np.zeros((0, d)),
            semi_axes=np.concatenate(ax) if ax else np.zeros((0, d)),
            velocities=np.concatenate(vel) if vel else np.zeros((0, d)),
            traj_problem=tp, xi0=self.xi0[keep].copy())


def straight_line_coeffs(start, goal) -> np.ndarray:
    """Bernstein coefficients of the constant-velocity segment start->goal.

    c_i = start + (goal - start) * i / 10, one row per axis: shape [dim, 11].
    Used only to centre the random initial guesses (an input, not a result).
    """
    start = np.asarray(start, dtype=np.float64)
    goal = np.asarray(goal, dtype=np.float64)
    i = np.arange(N_COEFF, dtype=np.float64) / (N_COEFF - 1)
    return start[:, None] + (goal - start)[:, None] * i[None, :]


def _inside(point, center, axes) -> bool:
    return float(np.sum(((np.asarray(point) - center) / axes) ** 2)) <= 1.0


# ---------------------------------------------------------------------------
# Config 1: 2D, 8 static circles, B=16, n_p=50, T=5 s (1' uses T=12 s).
# ---------------------------------------------------------------------------
def config1(seed: int = 0, feasible: bool = False) -> Batch:
    rng = np.random.default_rng(seed)
    radii = rng.uniform(0.3, 0.6, 8)
    centers = rng.uniform(1.0, 9.0, (8, 2))
    noise = rng.normal(0.0, 0.5, (16, 2, N_COEFF))
    start = np.array([0.0, 0.0]); goal = np.array([10.0, 10.0])
    T = 12.0 if feasible else 5.0
    xi0 = straight_line_coeffs(start, goal)[None] + noise
    return Batch(dim=2, n_steps=np.array([50], np.int32), duration=np.array([T]),
                 start=start[None].copy(), goal=goal[None].copy(),
                 offsets=np.array([0, 8], np.int32), centers=f32(centers),
                 semi_axes=f32(np.stack([radii, radii], 1)),
                 velocities=np.zeros((8, 2)), traj_problem=np.zeros(16, np.int32),
                 xi0=f32(xi0), vmax=1.5, amax=2.0, rho=1.0,
                 name="config1_feasible" if feasible else "config1")


# ---------------------------------------------------------------------------
# Moving ellipses (config 2 / config 4 / config 5 scenes).
# ---------------------------------------------------------------------------
def _draw_ellipses(rng, n_o, lo, hi, start, goal, T):
    cen, vel, ax = [], [], []
    while len(cen) < n_o:
        a = rng.uniform(0.2, 0.8, 2)
        c = rng.uniform(lo, hi, 2)
        speed = rng.uniform(0.0, 1.0)
        heading = rng.uniform(0.0, 2.0 * math.pi)
        v = speed * np.array([math.cos(heading), math.sin(heading)])
        # reject obstacles covering the start at t=0 or the goal at t=T
        if _inside(start, c, a) or _inside(goal, c + v * T, a):
            continue
        cen.append(c); vel.append(v); ax.append(a)
    return np.array(cen).reshape(-1, 2), np.array(ax).reshape(-1, 2), np.array(vel).reshape(-1, 2)


def config2(seed: int = 0, n_scenes: int = 128, inits: int = 8, n_obstacles: int = 50,
            n_steps: int = 100) -> Batch:
    """2D, n_p=100 over T=10 s, 50 constant-velocity ellipses, start (0,0), goal (8,8)."""
    rng = np.random.default_rng(seed)
    start = np.array([0.0, 0.0]); goal = np.array([8.0, 8.0]); T = 0.1 * n_steps
    line = straight_line_coeffs(start, goal)
    cen, ax, vel, xi0, tp, offs = [], [], [], [], [], [0]
    for s in range(n_scenes):
        c, a, v = _draw_ellipses(rng, n_obstacles, 0.0, 8.0, start, goal, T)
        cen.append(c); ax.append(a); vel.append(v); offs.append(offs[-1] + n_obstacles)
        xi0.append(line[None] + rng.normal(0.0, 0.5, (inits, 2, N_COEFF)))
        tp.extend([s] * inits)
    P = n_scenes
    return Batch(dim=2, n_steps=np.full(P, n_steps, np.int32), duration=np.full(P, T),
                 start=np.tile(start, (P, 1)), goal=np.tile(goal, (P, 1)),
                 offsets=np.array(offs, np.int32), centers=f32(np.concatenate(cen)),
                 semi_axes=f32(np.concatenate(ax)), velocities=f32(np.concatenate(vel)),
                 traj_problem=np.array(tp, np.int32), xi0=f32(np.concatenate(xi0)),
                 vmax=1.5, amax=2.0, rho=1.0, name=f"config2_seed{seed}")


def ellipse_scenes(seed: int, n_scenes: int, n_obstacles: int = 50, inits: int = 0,
                   n_steps: int = 100) -> Batch:
    """Many config-2-style scenes drawn in bulk (warm-start training and held-out sets).

    Same distributions as config2 (semi-axes U(0.2,0.8), centres U([0,8]^2), speed
    U(0,1), heading U(0,2pi), start/goal covering rejected), drawn per scene in
    vectorised rounds of candidates; the first n_obstacles accepted candidates of
    each scene are kept. `inits` random initialisations N(straight line, 0.5 m).
    """
    rng = np.random.default_rng(seed)
    start = np.array([0.0, 0.0]); goal = np.array([8.0, 8.0]); T = 0.1 * n_steps
    S, n = n_scenes, n_obstacles
    cen = np.zeros((S, n, 2)); ax = np.zeros((S, n, 2)); vel = np.zeros((S, n, 2))
    have = np.zeros(S, np.int64)
    while np.any(have < n):
        todo = np.nonzero(have < n)[0]
        m = 2 * n
        a = rng.uniform(0.2, 0.8, (todo.size, m, 2))
        c = rng.uniform(0.0, 8.0, (todo.size, m, 2))
        speed = rng.uniform(0.0, 1.0, (todo.size, m))
        head = rng.uniform(0.0, 2.0 * math.pi, (todo.size, m))
        v = speed[..., None] * np.stack([np.cos(head), np.sin(head)], -1)
        bad = (((start - c) / a) ** 2).sum(-1) <= 1.0
        bad |= (((goal - (c + v * T)) / a) ** 2).sum(-1) <= 1.0
        for r, sidx in enumerate(todo):
            ok = np.nonzero(~bad[r])[0][: n - have[sidx]]
            k0 = have[sidx]
            cen[sidx, k0:k0 + ok.size] = c[r, ok]; ax[sidx, k0:k0 + ok.size] = a[r, ok]
            vel[sidx, k0:k0 + ok.size] = v[r, ok]
            have[sidx] += ok.size
    line = straight_line_coeffs(start, goal)
    xi0 = (line[None] + rng.normal(0.0, 0.5, (S * inits, 2, N_COEFF))) if inits else \
        np.zeros((0, 2, N_COEFF))
    return Batch(dim=2, n_steps=np.full(S, n_steps, np.int32), duration=np.full(S, T),
                 start=np.tile(start, (S, 1)), goal=np.tile(goal, (S, 1)),
                 offsets=np.arange(S + 1, dtype=np.int32) * n, centers=f32(cen.reshape(-1, 2)),
                 semi_axes=f32(ax.reshape(-1, 2)), velocities=f32(vel.reshape(-1, 2)),
                 traj_problem=np.repeat(np.arange(S, dtype=np.int32), inits), xi0=f32(xi0),
                 vmax=1.5, amax=2.0, rho=1.0, name=f"ellipses_seed{seed}")


def long_horizon(seed: int = 0, n_scenes: int = 16, inits: int = 8, n_steps=1000,
                 n_obstacles: int = 10, dim: int = 2, moving: bool = True) -> Batch:
    """Long horizons in the spirit of Paper I (n_o = 10 obstacles, n_p = 1000 grid
    points; 2D static, 2D dynamic and 3D problems): grid spacing 0.01 s (T = 0.01 n_p),
    start at the origin, goal at distance 0.55 vmax T along the diagonal (in 3D with
    a rise of a quarter of the planar distance), n_obstacles axis-aligned ellipses
    (ellipsoids in 3D) with semi-axes U(0.2, 0.8) m, centres uniform in the box
    spanned by start and goal (z in [0, goal z + 1] in 3D), speed U(0, 1) m/s in a
    uniform random direction (zero when moving is False); obstacles covering the
    start at t = 0 or the goal at t = T are redrawn. n_steps is one horizon or one
    per scene. `inits` initialisations N(straight line, 0.5 m) per scene."""
    rng = np.random.default_rng(seed)
    vmax, amax = 1.5, 2.0
    n_np = np.broadcast_to(np.asarray(n_steps, np.int32), (n_scenes,)).copy()
    cen, ax, vel, xi0, tp, offs = [], [], [], [], [], [0]
    starts, goals, Ts = [], [], []
    for s in range(n_scenes):
        T = 0.01 * float(n_np[s])
        reach = 0.55 * vmax * T
        if dim == 2:
            goal = np.full(2, reach / math.sqrt(2.0))
        else:
            planar = reach / math.sqrt(1.0 + 1.0 / 16.0)
            goal = np.array([planar / math.sqrt(2.0), planar / math.sqrt(2.0), planar / 4.0])
        start = np.zeros(dim)
        hi = goal.copy()
        if dim == 3:
            hi[2] = goal[2] + 1.0
        c_l, a_l, v_l = [], [], []
        while len(c_l) < n_obstacles:
            a = rng.uniform(0.2, 0.8, dim)
            c = rng.uniform(np.zeros(dim), hi)
            speed = rng.uniform(0.0, 1.0) if moving else 0.0
            d = rng.normal(0.0, 1.0, dim)
            v = speed * d / max(np.linalg.norm(d), 1e-12)
            if _inside(start, c, a) or _inside(goal, c + v * T, a):
                continue
            c_l.append(c); a_l.append(a); v_l.append(v)
        cen.append(np.array(c_l)); ax.append(np.array(a_l)); vel.append(np.array(v_l))
        offs.append(offs[-1] + n_obstacles)
        xi0.append(straight_line_coeffs(start, goal)[None] +
                   rng.normal(0.0, 0.5, (inits, dim, N_COEFF)))
        tp.extend([s] * inits)
        starts.append(start); goals.append(goal); Ts.append(T)
    return Batch(dim=dim, n_steps=n_np, duration=np.array(Ts),
                 start=np.array(starts), goal=np.array(goals),
                 offsets=np.array(offs, np.int32), centers=f32(np.concatenate(cen)),
                 semi_axes=f32(np.concatenate(ax)), velocities=f32(np.concatenate(vel)),
                 traj_problem=np.array(tp, np.int32), xi0=f32(np.concatenate(xi0)),
                 vmax=vmax, amax=amax, rho=1.0,
                 name=f"long_horizon_{dim}d_seed{seed}")


def grazing(seed: int = 0, n_obstacles=(1, 2, 7, 24, 63, 64, 65, 130), inits: int = 4,
            n_steps=(33, 65, 100), dim: int = 2, noise: float = 0.02) -> Batch:
    """Obstacles that graze the straight start->goal path: one problem per
    (obstacle count, horizon) pair, obstacle j centred on the path at a uniform
    fraction of it and moved sideways by its own semi-axis times U(0.9, 1.1) along
    a random direction normal to the path (so that many grid points lie near an
    ellipse boundary), some static, some moving along or across the path at up to
    0.5 m/s; semi-axes U(0.2, 0.8) m, start at the origin, goal (8, 8) (3D: (8, 8,
    2)), T = 0.1 n_p s. `inits` initialisations: the straight line plus N(0, noise)
    on every coefficient."""
    rng = np.random.default_rng(seed)
    start = np.zeros(dim)
    goal = np.array([8.0, 8.0] if dim == 2 else [8.0, 8.0, 2.0])
    u = (goal - start) / np.linalg.norm(goal - start)
    problems = [(int(no), int(npt)) for no in n_obstacles for npt in n_steps]
    cen, ax, vel, offs, n_np, Ts = [], [], [], [0], [], []
    for no, npt in problems:
        T = 0.1 * npt
        a = rng.uniform(0.2, 0.8, (no, dim))
        frac = rng.uniform(0.05, 0.95, no)
        side = rng.normal(size=(no, dim))
        side -= (side @ u)[:, None] * u[None, :]
        side /= np.maximum(np.linalg.norm(side, axis=1, keepdims=True), 1e-12)
        # move by the semi-axis along the chosen direction (a point of the path then
        # sits near the ellipse boundary)
        reach = 1.0 / np.sqrt(((side / a) ** 2).sum(1))
        c = start + frac[:, None] * (goal - start) + side * (reach * rng.uniform(0.9, 1.1, no))[:, None]
        kind = rng.integers(0, 3, no)
        speed = rng.uniform(0.0, 0.5, no)
        v = np.where((kind == 0)[:, None], 0.0,
                     np.where((kind == 1)[:, None], u[None, :] * speed[:, None], side * speed[:, None]))
        c = c - v * (frac * T)[:, None]  # at the path point when the line passes it
        cen.append(c); ax.append(a); vel.append(v)
        offs.append(offs[-1] + no); n_np.append(npt); Ts.append(T)
    P = len(problems)
    line = straight_line_coeffs(start, goal)
    xi0 = line[None] + rng.normal(0.0, noise, (P * inits, dim, N_COEFF))
    return Batch(dim=dim, n_steps=np.array(n_np, np.int32), duration=np.array(Ts),
                 start=np.tile(start, (P, 1)), goal=np.tile(goal, (P, 1)),
                 offsets=np.array(offs, np.int32), centers=f32(np.concatenate(cen)),
                 semi_axes=f32(np.concatenate(ax)), velocities=f32(np.concatenate(vel)),
                 traj_problem=np.repeat(np.arange(P, dtype=np.int32), inits), xi0=f32(xi0),
                 vmax=1.5, amax=2.0, name=f"grazing_seed{seed}_{dim}d")


def config4(seed: int = 0, n_problems: int = 2048, inits: int = 8) -> Batch:
    """Uneven batch: n_o log-uniform in [4,256], n_p in {50,75,100,150}, T = 0.1 n_p."""
    rng = np.random.default_rng(seed)
    vmax = 1.5
    n_steps, dur, st, gl, cen, ax, vel, xi0, tp, offs = [], [], [], [], [], [], [], [], [], [0]
    for p in range(n_problems):
        n_o = int(round(math.exp(rng.uniform(math.log(4.0), math.log(256.0)))))
        n_p = int(rng.choice([50, 75, 100, 150]))
        T = 0.1 * n_p
        heading = rng.uniform(0.0, 2.0 * math.pi)
        dist = 0.55 * vmax * T
        start = np.zeros(2)
        goal = dist * np.array([math.cos(heading), math.sin(heading)])
        lo = np.minimum(start, goal) - 1.0; hi = np.maximum(start, goal) + 1.0
        c, a, v = _draw_ellipses(rng, n_o, lo, hi, start, goal, T)
        line = straight_line_coeffs(start, goal)
        n_steps.append(n_p); dur.append(T); st.append(start); gl.append(goal)
        cen.append(c); ax.append(a); vel.append(v); offs.append(offs[-1] + n_o)
        xi0.append(line[None] + rng.normal(0.0, 0.5, (inits, 2, N_COEFF)))
        tp.extend([p] * inits)
    return Batch(dim=2, n_steps=np.array(n_steps, np.int32), duration=np.array(dur),
                 start=np.array(st), goal=f32(np.array(gl)), offsets=np.array(offs, np.int32),
                 centers=f32(np.concatenate(cen)), semi_axes=f32(np.concatenate(ax)),
                 velocities=f32(np.concatenate(vel)), traj_problem=np.array(tp, np.int32),
                 xi0=f32(np.concatenate(xi0)), vmax=vmax, amax=2.0, rho=1.0,
                 name=f"config4_seed{seed}")


# ---------------------------------------------------------------------------
# Config 3: 3D, 256 spheres on the surfaces of 12 random boxes in 20x20x5 m.
# ---------------------------------------------------------------------------
def _box_surface_points(rng, lo, hi, n):
    """Uniform points on the union of box surfaces (box by area, face by area)."""
    size = hi - lo
    faces = []  # (box, axis, side, area)
    for b in range(lo.shape[0]):
        sx, sy, sz = size[b]
        for axis, area in ((0, sy * sz), (1, sx * sz), (2, sx * sy)):
            for side in (0, 1):
                faces.append((b, axis, side, area))
    areas = np.array([f[3] for f in faces])
    prob = areas / areas.sum()
    pts = np.empty((n, 3))
    for k in range(n):
        b, axis, side, _ = faces[int(rng.choice(len(faces), p=prob))]
        u = rng.uniform(0.0, 1.0, 3)
        p = lo[b] + u * size[b]
        p[axis] = hi[b, axis] if side else lo[b, axis]
        pts[k] = p
    return pts


def config3(seed: int = 0, n_traj: int = 4096, n_spheres: int = 256) -> dict:
    """Scene and sampler settings for the projection-guided sampler (3D)."""
    rng = np.random.default_rng(seed)
    start = np.array([1.0, 1.0, 1.0]); goal = np.array([19.0, 19.0, 4.0])
    ws_lo = np.array([0.0, 0.0, 0.0]); ws_hi = np.array([20.0, 20.0, 5.0])
    c = np.concatenate([rng.uniform(2.0, 18.0, (12, 2)), rng.uniform(0.0, 5.0, (12, 1))], 1)
    s = np.concatenate([rng.uniform(1.0, 4.0, (12, 2)), rng.uniform(1.0, 5.0, (12, 1))], 1)
    lo = np.clip(c - s / 2, ws_lo, ws_hi); hi = np.clip(c + s / 2, ws_lo, ws_hi)
    cen, rad = [], []
    while len(cen) < n_spheres:
        p = _box_surface_points(rng, lo, hi, 1)[0]
        r = rng.uniform(0.1, 0.3)
        if np.linalg.norm(p - start) <= r or np.linalg.norm(p - goal) <= r:
            continue
        cen.append(p); rad.append(r)
    cen = np.array(cen); rad = np.array(rad)
    batch = Batch(dim=3, n_steps=np.array([100], np.int32), duration=np.array([20.0]),
                  start=start[None].copy(), goal=goal[None].copy(),
                  offsets=np.array([0, n_spheres], np.int32), centers=f32(cen),
                  semi_axes=f32(np.stack([rad, rad, rad], 1)),
                  velocities=np.zeros((n_spheres, 3)),
                  traj_problem=np.zeros(n_traj, np.int32),
                  xi0=np.zeros((n_traj, 3, N_COEFF)), vmax=2.0, amax=2.0, rho=1.0,
                  name=f"config3_seed{seed}")
    mu0 = straight_line_coeffs(start, goal).reshape(-1)
    sigma0 = 4.0 * np.eye(3 * N_COEFF)
    return dict(batch=batch, mu0=f32(mu0), sigma0=f32(sigma0), n_outer=10, n_inner=20,
                n_proj=int(math.ceil(0.73 * n_traj)), n_elite=int(math.ceil(0.10 * n_traj)))


def normal_draws(seed: int, shape) -> np.ndarray:
    """Host-side standard normal draws (float32-exact) for sampler parity runs."""
    rng = np.random.default_rng(seed)
    return f32(rng.standard_normal(shape))


# ---- multi-agent scenes (Paper IV benchmarks) ---------------------------------------
@dataclasses.dataclass
class MAScenes:
    """A batch of multi-agent scenes with a common agent count and grid."""
    dim: int
    n_steps: int
    duration: np.ndarray      # [S]
    start: np.ndarray         # [S, N, dim]
    goal: np.ndarray          # [S, N, dim]
    radius: np.ndarray        # [S] agent radius r
    height: np.ndarray        # [S] agent half-height h (3D)
    obs_offsets: np.ndarray   # [S + 1]
    obs_centers: np.ndarray   # [n_obs, dim]
    obs_radii: np.ndarray     # [n_obs]
    name: str = ""

    @property
    def n_scenes(self):
        return self.start.shape[0]

    @property
    def n_agents(self):
        return self.start.shape[1]


def _ma_pack(dim, n_steps, T, start, goal, radius, obs, name):
    S = start.shape[0]
    offs = np.zeros(S + 1, np.int32)
    cen, rad = [], []
    for s in range(S):
        c, r = obs[s] if obs else (np.zeros((0, dim)), np.zeros(0))
        offs[s + 1] = offs[s] + len(r)
        cen.append(c)
        rad.append(r)
    return MAScenes(dim=dim, n_steps=n_steps, duration=np.full(S, float(T)),
                    start=f32(start), goal=f32(goal), radius=np.full(S, radius, np.float32),
                    height=np.full(S, radius, np.float32), obs_offsets=offs,
                    obs_centers=f32(np.concatenate(cen)) if cen else np.zeros((0, dim), np.float32),
                    obs_radii=f32(np.concatenate(rad)) if rad else np.zeros(0, np.float32),
                    name=name)


def ma_square(seed: int, n_scenes: int, n_agents: int, dim: int = 3, side: float = 8.0,
              radius: float = 0.25, jitter: float = 0.05, T: float = 10.0,
              n_steps: int = 100) -> MAScenes:
    """Square benchmark of Paper IV: agents evenly spaced on the perimeter of a
    side x side square (a random phase per scene), each going to the antipodal
    point through the centre; every coordinate jittered by U(-jitter, jitter);
    3D agents fly at z = 1 m. Agents are spheres (h = r)."""
    rng = np.random.default_rng(seed)
    start = np.zeros((n_scenes, n_agents, dim))
    goal = np.zeros_like(start)
    ctr = np.array([side / 2, side / 2])
    for s in range(n_scenes):
        phase = rng.uniform(0, 4 * side / n_agents)
        for k in range(n_agents):
            u = (phase + k * 4 * side / n_agents) % (4 * side)
            e, f = int(u // side), u % side
            p = [np.array([f, 0.0]), np.array([side, f]), np.array([side - f, side]),
                 np.array([0.0, side - f])][e]
            start[s, k, :2] = p
            goal[s, k, :2] = 2 * ctr - p
        if dim == 3:
            start[s, :, 2] = 1.0
            goal[s, :, 2] = 1.0
        start[s] += rng.uniform(-jitter, jitter, (n_agents, dim))
        goal[s] += rng.uniform(-jitter, jitter, (n_agents, dim))
    return _ma_pack(dim, n_steps, T, start, goal, radius, None,
                    f"ma_square_{n_agents}_seed{seed}")


def _separated(rng, n, lo, hi, min_sep, avoid=None):
    pts = []
    while len(pts) < n:
        p = rng.uniform(lo, hi)
        if all(np.linalg.norm(p - q) >= min_sep for q in pts):
            pts.append(p)
    return np.array(pts)


def ma_random(seed: int, n_scenes: int, n_agents: int, dim: int = 3, room: float = 8.0,
              radius: float = 0.25, n_obstacles: int = 0, obs_radius=(0.2, 0.4),
              T: float = 10.0, n_steps: int = 100) -> MAScenes:
    """Random benchmark of Paper IV: starts and goals uniform in a room x room
    square (3D: z in [0.5, 1.5] m) with pairwise separation >= 2r + 0.2 m among the
    starts and among the goals (rejection sampling); optionally n_obstacles static
    spheres of radius U(obs_radius), centres uniform in the room, redrawn while one
    covers a start or goal with margin r + 0.1 m."""
    rng = np.random.default_rng(seed)
    lo = np.array([0.0, 0.0, 0.5])[:dim]
    hi = np.array([room, room, 1.5])[:dim]
    start = np.zeros((n_scenes, n_agents, dim))
    goal = np.zeros_like(start)
    obs = []
    for s in range(n_scenes):
        start[s] = _separated(rng, n_agents, lo, hi, 2 * radius + 0.2)
        goal[s] = _separated(rng, n_agents, lo, hi, 2 * radius + 0.2)
        cen, rad = [], []
        while len(cen) < n_obstacles:
            c = rng.uniform(lo, hi)
            r = rng.uniform(*obs_radius)
            ends = np.concatenate([start[s], goal[s]])
            if np.all(np.linalg.norm(ends - c, axis=1) >= r + radius + 0.1):
                cen.append(c)
                rad.append(r)
        obs.append((np.array(cen).reshape(-1, dim), np.array(rad)))
    return _ma_pack(dim, n_steps, T, start, goal, radius, obs if n_obstacles else None,
                    f"ma_random_{n_agents}_seed{seed}")
