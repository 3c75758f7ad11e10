"""Python binding of libtrajbatch.so (include/trajbatch.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels. There is no CPU
fallback: if the shared library is missing, or no CUDA device is present,
the calls raise.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); they are
passed to the C ABI as raw pointers. The stream defaults to torch's current
CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_c_int, _c_double, _c_void_p, _c_float = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_float

STATUS_NAMES = {0: "TRAJ_OK", 1: "TRAJ_NOT_CONVERGED", -1: "TRAJ_EINVAL", -2: "TRAJ_ENOMEM",
                -3: "TRAJ_ECUDA", -4: "TRAJ_ESHAPE", -5: "TRAJ_ETIMEOUT", -6: "TRAJ_ENAN",
                -7: "TRAJ_ESTATE"}
TRAJ_CONVERGED, TRAJ_CAP, TRAJ_NAN, TRAJ_TIMEOUT = 0, 1, 2, 3
PRECISION = {"fp32": 0, "mixed": 1, "mixed_split": 2}
COST_MODE = {"smooth_track": 0, "project": 1}


class TrajConfig(ctypes.Structure):
    _fields_ = [("dim", _c_int), ("degree", _c_int), ("max_problems", _c_int),
                ("max_traj", _c_int), ("max_obstacles", _c_int), ("max_steps", _c_int),
                ("vmax", _c_double), ("amax", _c_double), ("rho", _c_double),
                ("w_smooth", _c_double), ("w_track", _c_double), ("precision", _c_int),
                ("cost_mode", _c_int), ("cuda_stream", _c_void_p)]


class SolveStats(ctypes.Structure):
    _fields_ = [("n_traj", _c_int), ("n_solved", _c_int), ("iters_min", _c_int),
                ("iters_median", _c_int), ("iters_max", _c_int), ("max_res_obs", _c_float),
                ("max_res_v", _c_float), ("max_res_a", _c_float), ("gpu_ms", _c_float)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class LaunchShape(ctypes.Structure):
    _fields_ = [("warps_per_block", _c_int), ("blocks_per_sm", _c_int),
                ("warps_per_trajectory", _c_int), ("occupancy", _c_int)]


class SamplerConfig(ctypes.Structure):
    _fields_ = [("n_inner", _c_int), ("n_proj", _c_int), ("n_elite", _c_int), ("gamma", _c_float),
                ("sigma_lr", _c_float), ("eps", _c_float), ("w_res", _c_float),
                ("seed", ctypes.c_ulonglong), ("w_curv", _c_float), ("w_path", _c_float)]


class SamplerTrace(ctypes.Structure):
    _fields_ = [("samples", _c_void_p), ("projected", _c_void_p), ("residual", _c_void_p),
                ("cost_aug", _c_void_p), ("proj_idx", _c_void_p), ("elite_idx", _c_void_p)]


class TrajBatchError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_LIB = None
_vp = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load_library():
    """Load the in-tree shared library; raise loudly if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libtrajbatch.so is not built ({path}); run "
                           "paper_2408_10731_b300.build.build() or __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    lib.traj_batch_create.argtypes = [ctypes.POINTER(TrajConfig), ctypes.POINTER(_vp)]
    lib.traj_batch_destroy.argtypes = [_vp]
    lib.traj_set_problems.argtypes = [_vp, _c_int, _vp, _vp, _vp, _vp]
    lib.traj_set_obstacles.argtypes = [_vp, _vp, _vp, _vp, _vp]
    lib.traj_set_initial.argtypes = [_vp, _c_int, _vp, _vp]
    lib.traj_solve.argtypes = [_vp, _c_int, _c_float, _c_double, ctypes.POINTER(SolveStats)]
    lib.traj_get_solve_stats.argtypes = [_vp, ctypes.POINTER(SolveStats)]
    lib.traj_get_trajectories.argtypes = [_vp, _vp, _vp, _vp, _vp]
    lib.traj_get_state.argtypes = [_vp, _vp, _vp]
    lib.traj_set_state.argtypes = [_vp, _vp, _vp, _vp]
    lib.traj_set_rho_schedule.argtypes = [_vp, _c_int, _c_double, _c_int]
    lib.traj_set_workspace.argtypes = [_vp, _vp, _vp]
    lib.traj_shift_horizon.argtypes = [_vp, _c_double, _vp]
    lib.traj_mpc_step.argtypes = [_vp, _c_double, _vp, _c_int, _c_float, _c_double]
    lib.traj_homotopy_signature.argtypes = [_vp, _vp]
    lib.traj_status_string.argtypes = [_c_int]
    lib.traj_status_string.restype = ctypes.c_char_p
    lib.traj_last_error.argtypes = [_vp]
    lib.traj_last_error.restype = ctypes.c_char_p
    lib.traj_measure_fp32_peak.argtypes = [_vp, _c_int, ctypes.POINTER(_c_double)]
    lib.traj_measure_mufu_peak.argtypes = [_vp, _c_int, ctypes.POINTER(_c_double)]
    lib.traj_set_launch_shape.argtypes = [_vp, ctypes.POINTER(LaunchShape)]
    lib.traj_get_launch_info.argtypes = [_vp, ctypes.POINTER(LaunchShape), ctypes.POINTER(_c_int),
                                         ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]
    lib.traj_autotune.argtypes = [_vp, _c_int, ctypes.POINTER(LaunchShape),
                                  ctypes.POINTER(_c_float)]
    lib.traj_sampler_step.argtypes = [_vp, ctypes.POINTER(SamplerConfig), _c_int, _vp, _vp, _vp,
                                      _vp, ctypes.POINTER(SamplerTrace)]
    lib.traj_sampler_step_multi.argtypes = [_vp, ctypes.POINTER(SamplerConfig), _c_int, _c_int,
                                            _vp, _vp, _vp, _vp, ctypes.POINTER(SamplerTrace)]
    lib.traj_gemm_bf16.argtypes = [_c_int, _c_int, _c_int, _vp, _vp, _vp, _vp, _vp]
    lib.traj_solve_noalloc.argtypes = [ctypes.POINTER(TrajConfig), _c_int, _vp, _vp, _vp, _vp,
                                       _vp, _vp, _vp, _vp, _c_int, _vp, _vp, _c_int, _c_float,
                                       _vp, _vp, _vp, _vp]
    for name in ("traj_batch_create", "traj_batch_destroy", "traj_set_problems",
                 "traj_set_obstacles", "traj_set_initial", "traj_solve", "traj_get_solve_stats",
                 "traj_get_trajectories", "traj_get_state", "traj_set_state", "traj_set_rho_schedule", "traj_set_workspace", "traj_shift_horizon", "traj_mpc_step", "traj_homotopy_signature", "traj_measure_fp32_peak", "traj_measure_mufu_peak",
                 "traj_solve_noalloc", "traj_set_launch_shape", "traj_get_launch_info", "traj_autotune",
                 "traj_sampler_step", "traj_sampler_step_multi", "traj_gemm_bf16"):
        getattr(lib, name).restype = _c_int
    _LIB = lib
    return lib


def _ptr(x, dtype):
    """(pointer, keepalive) of a numpy array or torch tensor, checked for dtype/contiguity."""
    if x is None:
        return None, None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32,
                   np.int8: torch.int8}[dtype]
            if x.dtype != tdt or not x.is_contiguous():
                raise TypeError(f"tensor must be contiguous {tdt}, got {x.dtype}")
            return x.data_ptr(), x
    except ImportError:
        pass
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
        x = np.ascontiguousarray(x, dtype=dtype)
    return x.ctypes.data, x


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def measure_fp32_peak(reps: int = 5, stream=None) -> float:
    lib = load_library()
    out = ctypes.c_double(0.0)
    rc = lib.traj_measure_fp32_peak(stream if stream is not None else _default_stream(), reps,
                                    ctypes.byref(out))
    if rc != 0:
        raise TrajBatchError(rc, "FFMA microbenchmark failed")
    return out.value


def measure_mufu_peak(reps: int = 5, stream=None) -> float:
    """rsqrtf/s of the MUFU microbenchmark (traj_measure_mufu_peak)."""
    lib = load_library()
    out = ctypes.c_double(0.0)
    rc = lib.traj_measure_mufu_peak(stream if stream is not None else _default_stream(), reps,
                                    ctypes.byref(out))
    if rc != 0:
        raise TrajBatchError(rc, "MUFU microbenchmark failed")
    return out.value


class TrajBatch:
    """Handle of one batch (C struct traj_batch); mirrors the C entry points."""

    def __init__(self, dim, max_problems, max_traj, max_obstacles, max_steps, vmax, amax,
                 rho=1.0, w_smooth=1.0, w_track=1.0, precision="fp32", cost_mode="smooth_track",
                 stream=None):
        self._lib = load_library()
        self.dim = dim
        self.stream = stream if stream is not None else _default_stream()
        cfg = TrajConfig(dim, 10, max_problems, max_traj, max_obstacles, max_steps, vmax, amax,
                         rho, w_smooth, w_track, PRECISION[precision], COST_MODE[cost_mode],
                         self.stream)
        h = _vp()
        rc = self._lib.traj_batch_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != 0:
            raise TrajBatchError(rc, self._lib.traj_last_error(None).decode())
        self._h = h
        self.n_traj = 0

    def _check(self, rc, ok=(0,)):
        if rc not in ok:
            raise TrajBatchError(rc, self._lib.traj_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._lib.traj_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_problems(self, n_steps, duration, start, goal):
        n, kn = _ptr(np.asarray(n_steps), np.int32)
        d, kd = _ptr(np.asarray(duration), np.float64)
        s, ks = _ptr(np.asarray(start), np.float64)
        g, kg = _ptr(np.asarray(goal), np.float64)
        self._check(self._lib.traj_set_problems(self._h, int(np.asarray(n_steps).shape[0]), n, d, s, g))

    def set_obstacles(self, offsets, centers, semi_axes, velocities):
        o, ko = _ptr(np.asarray(offsets), np.int32)
        c, kc = _ptr(centers, np.float32)
        a, ka = _ptr(semi_axes, np.float32)
        v, kv = _ptr(velocities, np.float32)
        self._check(self._lib.traj_set_obstacles(self._h, o, c, a, v))

    def set_initial(self, traj_problem, coeffs0):
        """traj_problem None: replace only the coefficients (same trajectories)."""
        x, kx = _ptr(coeffs0, np.float32)
        if traj_problem is None:
            self._check(self._lib.traj_set_initial(self._h, self.n_traj, None, x))
            return
        tp, kt = _ptr(np.asarray(traj_problem), np.int32)
        n = int(np.asarray(traj_problem).shape[0])
        self._check(self._lib.traj_set_initial(self._h, n, tp, x))
        self.n_traj = n

    def solve(self, max_iters, tol=1e-3, timeout_ms=0.0, stats=True):
        st = SolveStats()
        rc = self._lib.traj_solve(self._h, int(max_iters), float(tol), float(timeout_ms),
                                  ctypes.byref(st) if stats else None)
        self._check(rc, ok=(0, 1) if stats else (0,))
        return st.as_dict() if stats else None

    def last_stats(self):
        """Statistics of the last solve (synchronises)."""
        st = SolveStats()
        self._check(self._lib.traj_get_solve_stats(self._h, ctypes.byref(st)), ok=(0, 1))
        return st.as_dict()

    def get_trajectories(self, coeffs=None, residual=None, iters=None, status=None):
        """Into the given buffers (host or device); allocates numpy arrays if all are None."""
        alloc = coeffs is None and residual is None and iters is None and status is None
        if alloc:
            coeffs = np.zeros((self.n_traj, self.dim, 11), np.float32)
            residual = np.zeros((self.n_traj, 3), np.float32)
            iters = np.zeros(self.n_traj, np.int32)
            status = np.zeros(self.n_traj, np.int8)
        c, kc = _ptr(coeffs, np.float32)
        r, kr = _ptr(residual, np.float32)
        i, ki = _ptr(iters, np.int32)
        s, ks = _ptr(status, np.int8)
        self._check(self._lib.traj_get_trajectories(self._h, c, r, i, s))
        return dict(xi=coeffs, residual=residual, iters=iters, status=status)

    def set_launch_shape(self, warps_per_block, blocks_per_sm=0, warps_per_trajectory=1,
                         occupancy=0):
        self._check(self._lib.traj_set_launch_shape(
            self._h, ctypes.byref(LaunchShape(int(warps_per_block), int(blocks_per_sm),
                                              int(warps_per_trajectory), int(occupancy)))))

    def launch_info(self):
        """The shape the last solve launch resolved to (warps per block, resident blocks
        per SM, warps per trajectory) and its grid."""
        shape, grid, regs, smem = LaunchShape(), _c_int(0), _c_int(0), _c_int(0)
        self._check(self._lib.traj_get_launch_info(self._h, ctypes.byref(shape), ctypes.byref(grid),
                                                   ctypes.byref(regs), ctypes.byref(smem)))
        return dict(warps_per_block=shape.warps_per_block, blocks_per_sm=shape.blocks_per_sm,
                    warps_per_trajectory=shape.warps_per_trajectory, occupancy=shape.occupancy,
                    grid=grid.value, registers=regs.value, shared_bytes=smem.value)

    def autotune(self, iters=20):
        """Time the candidate launch shapes on this batch; keep and return the fastest."""
        shape, ms = LaunchShape(), _c_float(0.0)
        self._check(self._lib.traj_autotune(self._h, int(iters), ctypes.byref(shape),
                                            ctypes.byref(ms)))
        return dict(warps_per_block=shape.warps_per_block, blocks_per_sm=shape.blocks_per_sm,
                    warps_per_trajectory=shape.warps_per_trajectory, occupancy=shape.occupancy,
                    ms=ms.value)

    def sampler_step(self, cfg: dict, iteration, mu, sigma, best, z=None, trace=None,
                     n_dist=None):
        """One outer iteration of the projection-guided sampler (device tensors). With
        n_dist, the decentralised form: mu [n_dist][D], sigma [n_dist][D][D] and best
        [n_dist][D + 1], each distribution refined from its own n_traj / n_dist samples."""
        sc = SamplerConfig(int(cfg["n_inner"]), int(cfg["n_proj"]), int(cfg["n_elite"]),
                           float(cfg["gamma"]), float(cfg["sigma_lr"]), float(cfg["eps"]),
                           float(cfg.get("w_res", 1.0)), int(cfg.get("seed", 0)),
                           float(cfg.get("w_curv", 0.0)), float(cfg.get("w_path", 0.0)))
        tr = None
        if trace is not None:
            tr = SamplerTrace(*[_ptr(trace.get(k), dt)[0] for k, dt in (
                ("samples", np.float32), ("projected", np.float32), ("residual", np.float32),
                ("cost_aug", np.float32), ("proj_idx", np.int32), ("elite_idx", np.int32))])
        args = (_ptr(mu, np.float32)[0], _ptr(sigma, np.float32)[0], _ptr(z, np.float32)[0],
                _ptr(best, np.float32)[0], ctypes.byref(tr) if tr is not None else None)
        if n_dist is None:
            self._check(self._lib.traj_sampler_step(self._h, ctypes.byref(sc), int(iteration),
                                                    *args))
        else:
            self._check(self._lib.traj_sampler_step_multi(self._h, ctypes.byref(sc),
                                                          int(iteration), int(n_dist), *args))

    def get_state(self):
        lam = np.zeros((self.n_traj, self.dim, 11), np.float32)
        u = np.zeros((self.n_traj, self.dim, 11), np.float32)
        self._check(self._lib.traj_get_state(self._h, _ptr(lam, np.float32)[0],
                                             _ptr(u, np.float32)[0]))
        return dict(lam=lam, u=u)

    def set_workspace(self, lower=None, upper=None):
        """Workspace bounds lower <= p(t) <= upper per problem ([n_problems][dim]); None
        removes them."""
        if lower is None and upper is None:
            self._check(self._lib.traj_set_workspace(self._h, None, None))
            return
        lp, kl = _ptr(np.asarray(lower, np.float64), np.float64)
        hp, kh = _ptr(np.asarray(upper, np.float64), np.float64)
        self._check(self._lib.traj_set_workspace(self._h, lp, hp))

    def set_rho_schedule(self, levels=1, growth=1.0, every=0):
        """Penalty continuation: rho * growth^l for l < levels, one level up after every
        `every`-th unconverged iteration (levels = 1: the fixed penalty)."""
        self._check(self._lib.traj_set_rho_schedule(self._h, int(levels), float(growth), int(every)))

    def homotopy_signature(self):
        """uint64 [n_traj]: bit j set when obstacle j (j < 64) is on the trajectory's left
        as they pass, at the closest approach (2D)."""
        sig = np.zeros(self.n_traj, np.uint64)
        self._check(self._lib.traj_homotopy_signature(self._h, sig.ctypes.data))
        return sig

    def shift_horizon(self, delta, executed=None):
        """Receding-horizon step: the robot followed executed[p] (None: per problem the
        trajectory with the smallest worst residual) for delta seconds; the next solve
        starts from the shifted iterate and the carried multipliers."""
        ep, ke = (None, None) if executed is None else _ptr(np.asarray(executed), np.int32)
        self._check(self._lib.traj_shift_horizon(self._h, float(delta), ep))

    def mpc_step(self, delta, max_iters, tol=1e-3, executed=None, timeout_ms=0.0):
        """One control step, shift_horizon(delta, executed) then solve(max_iters, tol)
        without statistics, replayed as one CUDA graph (bitwise the two calls)."""
        ep, ke = (None, None) if executed is None else _ptr(np.asarray(executed), np.int32)
        self._check(self._lib.traj_mpc_step(self._h, float(delta), ep, int(max_iters),
                                            float(tol), float(timeout_ms)))

    def set_state(self, xi, lam, u):
        """Resume the next solves from an exported (xi, lambda, u) state."""
        xp, kx = _ptr(xi, np.float32)
        lp, kl = _ptr(lam, np.float32)
        up, ku = _ptr(u, np.float32)
        self._check(self._lib.traj_set_state(self._h, xp, lp, up))


def gemm_bf16(A, B, C, err, stream=None):
    """C = A B^T on the tensor cores (A [M,K], B [N,K] bf16 CUDA tensors, C [M,N] fp32)."""
    import torch
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and C.dtype == torch.float32
    M, K = A.shape
    N = B.shape[0]
    rc = load_library().traj_gemm_bf16(M, N, K, A.data_ptr(), B.data_ptr(), C.data_ptr(),
                                       err.data_ptr(),
                                       stream if stream is not None else _default_stream())
    if rc != 0:
        raise TrajBatchError(rc, load_library().traj_last_error(None).decode())


def solve_noalloc(dim, vmax, amax, rho, n_steps, duration, start, goal, obs_offsets, centers,
                  semi_axes, velocities, traj_problem, coeffs0, max_iters, tol, coeffs, residual,
                  iters, status, w_smooth=1.0, w_track=1.0, cost_mode="smooth_track", stream=None):
    """traj_solve_noalloc: the allocation-free solve. Obstacles, traj_problem, coeffs0 and
    the four outputs must be CUDA tensors of the sizes the problem arrays imply (the
    kernels read and write them directly, so a host array or a short tensor would be an
    out-of-bounds device access, not an error); the problem arrays are host arrays.
    Raises ValueError before any call into the library when one is not."""
    n_obs = int(np.asarray(obs_offsets)[-1])
    n_traj = int(traj_problem.shape[0]) if hasattr(traj_problem, "shape") else len(traj_problem)
    want = (("centers", centers, n_obs * dim), ("semi_axes", semi_axes, n_obs * dim),
            ("velocities", velocities, n_obs * dim), ("traj_problem", traj_problem, n_traj),
            ("coeffs0", coeffs0, n_traj * dim * 11), ("coeffs", coeffs, n_traj * dim * 11),
            ("residual", residual, n_traj * 3), ("iters", iters, n_traj),
            ("status", status, n_traj))
    for name, x, n in want:
        if not (hasattr(x, "is_cuda") and x.is_cuda):
            raise ValueError(f"solve_noalloc: {name} must be a CUDA tensor")
        if x.numel() < n:
            raise ValueError(f"solve_noalloc: {name} holds {x.numel()} values, needs {n}")
    lib = load_library()
    cfg = TrajConfig(dim, 10, 0, 0, 0, 0, vmax, amax, rho, w_smooth, w_track, 0,
                     COST_MODE[cost_mode], stream if stream is not None else _default_stream())
    n, kn = _ptr(np.asarray(n_steps), np.int32)
    d, kd = _ptr(np.asarray(duration), np.float64)
    s, ks = _ptr(np.asarray(start), np.float64)
    g, kg = _ptr(np.asarray(goal), np.float64)
    o, ko = _ptr(np.asarray(obs_offsets), np.int32)
    args = [_ptr(x, dt)[0] for x, dt in ((centers, np.float32), (semi_axes, np.float32),
                                         (velocities, np.float32))]
    tp = _ptr(traj_problem, np.int32)[0]
    x0 = _ptr(coeffs0, np.float32)[0]
    outs = [_ptr(x, dt)[0] for x, dt in ((coeffs, np.float32), (residual, np.float32),
                                         (iters, np.int32), (status, np.int8))]
    rc = lib.traj_solve_noalloc(ctypes.byref(cfg), int(np.asarray(n_steps).shape[0]), n, d, s, g,
                                o, *args, int(traj_problem.shape[0]), tp, x0, int(max_iters),
                                float(tol), *outs)
    if rc != 0:
        raise TrajBatchError(rc, lib.traj_last_error(None).decode())
    return rc


def from_batch(batch, precision="fp32", cost_mode="smooth_track", w_smooth=1.0, w_track=1.0,
               stream=None, max_traj=None) -> TrajBatch:
    """Create a handle sized for a scenes.Batch and load its problems, obstacles and xi0."""
    tb = TrajBatch(batch.dim, batch.n_problems, max_traj or batch.n_traj,
                   max(1, int(batch.offsets[-1])), int(batch.n_steps.max()), batch.vmax,
                   batch.amax, batch.rho, w_smooth, w_track, precision, cost_mode, stream)
    tb.set_problems(batch.n_steps, batch.duration, batch.start, batch.goal)
    tb.set_obstacles(batch.offsets, batch.centers.astype(np.float32),
                     batch.semi_axes.astype(np.float32), batch.velocities.astype(np.float32))
    tb.set_initial(batch.traj_problem, batch.xi0.astype(np.float32))
    return tb
