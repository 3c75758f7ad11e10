"""Python binding of the multi-circle footprint optimizer with heading (Paper II,
Algorithm 2) in libtrajbatch.so (traj_fp_* in include/trajbatch.h): argument
marshalling only. Every step runs in the library's CUDA kernels; without the
built library or a CUDA device the calls raise."""
from __future__ import annotations

import ctypes

import numpy as np

from . import trajbatch as _tb

_c_int, _c_float, _vp = ctypes.c_int, ctypes.c_float, ctypes.c_void_p


class FPConfig(ctypes.Structure):
    _fields_ = [("max_problems", _c_int), ("max_traj", _c_int), ("max_obstacles", _c_int),
                ("max_steps", _c_int), ("n_circles", _c_int), ("circle_offsets", _c_float * 8),
                ("r_circle", _c_float), ("vmax", _c_float), ("amax", _c_float),
                ("rho", _c_float), ("rho_psi", _c_float)]


class FPStats(ctypes.Structure):
    _fields_ = [("gpu_ms", _c_float), ("n_solved", _c_int), ("max_iters_run", _c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_BOUND = False


def _lib():
    global _BOUND
    lib = _tb.load_library()
    if not _BOUND:
        lib.traj_fp_create.argtypes = [ctypes.POINTER(FPConfig), _vp, ctypes.POINTER(_vp)]
        lib.traj_fp_destroy.argtypes = [_vp]
        lib.traj_fp_set_problems.argtypes = [_vp, _c_int] + [_vp] * 10
        lib.traj_fp_set_initial.argtypes = [_vp, _c_int, _vp, _vp]
        lib.traj_fp_solve.argtypes = [_vp, _c_int, _c_float, ctypes.POINTER(FPStats)]
        lib.traj_fp_get_trajectories.argtypes = [_vp, _vp, _vp, _vp]
        lib.traj_fp_last_error.argtypes = [_vp]
        lib.traj_fp_last_error.restype = ctypes.c_char_p
        for n in ("traj_fp_create", "traj_fp_destroy", "traj_fp_set_problems",
                  "traj_fp_set_initial", "traj_fp_solve", "traj_fp_get_trajectories"):
            getattr(lib, n).restype = _c_int
        _BOUND = True
    return lib


class FootprintBatch:
    """Handle of the C struct traj_fp_batch."""

    def __init__(self, max_problems, max_traj, max_obstacles, max_steps, offsets, r_circle,
                 vmax, amax, rho=1.0, rho_psi=1.0, stream=None):
        self._lib = _lib()
        offs = (_c_float * 8)(*([float(o) for o in offsets] + [0.0] * (8 - len(offsets))))
        cfg = FPConfig(max_problems, max_traj, max_obstacles, max_steps, len(offsets), offs,
                       r_circle, vmax, amax, rho, rho_psi)
        self.stream = stream if stream is not None else _tb._default_stream()
        h = _vp()
        rc = self._lib.traj_fp_create(ctypes.byref(cfg), self.stream, ctypes.byref(h))
        if rc != 0:
            raise _tb.TrajBatchError(rc, self._lib.traj_fp_last_error(None).decode())
        self._h = h
        self.n_traj = 0

    def _check(self, rc):
        if rc < 0:
            raise _tb.TrajBatchError(rc, self._lib.traj_fp_last_error(self._h).decode())
        return rc

    def set_problems(self, n_steps, duration, start, goal, heading_start, heading_goal,
                     obs_offsets, centers, semi_axes, velocities):
        keep = []

        def p(x, dt):
            ptr, k = _tb._ptr(x, dt)
            keep.append(k)
            return ptr
        n = len(n_steps)
        has = int(np.asarray(obs_offsets)[-1]) > 0
        self._check(self._lib.traj_fp_set_problems(
            self._h, n, p(n_steps, np.int32), p(duration, np.float64), p(start, np.float64),
            p(goal, np.float64), p(heading_start, np.float64), p(heading_goal, np.float64),
            p(obs_offsets, np.int32), p(centers if has else None, np.float32),
            p(semi_axes if has else None, np.float32), p(velocities if has else None, np.float32)))

    def set_initial(self, traj_problem, xi0):
        xi0 = np.ascontiguousarray(xi0, np.float32)
        tp = np.ascontiguousarray(traj_problem, np.int32)
        self._check(self._lib.traj_fp_set_initial(self._h, len(tp), tp.ctypes.data, xi0.ctypes.data))
        self.n_traj = len(tp)

    def solve(self, max_iters, tol=-1.0, stats=True):
        st = FPStats()
        self._check(self._lib.traj_fp_solve(self._h, int(max_iters), float(tol),
                                            ctypes.byref(st) if stats else None))
        return st.as_dict() if stats else None

    def get_trajectories(self):
        xi = np.zeros((self.n_traj, 5, 11), np.float32)
        res = np.zeros((self.n_traj, 4), np.float32)
        it = np.zeros(self.n_traj, np.int32)
        self._check(self._lib.traj_fp_get_trajectories(self._h, xi.ctypes.data, res.ctypes.data,
                                                       it.ctypes.data))
        return dict(xi=xi, residual=res, iterations=it)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.traj_fp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_batch(batch, heading_start, heading_goal, xi_psi0, offsets, r_circle, rho_psi=1.0,
               stream=None):
    """A handle over a scenes.Batch (2D): its problems, obstacles and initial x, y,
    with the given end headings [P] and initial heading coefficients [n_traj][11]."""
    B = batch.n_traj
    xi0 = np.concatenate([np.asarray(batch.xi0, np.float64)[:, :2],
                          np.asarray(xi_psi0, np.float64).reshape(B, 1, 11)], 1)
    h = FootprintBatch(batch.n_problems, B, max(1, int(batch.offsets[-1])),
                       int(np.max(batch.n_steps)), offsets, r_circle, batch.vmax, batch.amax,
                       batch.rho, rho_psi, stream)
    h.set_problems(batch.n_steps, batch.duration, batch.start, batch.goal, heading_start,
                   heading_goal, batch.offsets, batch.centers, batch.semi_axes, batch.velocities)
    h.set_initial(batch.traj_problem, xi0)
    return h
