"""Python binding of the joint multi-agent optimizer (Paper IV, Algorithm 5) in
libtrajbatch.so (traj_ma_* in include/trajbatch.h): argument marshalling only.

Every step runs in the library's CUDA kernels (one CTA per scene); without the
built library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
import numpy as np

from . import trajbatch as _tb
from .scenes import MAScenes

_c_int, _c_float, _vp = ctypes.c_int, ctypes.c_float, ctypes.c_void_p


class MAConfig(ctypes.Structure):
    _fields_ = [("dim", _c_int), ("max_scenes", _c_int), ("max_agents", _c_int),
                ("max_obstacles", _c_int), ("n_steps", _c_int), ("rho", _c_float),
                ("rho_levels", _c_int), ("rho_growth", _c_float), ("rho_every", _c_int)]


class MAStats(ctypes.Structure):
    _fields_ = [("gpu_ms", _c_float), ("n_converged", _c_int), ("max_iters_run", _c_int),
                ("lambda_in_shared", _c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_BOUND = False


def _lib():
    global _BOUND
    lib = _tb.load_library()
    if not _BOUND:
        lib.traj_ma_create.argtypes = [ctypes.POINTER(MAConfig), _vp, ctypes.POINTER(_vp)]
        lib.traj_ma_destroy.argtypes = [_vp]
        lib.traj_ma_set_problems.argtypes = [_vp, _c_int, _c_int] + [_vp] * 8
        lib.traj_ma_solve.argtypes = [_vp, _c_int, _c_float, ctypes.POINTER(MAStats)]
        lib.traj_ma_get_trajectories.argtypes = [_vp, _vp, _vp, _vp]
        lib.traj_ma_last_error.argtypes = [_vp]
        lib.traj_ma_last_error.restype = ctypes.c_char_p
        for n in ("traj_ma_create", "traj_ma_destroy", "traj_ma_set_problems", "traj_ma_solve",
                  "traj_ma_get_trajectories"):
            getattr(lib, n).restype = _c_int
        _BOUND = True
    return lib


class MultiAgentBatch:
    """Handle of the C struct traj_ma_batch."""

    def __init__(self, dim, max_scenes, max_agents, max_obstacles, n_steps, rho=1.0,
                 rho_levels=1, rho_growth=1.0, rho_every=0, stream=None):
        self._lib = _lib()
        self.dim, self.n_steps = dim, n_steps
        self.stream = stream if stream is not None else _tb._default_stream()
        cfg = MAConfig(dim, max_scenes, max_agents, max_obstacles, n_steps, rho, rho_levels,
                       rho_growth, rho_every)
        h = _vp()
        rc = self._lib.traj_ma_create(ctypes.byref(cfg), self.stream, ctypes.byref(h))
        if rc != 0:
            raise _tb.TrajBatchError(rc, self._lib.traj_ma_last_error(None).decode())
        self._h = h
        self.n_scenes = self.n_agents = 0

    def _check(self, rc):
        if rc < 0:
            raise _tb.TrajBatchError(rc, self._lib.traj_ma_last_error(self._h).decode())
        return rc

    def set_problems(self, sc: MAScenes):
        keep = []

        def p(x, dt):
            ptr, k = _tb._ptr(x, dt)
            keep.append(k)
            return ptr
        self._check(self._lib.traj_ma_set_problems(
            self._h, sc.n_scenes, sc.n_agents, p(sc.duration, np.float64),
            p(sc.start, np.float64), p(sc.goal, np.float64), p(sc.radius, np.float32),
            p(sc.height, np.float32), p(sc.obs_offsets, np.int32),
            p(sc.obs_centers if len(sc.obs_radii) else None, np.float32),
            p(sc.obs_radii if len(sc.obs_radii) else None, np.float32)))
        self.n_scenes, self.n_agents = sc.n_scenes, sc.n_agents

    def solve(self, max_iters, tol=-1.0, stats=True):
        st = MAStats()
        self._check(self._lib.traj_ma_solve(self._h, int(max_iters), float(tol),
                                            ctypes.byref(st) if stats else None))
        return st.as_dict() if stats else None

    def get_trajectories(self):
        xi = np.zeros((self.n_scenes, self.n_agents, self.dim, 11), np.float32)
        res = np.zeros(self.n_scenes, np.float32)
        it = np.zeros(self.n_scenes, np.int32)
        self._check(self._lib.traj_ma_get_trajectories(self._h, xi.ctypes.data, res.ctypes.data,
                                                       it.ctypes.data))
        return dict(xi=xi, residual=res, iterations=it)

    def get_into(self, coeffs=None, residual=None, iters=None):
        """Copy results into caller-owned arrays or tensors (host or device)."""
        self._check(self._lib.traj_ma_get_trajectories(
            self._h, _tb._ptr(coeffs, np.float32)[0], _tb._ptr(residual, np.float32)[0],
            _tb._ptr(iters, np.int32)[0]))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.traj_ma_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_scenes(sc: MAScenes, rho=1.0, rho_levels=1, rho_growth=1.0, rho_every=0, stream=None):
    h = MultiAgentBatch(sc.dim, sc.n_scenes, sc.n_agents, max(1, len(sc.obs_radii)), sc.n_steps,
                        rho, rho_levels, rho_growth, rho_every, stream)
    h.set_problems(sc)
    return h
