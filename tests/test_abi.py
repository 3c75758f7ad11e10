"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point that include/trajbatch.h declares, and rejects bad
configurations before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2408_10731_b300 import trajbatch as tb

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "trajbatch.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(traj_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("traj_batch_create", "traj_batch_destroy", "traj_set_problems",
              "traj_set_obstacles", "traj_set_initial", "traj_solve", "traj_get_trajectories",
              "traj_status_string", "traj_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(tb.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    lib = tb.load_library()
    assert lib.traj_status_string(0) == b"TRAJ_OK"
    assert lib.traj_status_string(-4) == b"TRAJ_ESHAPE"


@pytest.mark.parametrize("kw,frag", [
    (dict(dim=4), "dim"), (dict(max_steps=1025), "capacities"), (dict(vmax=-1.0), "vmax"),
    (dict(max_traj=0), "capacities"), (dict(precision="fp32", rho=0.0), "rho")])
def test_config_validation_without_device(kw, frag):
    args = dict(dim=2, max_problems=1, max_traj=4, max_obstacles=4, max_steps=50, vmax=1.5,
                amax=2.0)
    args.update(kw)
    with pytest.raises(tb.TrajBatchError) as e:
        tb.TrajBatch(**args)
    assert e.value.code == -1 and frag in str(e.value)


def test_no_cpu_fallback_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tb.TrajBatchError) as e:
        tb.TrajBatch(2, 1, 4, 4, 50, 1.5, 2.0)
    assert e.value.code == -3  # TRAJ_ECUDA: no CPU path exists


def test_solve_noalloc_refuses_host_arrays_and_short_tensors_before_the_library():
    """The allocation-free solve hands its array arguments to the kernels as they
    are; the binding refuses a numpy array or a CPU tensor (a host pointer the
    kernels would dereference) with ValueError, before any call into the library."""
    import numpy as np
    import torch
    from paper_2408_10731_b300 import scenes
    b = scenes.config2(0, n_scenes=1, inits=2)
    n_obs = int(b.offsets[-1])
    args = dict(centers=torch.zeros(n_obs, 2), semi_axes=torch.zeros(n_obs, 2),
                velocities=torch.zeros(n_obs, 2), traj_problem=torch.zeros(2, dtype=torch.int32),
                coeffs0=torch.zeros(2, 2, 11), coeffs=torch.zeros(2, 2, 11),
                residual=torch.zeros(2, 3), iters=torch.zeros(2, dtype=torch.int32),
                status=torch.zeros(2, dtype=torch.int8))

    def call(**over):
        a = dict(args, **over)
        tb.solve_noalloc(2, 1.5, 2.0, 1.0, b.n_steps, b.duration, b.start, b.goal, b.offsets,
                         a["centers"], a["semi_axes"], a["velocities"], a["traj_problem"],
                         a["coeffs0"], 10, 1e-3, a["coeffs"], a["residual"], a["iters"],
                         a["status"])

    with pytest.raises(ValueError, match="centers must be a CUDA tensor"):
        call(centers=np.zeros((n_obs, 2), np.float32))
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        call()  # CPU tensors are host memory too
