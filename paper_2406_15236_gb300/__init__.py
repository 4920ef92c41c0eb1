"""Python binding of the GB300 MPC step library (C ABI in include/mpc.h).

Argument marshalling only: every step of the method runs in the CUDA kernels of
``csrc/``.  Functions carry the C names (``mpc_create``, ``mpc_step``, ...); the
``Simulation`` class wraps a handle.  PyTorch supplies device memory (through the
handle's allocator callbacks) and the CUDA stream.

The library must be built (``paper_2406_15236_gb300._build.build()``) before import;
there is no CPU fallback -- import fails loudly when the CUDA library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

_LIB_PATH = _build.LIB

MPC_SRD, MPC_AT_A, MPC_SRD_A = 0, 1, 2
MPC_WALLS_NONE, MPC_WALLS_NO_SLIP, MPC_WALLS_SLIP = 0, 1, 2
MPC_OK, MPC_EINVAL, MPC_ENOMEM, MPC_ECUDA, MPC_ETIMEOUT, MPC_ESTATE = range(6)
MPC_FLAG_OBSERVABLES, MPC_FLAG_DEBUG_CELLS, MPC_FLAG_DETERMINISTIC = 1, 2, 4
MPC_BATCH_DETERMINISTIC, MPC_BATCH_AUTOTUNE, MPC_BATCH_PACK_ALL = 1, 2, 4
STATUS_NAMES = {0: "MPC_OK", 1: "MPC_EINVAL", 2: "MPC_ENOMEM", 3: "MPC_ECUDA",
                4: "MPC_ETIMEOUT", 5: "MPC_ESTATE"}
OBS_ROW = ["px", "py", "pz", "sum_v2", "skin_xy", "skin_yz", "skin_zx", "scol_xy", "scol_yx",
           "scol_yz", "scol_zy", "scol_zx", "scol_xz", "step", "r0", "r1"]


class MpcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class mpc_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32 * 3), ("a", ctypes.c_double), ("n_c", ctypes.c_double),
                ("h", ctypes.c_double), ("alpha_deg", ctypes.c_double), ("kT", ctypes.c_double),
                ("m", ctypes.c_double), ("variant", ctypes.c_int32),
                ("thermostat", ctypes.c_int32), ("walls_z", ctypes.c_int32),
                ("gravity", ctypes.c_double * 3), ("seed", ctypes.c_uint64),
                ("box_id", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("capacity", ctypes.c_int32), ("graph_steps", ctypes.c_int32),
                ("tile_particles", ctypes.c_int32), ("threads_per_cell", ctypes.c_int32),
                ("obs_ring", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("wall_u", ctypes.c_double * 2)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                               ctypes.c_void_p)


class mpc_allocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", _ALLOC_FN), ("release", _RELEASE_FN)]


class mpc_obs(ctypes.Structure):
    _fields_ = [("momentum", ctypes.c_double * 3), ("ekin", ctypes.c_double),
                ("temperature", ctypes.c_double), ("stress_kin", ctypes.c_double * 3),
                ("stress_col", ctypes.c_double * 6), ("n_particles", ctypes.c_int64),
                ("step", ctypes.c_int64), ("has_stress", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class mpc_info(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("step", ctypes.c_int64), ("fixed_bits", ctypes.c_int32),
                ("capacity", ctypes.c_int32), ("brick", ctypes.c_int32 * 3),
                ("n_bricks", ctypes.c_int32 * 3), ("device_bytes", ctypes.c_uint64),
                ("recoveries", ctypes.c_int32), ("threads_per_cell", ctypes.c_int32)]


class mpc_batch_config(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_uint64), ("graph_steps", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("max_boxes", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class mpc_batch_info(ctypes.Structure):
    _fields_ = [("n_boxes", ctypes.c_int32), ("work_items", ctypes.c_int32),
                ("n_particles", ctypes.c_int64), ("arena_bytes", ctypes.c_uint64),
                ("arena_used", ctypes.c_uint64), ("arena_largest_free", ctypes.c_uint64),
                ("grid", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("graph_builds", ctypes.c_int32),
                ("tuned_classes", ctypes.c_int32), ("solo_boxes", ctypes.c_int32),
                ("packed_launches", ctypes.c_int32), ("plan_ms", ctypes.c_float)]


MPC_SERVER_DETERMINISTIC, MPC_SERVER_SEQUENTIAL, MPC_SERVER_SHARE_ALL = 1, 2, 4
MPC_SERVER_FIRST_COME = 8
MPC_SERVER_AGED = 16
MPC_SERVER_BACKFILL = 32
MPC_SERVER_PRIORITY_HEAD = 64
MPC_JOB_QUEUED, MPC_JOB_RUNNING, MPC_JOB_DONE, MPC_JOB_FAILED = 0, 1, 2, 3
MPC_JOB_KEEP_SERIES, MPC_JOB_KEEP_STATE = 1, 2


class mpc_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("chunk_steps", ctypes.c_int32),
                ("max_active", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("fill_kparticles", ctypes.c_int32)]


class mpc_job(ctypes.Structure):
    _fields_ = [("params", mpc_params), ("steps", ctypes.c_int64), ("arrival_s", ctypes.c_double),
                ("keep", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


class mpc_job_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("error", ctypes.c_int32),
                ("arrival_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("finish_s", ctypes.c_double), ("steps", ctypes.c_int64),
                ("n_particles", ctypes.c_int64), ("eta_gk", ctypes.c_double),
                ("temperature", ctypes.c_double)]


class mpc_server_stats(ctypes.Structure):
    _fields_ = [("chunks", ctypes.c_int64), ("chunk_steps", ctypes.c_int64),
                ("gpu_ms", ctypes.c_double), ("host_gap_ms", ctypes.c_double),
                ("plan_ms", ctypes.c_double), ("graph_builds", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load the CUDA library; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"CUDA library {_LIB_PATH} is missing: run "
                          "paper_2406_15236_gb300._build.build() (needs nvcc, sm_103a)")
    L = ctypes.CDLL(_LIB_PATH)
    P, vp = ctypes.POINTER, ctypes.c_void_p
    L.mpc_create.argtypes = [P(mpc_params), vp, P(mpc_allocator), P(vp)]
    L.mpc_destroy.argtypes = [vp]
    L.mpc_step.argtypes = [vp, ctypes.c_int64]
    L.mpc_synchronize.argtypes = [vp]
    L.mpc_get_state.argtypes = [vp, vp, vp, vp, vp, P(ctypes.c_int64), ctypes.c_int]
    L.mpc_set_state.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int]
    L.mpc_get_cell_counts.argtypes = [vp, vp, ctypes.c_int]
    L.mpc_observables.argtypes = [vp, P(mpc_obs)]
    L.mpc_observable_series.argtypes = [vp, vp, ctypes.c_int64, P(ctypes.c_int64)]
    L.mpc_velocity_profile.argtypes = [vp, ctypes.c_int32, vp]
    L.mpc_get_info.argtypes = [vp, P(mpc_info)]
    L.mpc_set_profiling.argtypes = [vp, ctypes.c_int]
    L.mpc_profile_step_kernel.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_int32)]
    L.mpc_sort_by_cell_noalloc.argtypes = [P(ctypes.c_int32), ctypes.c_int64, vp, vp, vp, vp, vp,
                                           vp, vp]
    L.mpc_set_step_limit.argtypes = [vp, ctypes.c_int64]
    L.mpc_checkpoint_write.argtypes = [vp, ctypes.c_char_p]
    L.mpc_checkpoint_read.argtypes = [ctypes.c_char_p, vp, P(mpc_allocator), P(vp)]
    L.mpc_footprint.argtypes = [P(mpc_params), P(ctypes.c_uint64), P(ctypes.c_uint64)]
    L.mpc_autotune.argtypes = [P(mpc_params), vp, ctypes.c_uint64, P(ctypes.c_int32),
                               P(ctypes.c_int32), P(ctypes.c_double)]
    L.mpc_batch_create.argtypes = [P(mpc_batch_config), vp, P(vp)]
    L.mpc_batch_destroy.argtypes = [vp]
    L.mpc_batch_add.argtypes = [vp, P(mpc_params), P(vp)]
    L.mpc_batch_remove.argtypes = [vp, vp]
    L.mpc_batch_step.argtypes = [vp, ctypes.c_int64]
    L.mpc_batch_synchronize.argtypes = [vp]
    L.mpc_batch_get_info.argtypes = [vp, P(mpc_batch_info)]
    L.mpc_batch_last_error.argtypes = [vp]
    L.mpc_batch_last_error.restype = ctypes.c_char_p
    L.mpc_server_create.argtypes = [P(mpc_server_config), vp, P(vp)]
    L.mpc_server_destroy.argtypes = [vp]
    L.mpc_server_submit.argtypes = [vp, P(mpc_job), P(ctypes.c_int64)]
    L.mpc_server_run.argtypes = [vp, ctypes.c_double]
    L.mpc_server_job.argtypes = [vp, ctypes.c_int64, P(mpc_job_result)]
    L.mpc_server_get_stats.argtypes = [vp, P(mpc_server_stats)]
    L.mpc_server_job_series.argtypes = [vp, ctypes.c_int64, vp, ctypes.c_int64]
    L.mpc_server_job_state.argtypes = [vp, ctypes.c_int64, vp, vp, vp]
    L.mpc_server_last_error.argtypes = [vp]
    L.mpc_server_last_error.restype = ctypes.c_char_p
    L.mpc_last_error.argtypes = [vp]
    L.mpc_last_error.restype = ctypes.c_char_p
    L.mpc_version.restype = ctypes.c_char_p
    for name in ("mpc_create", "mpc_destroy", "mpc_step", "mpc_synchronize", "mpc_get_state",
                 "mpc_set_state", "mpc_get_cell_counts", "mpc_observables",
                 "mpc_observable_series", "mpc_velocity_profile", "mpc_get_info",
                 "mpc_set_profiling",
                 "mpc_profile_step_kernel", "mpc_sort_by_cell_noalloc", "mpc_set_step_limit",
                 "mpc_checkpoint_write", "mpc_checkpoint_read",
                 "mpc_footprint", "mpc_autotune", "mpc_batch_create", "mpc_batch_destroy",
                 "mpc_batch_add", "mpc_batch_remove", "mpc_batch_step", "mpc_batch_synchronize",
                 "mpc_batch_get_info", "mpc_server_create", "mpc_server_destroy",
                 "mpc_server_submit", "mpc_server_run", "mpc_server_job",
                 "mpc_server_job_series", "mpc_server_job_state", "mpc_server_get_stats"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status, handle=None):
    if status != MPC_OK:
        msg = lib().mpc_last_error(handle)
        raise MpcError(status, msg.decode() if msg else "")


def _check_server(status, server=None):
    if status != MPC_OK:
        msg = lib().mpc_server_last_error(server)
        raise MpcError(status, msg.decode() if msg else "")


def _check_batch(status, batch=None):
    if status != MPC_OK:
        msg = lib().mpc_batch_last_error(batch)
        raise MpcError(status, msg.decode() if msg else "")


def make_params(L=(16, 16, 16), n_c=10.0, h=0.1, alpha_deg=130.0, kT=1.0, m=1.0,
                variant=MPC_SRD, thermostat=0, walls_z=0, gravity=(0.0, 0.0, 0.0), seed=1,
                box_id=0, flags=0, capacity=0, graph_steps=0, tile_particles=0,
                threads_per_cell=0, obs_ring=0, wall_u=(0.0, 0.0)) -> mpc_params:
    if isinstance(L, int):
        L = (L, L, L)
    p = mpc_params()
    p.L[:] = list(L)
    p.a = 1.0
    p.n_c, p.h, p.alpha_deg, p.kT, p.m = n_c, h, alpha_deg, kT, m
    p.variant, p.thermostat, p.walls_z = variant, thermostat, walls_z
    p.gravity[:] = list(gravity)
    p.seed, p.box_id, p.flags = seed, box_id, flags
    p.capacity, p.graph_steps = capacity, graph_steps
    p.tile_particles, p.threads_per_cell, p.obs_ring = tile_particles, threads_per_cell, obs_ring
    p.reserved = 0
    p.wall_u[:] = list(wall_u)
    return p


def torch_allocator():
    """An mpc_allocator backed by PyTorch's caching allocator on the current device."""
    import torch

    device = torch.cuda.current_device()

    @_ALLOC_FN
    def _alloc(ctx, nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:  # out of memory -> NULL, reported as MPC_ENOMEM
            return None

    @_RELEASE_FN
    def _release(ctx, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    a = mpc_allocator()
    a.ctx = None
    a.alloc = _alloc
    a.release = _release
    return a


# --- C-ABI functions, same names -------------------------------------------------------

def mpc_version() -> str:
    return lib().mpc_version().decode()


def mpc_last_error(handle=None) -> str:
    s = lib().mpc_last_error(handle)
    return s.decode() if s else ""


def mpc_create(params: mpc_params, stream=None, allocator: mpc_allocator | None = None):
    h = ctypes.c_void_p()
    st = lib().mpc_create(ctypes.byref(params), ctypes.c_void_p(stream or 0),
                          ctypes.byref(allocator) if allocator is not None else None,
                          ctypes.byref(h))
    _check(st)
    return h


def mpc_destroy(handle) -> None:
    _check(lib().mpc_destroy(handle), handle)


def mpc_step(handle, nsteps: int) -> None:
    _check(lib().mpc_step(handle, int(nsteps)), handle)


def mpc_synchronize(handle) -> None:
    _check(lib().mpc_synchronize(handle), handle)


def _addr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def mpc_get_state(handle, X, V, ids=None, cell=None, device_ptrs=False) -> int:
    step = ctypes.c_int64()
    _check(lib().mpc_get_state(handle, _addr(X), _addr(V), _addr(ids), _addr(cell),
                               ctypes.byref(step), int(bool(device_ptrs))), handle)
    return step.value


def mpc_set_state(handle, X, V, ids, step: int, device_ptrs=False) -> None:
    _check(lib().mpc_set_state(handle, _addr(X), _addr(V), _addr(ids), int(step),
                               int(bool(device_ptrs))), handle)


def mpc_get_cell_counts(handle, counts, device_ptrs=False) -> None:
    _check(lib().mpc_get_cell_counts(handle, _addr(counts), int(bool(device_ptrs))), handle)


def mpc_observables(handle) -> mpc_obs:
    o = mpc_obs()
    _check(lib().mpc_observables(handle, ctypes.byref(o)), handle)
    return o


def mpc_observable_series(handle, rows: np.ndarray) -> int:
    n = ctypes.c_int64()
    _check(lib().mpc_observable_series(handle, rows.ctypes.data, rows.shape[0], ctypes.byref(n)),
           handle)
    return n.value


def mpc_velocity_profile(handle, out: np.ndarray) -> None:
    """out: float64 (nbins, 4) host array: per z slab count, sum vx, sum vy, sum vz"""
    assert out.dtype == np.float64 and out.ndim == 2 and out.shape[1] == 4 and out.flags.c_contiguous
    _check(lib().mpc_velocity_profile(handle, out.shape[0], out.ctypes.data), handle)


def mpc_get_info(handle) -> mpc_info:
    i = mpc_info()
    _check(lib().mpc_get_info(handle, ctypes.byref(i)), handle)
    return i


def mpc_set_profiling(handle, enable: bool) -> None:
    _check(lib().mpc_set_profiling(handle, int(bool(enable))), handle)


def mpc_profile_step_kernel(handle):
    ms = ctypes.c_double()
    n = ctypes.c_int32()
    _check(lib().mpc_profile_step_kernel(handle, ctypes.byref(ms), ctypes.byref(n)), handle)
    return ms.value, n.value


def mpc_sort_by_cell_noalloc(L, n, X, V, ids, X_out, V_out, ids_out, stream=None) -> None:
    """Sort n particles (device arrays) by unshifted cell without allocating device
    memory; see include/mpc.h for who needs this and its limits."""
    if isinstance(L, int):
        L = (L, L, L)
    Lc = (ctypes.c_int32 * 3)(*L)
    _check(lib().mpc_sort_by_cell_noalloc(Lc, int(n), _addr(X), _addr(V), _addr(ids), _addr(X_out),
                                          _addr(V_out), _addr(ids_out), ctypes.c_void_p(stream or 0)))


def mpc_checkpoint_write(handle, prefix: str) -> None:
    _check(lib().mpc_checkpoint_write(handle, os.fsencode(prefix)), handle)


def mpc_checkpoint_read(prefix: str, stream=None, allocator: mpc_allocator | None = None):
    h = ctypes.c_void_p()
    _check(lib().mpc_checkpoint_read(os.fsencode(prefix), ctypes.c_void_p(stream or 0),
                                     ctypes.byref(allocator) if allocator is not None else None,
                                     ctypes.byref(h)))
    return h


def mpc_set_step_limit(handle, limit: int) -> None:
    _check(lib().mpc_set_step_limit(handle, int(limit)), handle)


def mpc_footprint(params: mpc_params):
    """(steady, peak) device bytes of a box with these parameters."""
    s, p = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().mpc_footprint(ctypes.byref(params), ctypes.byref(s), ctypes.byref(p)))
    return s.value, p.value


def mpc_autotune(params: mpc_params, stream=None, max_smem_bytes=0):
    """(tile_particles, threads_per_cell, ns per particle-step) picked by timing."""
    t, c, ns = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(lib().mpc_autotune(ctypes.byref(params), ctypes.c_void_p(stream or 0),
                              int(max_smem_bytes), ctypes.byref(t), ctypes.byref(c),
                              ctypes.byref(ns)))
    return t.value, c.value, ns.value


def mpc_batch_create(config: mpc_batch_config | None = None, stream=None):
    b = ctypes.c_void_p()
    _check_batch(lib().mpc_batch_create(ctypes.byref(config) if config is not None else None,
                                        ctypes.c_void_p(stream or 0), ctypes.byref(b)))
    return b


def mpc_batch_destroy(batch) -> None:
    _check_batch(lib().mpc_batch_destroy(batch), batch)


def mpc_batch_add(batch, params: mpc_params):
    h = ctypes.c_void_p()
    _check_batch(lib().mpc_batch_add(batch, ctypes.byref(params), ctypes.byref(h)), batch)
    return h


def mpc_batch_remove(batch, handle) -> None:
    _check_batch(lib().mpc_batch_remove(batch, handle), batch)


def mpc_batch_step(batch, nsteps: int) -> None:
    _check_batch(lib().mpc_batch_step(batch, int(nsteps)), batch)


def mpc_batch_synchronize(batch) -> None:
    _check_batch(lib().mpc_batch_synchronize(batch), batch)


def mpc_batch_get_info(batch) -> mpc_batch_info:
    i = mpc_batch_info()
    _check_batch(lib().mpc_batch_get_info(batch, ctypes.byref(i)), batch)
    return i


def mpc_batch_last_error(batch=None) -> str:
    s = lib().mpc_batch_last_error(batch)
    return s.decode() if s else ""


def mpc_server_create(config: mpc_server_config, stream=None):
    srv = ctypes.c_void_p()
    _check_server(lib().mpc_server_create(ctypes.byref(config), ctypes.c_void_p(stream or 0),
                                          ctypes.byref(srv)))
    return srv


def mpc_server_destroy(server) -> None:
    _check_server(lib().mpc_server_destroy(server), server)


def mpc_server_submit(server, job: mpc_job) -> int:
    jid = ctypes.c_int64()
    _check_server(lib().mpc_server_submit(server, ctypes.byref(job), ctypes.byref(jid)), server)
    return jid.value


def mpc_server_run(server, timeout_s: float = 0.0) -> None:
    _check_server(lib().mpc_server_run(server, float(timeout_s)), server)


def mpc_server_job(server, job_id: int) -> mpc_job_result:
    r = mpc_job_result()
    _check_server(lib().mpc_server_job(server, int(job_id), ctypes.byref(r)), server)
    return r


def mpc_server_get_stats(server) -> mpc_server_stats:
    st = mpc_server_stats()
    _check_server(lib().mpc_server_get_stats(server, ctypes.byref(st)), server)
    return st


def mpc_server_job_series(server, job_id: int, rows: np.ndarray) -> None:
    _check_server(lib().mpc_server_job_series(server, int(job_id), rows.ctypes.data, rows.shape[0]),
                  server)


def mpc_server_job_state(server, job_id: int, X, V, ids) -> None:
    _check_server(lib().mpc_server_job_state(server, int(job_id), _addr(X), _addr(V), _addr(ids)),
                  server)


def mpc_server_last_error(server=None) -> str:
    s = lib().mpc_server_last_error(server)
    return s.decode() if s else ""


# --- convenience wrapper -----------------------------------------------------------------

class Box:
    """State access for one MPC box (a standalone Simulation or a batch member)."""

    def __init__(self, handle, params: mpc_params):
        self.handle = handle
        self.params = params
        self.info = mpc_get_info(handle)
        self.N = self.info.n_particles

    def step(self, n: int = 1):
        mpc_step(self.handle, n)

    def synchronize(self):
        mpc_synchronize(self.handle)

    def set_step_limit(self, limit: int):
        mpc_set_step_limit(self.handle, limit)

    def checkpoint(self, prefix: str):
        """Write <prefix>.txt / .particles / .cells (Sec. III.G.2 checkpoint layout)."""
        mpc_checkpoint_write(self.handle, prefix)

    def get_state(self, cells=False):
        """(X (3,N) uint32, V (3,N) float32, ids (N,), step[, cell]) on the host, sorted by
        unshifted cell."""
        N = self.N
        X = np.empty((3, N), dtype=np.uint32)
        V = np.empty((3, N), dtype=np.float32)
        ids = np.empty(N, dtype=np.uint32)
        cell = np.empty(N, dtype=np.uint32) if cells else None
        step = mpc_get_state(self.handle, X, V, ids, cell)
        return (X, V, ids, step, cell) if cells else (X, V, ids, step)

    def set_state(self, X, V, ids, step):
        X = np.ascontiguousarray(X, dtype=np.uint32)
        V = np.ascontiguousarray(V, dtype=np.float32)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        mpc_set_state(self.handle, X, V, ids, step)

    def cell_counts(self):
        c = np.empty(self.info.n_cells, dtype=np.uint32)
        mpc_get_cell_counts(self.handle, c)
        return c

    def observables(self) -> dict:
        o = mpc_observables(self.handle)
        return {"momentum": np.array(o.momentum[:]), "ekin": o.ekin,
                "temperature": o.temperature, "stress_kin": np.array(o.stress_kin[:]),
                "stress_col": np.array(o.stress_col[:]), "n_particles": o.n_particles,
                "step": o.step, "has_stress": bool(o.has_stress)}

    def observable_series(self, count: int) -> np.ndarray:
        rows = np.zeros((count, 16), dtype=np.float64)
        n = mpc_observable_series(self.handle, rows)
        return rows[:n]

    def velocity_profile(self, nbins: int):
        """(counts (nbins,), summed velocities (nbins, 3)) per z slab of the box"""
        out = np.zeros((nbins, 4), dtype=np.float64)
        mpc_velocity_profile(self.handle, out)
        return out[:, 0], out[:, 1:]


class Simulation(Box):
    """One MPC box on the current CUDA device."""

    def __init__(self, stream=None, use_torch_allocator=True, **kw):
        import torch

        params = make_params(**kw)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self._alloc = torch_allocator() if use_torch_allocator else None
        super().__init__(mpc_create(params, stream, self._alloc), params)

    @classmethod
    def from_checkpoint(cls, prefix: str, stream=None, use_torch_allocator=True):
        """A box restored from a checkpoint written by `checkpoint`."""
        import torch

        self = cls.__new__(cls)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self._alloc = torch_allocator() if use_torch_allocator else None
        h = mpc_checkpoint_read(prefix, stream, self._alloc)
        Box.__init__(self, h, None)
        return self

    def close(self):
        if self.handle is not None:
            mpc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent boxes advanced together: small boxes packed by variant into
    persistent launches, large ones in their own launches, one CUDA graph per chunk."""

    def __init__(self, arena_bytes=0, graph_steps=0, deterministic=False, autotune=False,
                 max_boxes=0, stream=None, pack_all=False):
        import torch

        cfg = mpc_batch_config()
        cfg.arena_bytes = int(arena_bytes)
        cfg.graph_steps = int(graph_steps)
        cfg.flags = (MPC_BATCH_DETERMINISTIC if deterministic else 0) | \
            (MPC_BATCH_AUTOTUNE if autotune else 0) | (MPC_BATCH_PACK_ALL if pack_all else 0)
        cfg.max_boxes = int(max_boxes)
        cfg.reserved = 0
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self.handle = mpc_batch_create(cfg, stream)
        self.boxes: list[Box] = []

    def add(self, **kw) -> Box:
        params = make_params(**kw)
        box = Box(mpc_batch_add(self.handle, params), params)
        self.boxes.append(box)
        return box

    def remove(self, box: Box) -> None:
        mpc_batch_remove(self.handle, box.handle)
        self.boxes.remove(box)
        box.handle = None

    def step(self, n: int = 1) -> None:
        mpc_batch_step(self.handle, n)

    def synchronize(self) -> None:
        mpc_batch_synchronize(self.handle)

    def info(self) -> mpc_batch_info:
        return mpc_batch_get_info(self.handle)

    def close(self):
        if self.handle is not None:
            mpc_batch_destroy(self.handle)
            self.handle = None
            for b in self.boxes:
                b.handle = None
            self.boxes = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching request loop: jobs (box parameters, step count, arrival time)
    are admitted by HBM budget, advanced together while resident, and retired with a
    Green-Kubo viscosity."""

    def __init__(self, hbm_budget_bytes, chunk_steps=0, max_active=0, deterministic=False,
                 sequential=False, share_all=False, first_come=False, fill_kparticles=0,
                 aged=False, backfill=False, priority_head=False, stream=None):
        import torch

        cfg = mpc_server_config()
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.chunk_steps = int(chunk_steps)
        cfg.max_active = int(max_active)
        cfg.flags = (MPC_SERVER_DETERMINISTIC if deterministic else 0) | \
            (MPC_SERVER_SEQUENTIAL if sequential else 0) | \
            (MPC_SERVER_SHARE_ALL if share_all else 0) | \
            (MPC_SERVER_FIRST_COME if first_come else 0) | \
            (MPC_SERVER_AGED if aged else 0) | (MPC_SERVER_BACKFILL if backfill else 0) | \
            (MPC_SERVER_PRIORITY_HEAD if priority_head else 0)
        cfg.fill_kparticles = int(fill_kparticles)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.handle = mpc_server_create(cfg, stream)
        self.steps = []
        self.N = []

    def submit(self, steps, arrival_s=0.0, keep_series=False, keep_state=False, **kw) -> int:
        job = mpc_job()
        job.params = make_params(**kw)
        job.steps = int(steps)
        job.arrival_s = float(arrival_s)
        job.keep = (MPC_JOB_KEEP_SERIES if keep_series else 0) | \
            (MPC_JOB_KEEP_STATE if keep_state else 0)
        job.reserved = 0
        jid = mpc_server_submit(self.handle, job)
        self.steps.append(int(steps))
        L = job.params.L
        self.N.append(int(round(L[0] * L[1] * L[2] * job.params.n_c)))
        return jid

    def run(self, timeout_s: float = 0.0) -> None:
        mpc_server_run(self.handle, timeout_s)

    def job(self, job_id: int) -> dict:
        r = mpc_server_job(self.handle, job_id)
        return {"status": r.status, "error": r.error, "arrival_s": r.arrival_s,
                "admit_s": r.admit_s, "finish_s": r.finish_s, "steps": r.steps,
                "n_particles": r.n_particles, "eta_gk": r.eta_gk, "temperature": r.temperature,
                "latency_s": r.finish_s - r.arrival_s}

    def stats(self) -> dict:
        st = mpc_server_get_stats(self.handle)
        return {k: getattr(st, k) for k, _ in mpc_server_stats._fields_ if k != "reserved"}

    def series(self, job_id: int) -> np.ndarray:
        rows = np.zeros((self.steps[job_id], 16), dtype=np.float64)
        mpc_server_job_series(self.handle, job_id, rows)
        return rows

    def state(self, job_id: int):
        N = self.N[job_id]
        X = np.empty((3, N), dtype=np.uint32)
        V = np.empty((3, N), dtype=np.float32)
        ids = np.empty(N, dtype=np.uint32)
        mpc_server_job_state(self.handle, job_id, X, V, ids)
        return X, V, ids

    def close(self):
        if self.handle is not None:
            mpc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
