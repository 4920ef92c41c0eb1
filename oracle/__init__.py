"""Oracle for one MPC step (arXiv 2406.15236, Sec. II) -- TEST INFRASTRUCTURE ONLY.

A plain single-threaded FP64 C implementation (``mpc_oracle.c``) wrapped with ctypes.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package; the product path (``paper_2406_15236_gb300``) never does.
It shares no code with the CUDA implementation.

Every function cites the passage of the paper it follows in ``mpc_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpc_oracle.c")
_HDR = os.path.join(_HERE, "mpc_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SRD, AT_A, SRD_A = 0, 1, 2
FLAG_MBS_NEAR_TIE, FLAG_POISSON_NEAR_TIE, FLAG_ILL_CONDITIONED, FLAG_DEGENERATE = 1, 2, 4, 8
OBS_NAMES = ["px", "py", "pz", "ekin", "temperature", "skin_xy", "skin_yz", "skin_zx",
             "scol_xy", "scol_yx", "scol_yz", "scol_zy", "scol_zx", "scol_xz"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE float: no contraction, no fast math)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fexcess-precision=standard", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True, capture_output=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32 * 3), ("n_c", ctypes.c_double), ("h", ctypes.c_double),
                ("alpha_deg", ctypes.c_double), ("kT", ctypes.c_double), ("m", ctypes.c_double),
                ("variant", ctypes.c_int32), ("thermostat", ctypes.c_int32),
                ("walls_z", ctypes.c_int32), ("g", ctypes.c_double * 3),
                ("seed", ctypes.c_uint64), ("box", ctypes.c_uint32),
                ("wall_u", ctypes.c_double * 2)]


NO_SLIP, SLIP = 1, 2


def params(L=(16, 16, 16), n_c=10.0, h=0.1, alpha_deg=130.0, kT=1.0, m=1.0, variant=SRD,
           thermostat=0, walls_z=0, g=(0.0, 0.0, 0.0), seed=1, box=0,
           wall_u=(0.0, 0.0)) -> Params:
    if isinstance(L, int):
        L = (L, L, L)
    p = Params()
    p.L[:] = list(L)
    p.n_c, p.h, p.alpha_deg, p.kT, p.m = n_c, h, alpha_deg, kT, m
    p.variant, p.thermostat, p.walls_z = variant, thermostat, walls_z
    p.g[:] = list(g)
    p.seed, p.box = seed, box
    p.wall_u[:] = list(wall_u)
    return p


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            u32, f64, i64 = ctypes.c_uint32, ctypes.c_double, ctypes.c_int64
            L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
            L.orc_fixed_bits.argtypes = [P(Params)]
            L.orc_fixed_bits.restype = ctypes.c_int
            L.orc_num_particles.argtypes = [P(Params)]
            L.orc_num_particles.restype = i64
            L.orc_num_cells.argtypes = [P(Params)]
            L.orc_num_cells.restype = i64
            L.orc_shift.argtypes = [P(Params), i64, P(u32)]
            L.orc_init.argtypes = [P(Params), i64, P(u32), P(f64), P(u32)]
            L.orc_step.argtypes = [P(Params), i64, P(u32), P(f64), P(u32), i64, P(u32), P(u32),
                                   P(f64), P(f64), P(ctypes.c_uint8), P(f64)]
            L.orc_step.restype = ctypes.c_int
            L.orc_cell_of.argtypes = [P(Params), P(u32), P(u32), P(u32), P(f64)]
            L.orc_srd_axis.argtypes = [P(Params), i64, u32, P(f64)]
            L.orc_rotate.argtypes = [P(f64), f64, P(f64), P(f64)]
            L.orc_stream_one.argtypes = [P(Params), P(u32), P(f64)]
            L.orc_min_eigenvalue_sym3.argtypes = [P(f64)]
            L.orc_min_eigenvalue_sym3.restype = f64
            L.orc_max_eigenvalue_sym3.argtypes = [P(f64)]
            L.orc_max_eigenvalue_sym3.restype = f64
            L.orc_cell_omega.argtypes = [i64, P(f64), P(f64), P(f64), P(f64), P(f64)]
            L.orc_cell_omega.restype = ctypes.c_int
            L.orc_phantoms.argtypes = [P(Params), i64, u32, f64, ctypes.c_int, P(f64), P(f64),
                                       P(f64)]
            L.orc_phantoms.restype = ctypes.c_int
            L.orc_phantom_particles.argtypes = [P(Params), i64, u32, u32, ctypes.c_int,
                                                ctypes.c_int32, P(f64), P(f64), P(f64)]
            L.orc_sample_normal.argtypes = [ctypes.c_uint64, i64, P(f64)]
            L.orc_sample_gamma.argtypes = [ctypes.c_uint64, f64, i64, P(f64)]
            L.orc_sample_poisson.argtypes = [ctypes.c_uint64, f64, i64, P(ctypes.c_int32)]
            _lib = L
    return _lib


def philox(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def fixed_bits(p: Params) -> int:
    return lib().orc_fixed_bits(ctypes.byref(p))


def num_particles(p: Params) -> int:
    return lib().orc_num_particles(ctypes.byref(p))


def num_cells(p: Params) -> int:
    return lib().orc_num_cells(ctypes.byref(p))


def shift(p: Params, step: int) -> np.ndarray:
    S = np.zeros(3, dtype=np.uint32)
    lib().orc_shift(ctypes.byref(p), step, _ptr(S, ctypes.c_uint32))
    return S


def init(p: Params):
    """Initial state: uniform fixed-point positions, Maxwell-Boltzmann velocities with the
    net momentum removed, consecutive ids.  Returns X (3,N) uint32, V (3,N) f64, id (N,)."""
    N = num_particles(p)
    X = np.zeros((3, N), dtype=np.uint32)
    V = np.zeros((3, N), dtype=np.float64)
    ids = np.zeros(N, dtype=np.uint32)
    lib().orc_init(ctypes.byref(p), N, _ptr(X, ctypes.c_uint32), _ptr(V, ctypes.c_double),
                   _ptr(ids, ctypes.c_uint32))
    return X, V, ids


def step(p: Params, X, V, ids, step_index: int, cells=False, counts=False, vpre=False,
         obs=False, flags=False, sens=False):
    """One MPC step in place on copies of (X, V); returns a dict with the new state and
    the requested diagnostics."""
    X = np.ascontiguousarray(X, dtype=np.uint32).copy()
    V = np.ascontiguousarray(V, dtype=np.float64).copy()
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    N = X.shape[1]
    C = num_cells(p)
    out = {"X": X, "V": V}
    cell = np.zeros(N, dtype=np.uint32) if cells else None
    cnt = np.zeros(C, dtype=np.uint32) if counts else None
    vp = np.zeros((3, N), dtype=np.float64) if vpre else None
    ob = np.zeros(16, dtype=np.float64) if obs else None
    fl = np.zeros(C, dtype=np.uint8) if flags else None
    se = np.zeros(N, dtype=np.float64) if sens else None
    rc = lib().orc_step(ctypes.byref(p), N, _ptr(X, ctypes.c_uint32), _ptr(V, ctypes.c_double),
                        _ptr(ids, ctypes.c_uint32), step_index, _ptr(cell, ctypes.c_uint32),
                        _ptr(cnt, ctypes.c_uint32), _ptr(vp, ctypes.c_double),
                        _ptr(ob, ctypes.c_double), _ptr(fl, ctypes.c_uint8),
                        _ptr(se, ctypes.c_double))
    if rc != 0:
        raise MemoryError("oracle step failed")
    if cells:
        out["cell"] = cell
    if counts:
        out["counts"] = cnt
    if vpre:
        out["vpre"] = vp
    if obs:
        out["obs"] = dict(zip(OBS_NAMES, ob[:len(OBS_NAMES)]))
    if flags:
        out["flags"] = fl
    if sens:
        # per particle: |r_ic| sum_j |r_jc||w_j| / lambda_min(J) for the angular-momentum
        # variants (0 for SRD): how strongly float32 rounding of the cell sums is
        # amplified into this particle's new velocity
        out["sens"] = se
    return out


def run(p: Params, nsteps: int, state=None, first_step: int = 0, obs=False):
    """Advance `nsteps` steps from `state` (or from init); returns (X, V, ids, obs_list)."""
    X, V, ids = state if state is not None else init(p)
    obs_list = []
    for s in range(first_step, first_step + nsteps):
        r = step(p, X, V, ids, s, obs=obs)
        X, V = r["X"], r["V"]
        if obs:
            obs_list.append(r["obs"])
    return X, V, ids, obs_list


def cell_of(p: Params, x, S):
    xa = np.asarray(x, dtype=np.uint32).copy()
    Sa = np.asarray(S, dtype=np.uint32).copy()
    c = np.zeros(1, dtype=np.uint32)
    rho = np.zeros(3, dtype=np.float64)
    lib().orc_cell_of(ctypes.byref(p), _ptr(xa, ctypes.c_uint32), _ptr(Sa, ctypes.c_uint32),
                      _ptr(c, ctypes.c_uint32), _ptr(rho, ctypes.c_double))
    return int(c[0]), rho


def srd_axis(p: Params, step_index: int, cell: int) -> np.ndarray:
    a = np.zeros(3, dtype=np.float64)
    lib().orc_srd_axis(ctypes.byref(p), step_index, cell, _ptr(a, ctypes.c_double))
    return a


def rotate(axis, alpha_rad: float, v) -> np.ndarray:
    a = np.ascontiguousarray(axis, dtype=np.float64)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(3, dtype=np.float64)
    lib().orc_rotate(_ptr(a, ctypes.c_double), alpha_rad, _ptr(vv, ctypes.c_double),
                     _ptr(out, ctypes.c_double))
    return out


def stream_one(p: Params, x, v):
    xa = np.asarray(x, dtype=np.uint32).copy()
    va = np.asarray(v, dtype=np.float64).copy()
    lib().orc_stream_one(ctypes.byref(p), _ptr(xa, ctypes.c_uint32), _ptr(va, ctypes.c_double))
    return xa, va


def min_eigenvalue_sym3(A) -> float:
    a = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
    return lib().orc_min_eigenvalue_sym3(_ptr(a, ctypes.c_double))


def cell_omega(rho, w):
    """The angular-momentum restoring rotation of one cell (Eqs. 3-4): rho (n, 3) positions
    relative to the cell centre, w (n, 3) the velocities whose angular momentum about the
    centre of mass is restored.  Returns (omega, rcm, sens, flags)."""
    r = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1, 3)
    ww = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 3)
    n = r.shape[0]
    om, rc = np.zeros(3), np.zeros(3)
    se = np.zeros(max(n, 1))
    fl = lib().orc_cell_omega(n, _ptr(r, ctypes.c_double), _ptr(ww, ctypes.c_double),
                              _ptr(om, ctypes.c_double), _ptr(rc, ctypes.c_double),
                              _ptr(se, ctypes.c_double))
    return om, rc, se[:n], fl


def phantoms(p: Params, step_index: int, cell: int, phi: float, wall: int):
    """Aggregate phantom particles of one wall-cut cell: (count, momentum[3], internal
    kinetic energy, flags)."""
    nph = np.zeros(1)
    P = np.zeros(3)
    K = np.zeros(1)
    fl = lib().orc_phantoms(ctypes.byref(p), step_index, cell, phi, wall, _ptr(nph, ctypes.c_double),
                            _ptr(P, ctypes.c_double), _ptr(K, ctypes.c_double))
    return int(nph[0]), P, float(K[0]), fl


def phantom_particles(p: Params, step_index: int, cell: int, Sz: int, wall: int, k: int):
    """k phantom particles of a wall-cut cell, one by one: positions relative to the cell
    centre (k, 3), velocities (k, 3), random velocities (k, 3)"""
    rho, v, vr = (np.zeros((max(k, 1), 3)) for _ in range(3))
    lib().orc_phantom_particles(ctypes.byref(p), step_index, cell, Sz, wall, k,
                                _ptr(rho, ctypes.c_double), _ptr(v, ctypes.c_double),
                                _ptr(vr, ctypes.c_double))
    return rho[:k], v[:k], vr[:k]


def max_eigenvalue_sym3(A) -> float:
    a = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
    return lib().orc_max_eigenvalue_sym3(_ptr(a, ctypes.c_double))


COND_FLOAT32 = 10.0  # cond(J) above which a cell is flagged FLAG_ILL_CONDITIONED
TIGHT_RMS = 0.05  # rms radius below which a cell of n >= 2 is flagged FLAG_ILL_CONDITIONED


def sample_normal(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    lib().orc_sample_normal(seed, n, _ptr(out, ctypes.c_double))
    return out


def sample_gamma(seed: int, shape: float, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    lib().orc_sample_gamma(seed, shape, n, _ptr(out, ctypes.c_double))
    return out


def sample_poisson(seed: int, lam: float, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.int32)
    lib().orc_sample_poisson(seed, lam, n, _ptr(out, ctypes.c_int32))
    return out
