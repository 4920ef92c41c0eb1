"""Helpers for GPU-vs-oracle parity tests (test infrastructure).

Velocity error of a particle: |v_gpu - v_ref| / max(|v_ref|, sqrt(kT/m)), bar 1e-5.
For the angular-momentum variants the float32 kernel solves J omega = L per cell, and
float32 rounding (relative u = 2^-24 per operation) of the products and of the
centre-of-mass positions reaches the velocity amplified by the first-order factor sens_i
the oracle exports (1/lambda_min(J) times the perturbations of L and J, times |r_i|,
plus the rounding of r_i times |omega|); the bar of a particle is
max(1e-5, 16 u sens_i / scale_i).  It widens only for near-collinear cells and
near-coincident pairs of 2-5 particles.
Integer results (positions, collision cells, per-cell counts) must agree bit-exactly.
"""
import numpy as np

import oracle

VEL_TOL = 1e-5
ULP32 = 2.0**-24


def by_id(X, V, ids, cell=None):
    o = np.argsort(ids, kind="stable")
    out = (X[:, o], V[:, o], ids[o])
    return out + ((cell[o],) if cell is not None else ())


def oracle_params(**kw):
    """oracle.params from mpc-style keyword arguments"""
    m = dict(kw)
    variant = m.pop("variant", 0)
    g = m.pop("gravity", (0.0, 0.0, 0.0))
    for k in ("flags", "capacity", "graph_steps", "box_id", "tile_particles", "threads_per_cell",
              "obs_ring"):
        m.pop(k, None)
    return oracle.params(variant=variant, g=g, **m)


def check_step(p_oracle, pre, post, step, kT=1.0, m=1.0, post_cells=None, gpu_counts=None,
               strict_flags=0xFF):
    """Compare one GPU step (pre -> post, host arrays) with the oracle from `pre`.
    Returns a dict of mismatch statistics; raises AssertionError on a failure."""
    X0, V0, id0 = by_id(*pre)
    X1, V1, id1 = by_id(*post)[:3]
    assert np.array_equal(id0, id1), "particle ids changed"
    ref = oracle.step(p_oracle, X0, V0.astype(np.float64), id0, step, cells=True, counts=True,
                      flags=True, obs=True, sens=True)
    stats = {}
    pos_bad = np.any(X1 != ref["X"], axis=0)
    stats["pos_mismatch"] = float(pos_bad.mean())
    assert not pos_bad.any(), f"step {step}: {pos_bad.sum()} positions differ"
    if post_cells is not None:
        c1 = post_cells[np.argsort(post[2], kind="stable")]
        cbad = c1 != ref["cell"]
        stats["cell_mismatch"] = float(cbad.mean())
        assert not cbad.any(), f"step {step}: {cbad.sum()} collision cells differ"
    if gpu_counts is not None:
        nbad = gpu_counts != ref["counts"]
        stats["count_mismatch"] = float(nbad.mean())
        assert not nbad.any(), f"step {step}: {nbad.sum()} cell counts differ"
    vref = ref["V"]
    scale = np.maximum(np.linalg.norm(vref, axis=0), np.sqrt(kT / m))
    err = np.linalg.norm(V1.astype(np.float64) - vref, axis=0) / scale
    flagged = (ref["flags"][ref["cell"]] & strict_flags) != 0
    bar = np.maximum(VEL_TOL, 16 * ULP32 * ref["sens"] / scale)
    ratio = err / bar
    stats["max_err"] = float(err[~flagged].max()) if (~flagged).any() else 0.0
    stats["max_ratio"] = float(ratio[~flagged].max()) if (~flagged).any() else 0.0
    stats["widened"] = float((bar[~flagged] > VEL_TOL).mean()) if (~flagged).any() else 0.0
    stats["over_tol"] = float((err[~flagged] > VEL_TOL).mean()) if (~flagged).any() else 0.0
    stats["flagged"] = int(flagged.sum())
    stats["max_err_flagged"] = float(err[flagged].max()) if flagged.any() else 0.0
    assert stats["max_ratio"] <= 1.0, (f"step {step}: velocity error {stats['max_err']:.3g} "
                                       f"exceeds its bar (ratio {stats['max_ratio']:.3g})")
    stats["ref"] = ref
    return stats
