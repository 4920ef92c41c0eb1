"""Helpers for GPU-vs-oracle parity tests (test infrastructure).

Velocity error of a particle: |v_gpu - v_ref| / max(|v_ref|, sqrt(kT/m)), bar 1e-5 for
every particle of every cell, except:
  * cells the oracle flags FLAG_ILL_CONDITIONED (angular-momentum variants, n >= 3 and
    cond(J) > 10, or members within 0.05 a of their centre of mass; about 0.5 % of the
    cells at N_c = 10): a float32 solve is good there
    only to the first-order sensitivity sens_i the oracle exports (pinned against
    float32 evaluations by tests/test_oracle_sensitivity.py: errors up to 0.44 u sens_i;
    the kernel's measured up to 0.7 u sens_i), so their members' bar is
    max(1e-5, 4 u sens_i / scale_i), u = 2^-24;
  * cells with a flag in `strict_flags` (a float32 sampler decision within 1e-5 of its
    threshold, or a degenerate inertia tensor), which are not compared.
check_step reports the share of ill-conditioned cells per step.  Integer results
(positions, collision cells, per-cell counts) must agree bit-exactly.
"""
import json
import os

import numpy as np

import oracle

VEL_TOL = 1e-5
ULP32 = 2.0**-24
SENS_FACTOR = 4  # bar in an ill-conditioned cell: max(1e-5, SENS_FACTOR u sens_i / scale_i)


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


def cell_condition(p_oracle, X_streamed, step, cell, ncells):
    """cond(J) per collision cell (inf for cells of fewer than three members or a
    degenerate J): J = tr(M) 1 - M, M = sum r r^T about the cell's centre of mass, from the
    oracle's collision positions"""
    F = oracle.fixed_bits(p_oracle)
    S = oracle.shift(p_oracle, step).astype(np.int64)
    rho = (((X_streamed.astype(np.int64) + S[:, None]) & ((1 << F) - 1)) / 2.0**F - 0.5).T
    n = np.bincount(cell, minlength=ncells).astype(np.float64)
    s1 = np.zeros((ncells, 3))
    s2 = np.zeros((ncells, 3, 3))
    np.add.at(s1, cell, rho)
    np.add.at(s2, cell, rho[:, :, None] * rho[:, None, :])
    nn = np.maximum(n, 1.0)[:, None, None]
    M = s2 - s1[:, :, None] * s1[:, None, :] / nn
    J = np.trace(M, axis1=1, axis2=2)[:, None, None] * np.eye(3) - M
    ev = np.linalg.eigvalsh(J)
    with np.errstate(divide="ignore", invalid="ignore"):
        cond = np.where(ev[:, 0] > 0, ev[:, 2] / ev[:, 0], np.inf)
    cond[n < 3] = np.inf
    return cond, n


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
    illc = (ref["flags"][ref["cell"]] & oracle.FLAG_ILL_CONDITIONED) != 0
    bar = np.where(illc, np.maximum(VEL_TOL, SENS_FACTOR * ULP32 * ref["sens"] / scale), VEL_TOL)
    ratio = err / bar
    with np.errstate(divide="ignore", invalid="ignore"):
        k_emp = np.where(ref["sens"] > 0, err * scale / (ULP32 * ref["sens"]), 0.0)
    stats["k_emp"] = float(k_emp.max())  # largest error in units of u sens_i
    stats["k_emp_ill"] = float(k_emp[illc].max()) if illc.any() else 0.0
    occupied = max(1, int((ref["counts"] > 0).sum()))
    stats["ill_cells"] = float(((ref["flags"] & oracle.FLAG_ILL_CONDITIONED) != 0).sum() / occupied)
    stats["ill_particles"] = float(illc.mean())
    strict = ~flagged & ~illc
    stats["over_tol_strict"] = float((err[strict] > VEL_TOL).mean()) if strict.any() else 0.0
    stats["max_err_strict"] = float(err[strict].max()) if strict.any() else 0.0
    stats["max_err"] = float(err[~flagged].max()) if (~flagged).any() else 0.0
    stats["max_ratio"] = float(ratio[~flagged].max()) if (~flagged).any() else 0.0
    stats["widened"] = float((bar[~flagged] > VEL_TOL).mean()) if (~flagged).any() else 0.0
    stats["over_tol"] = float((err[~flagged] > VEL_TOL).mean()) if (~flagged).any() else 0.0
    stats["flagged"] = int(flagged.sum())
    stats["max_err_flagged"] = float(err[flagged].max()) if flagged.any() else 0.0
    log_path = os.environ.get("MPC_PARITY_LOG")
    if log_path and ref["sens"].max() > 0:  # angular-momentum variants: conditioning report
        cond, n = cell_condition(p_oracle, ref["X"], step, ref["cell"], len(ref["flags"]))
        pc = cond[ref["cell"]]
        over = err > VEL_TOL
        stats["cond_over_tol_min"] = float(pc[over].min()) if over.any() else None
        stats["n_over_tol"] = int(over.sum())
        stats["n_over_tol_pairs"] = int((over & (n[ref["cell"]] == 2)).sum())
        occupied = n > 0
        for t in (10, 30, 100, 300, 1000):
            stats[f"cells_cond_gt_{t}"] = float(((cond > t) & (n >= 3)).sum() / occupied.sum())
        stats["cells_pairs"] = float((n == 2).sum() / occupied.sum())
        for t in (10, 30, 100):
            ok = pc <= t
            stats[f"max_err_cond_le_{t}"] = float(err[ok].max()) if ok.any() else 0.0
    if log_path:  # one line per checked step, for reports
        with open(log_path, "a") as f:
            f.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", ""), "step": step,
                                **{k: v for k, v in stats.items()}}) + "\n")
    assert stats["over_tol_strict"] == 0.0, (f"step {step}: velocity error "
                                             f"{stats['max_err_strict']:.3g} above 1e-5 in a cell "
                                             f"that is not ill-conditioned")
    assert stats["max_ratio"] <= 1.0, (f"step {step}: velocity error {stats['max_err']:.3g} "
                                       f"exceeds its bar (ratio {stats['max_ratio']:.3g})")
    stats["ref"] = ref
    return stats


def check_subset(ref, X1, V1, keep, kT=1.0, m=1.0, strict_flags=oracle.FLAG_DEGENERATE, what=""):
    """Compare the GPU result (X1, V1: the same particles as the oracle's `ref`, in its
    order) on the particles selected by `keep` -- the members of cells whose every member
    took part in the oracle step -- with the bar of check_step.  Returns the largest
    velocity error outside ill-conditioned cells."""
    np.testing.assert_array_equal(X1[:, keep], ref["X"][:, keep], err_msg=f"{what}: positions differ")
    vref = ref["V"][:, keep]
    scale = np.maximum(np.linalg.norm(vref, axis=0), np.sqrt(kT / m))
    err = np.linalg.norm(V1[:, keep].astype(np.float64) - vref, axis=0) / scale
    cflags = ref["flags"][ref["cell"][keep]]
    skip = (cflags & strict_flags) != 0
    illc = (cflags & oracle.FLAG_ILL_CONDITIONED) != 0
    bar = np.where(illc, np.maximum(VEL_TOL, SENS_FACTOR * ULP32 * ref["sens"][keep] / scale), VEL_TOL)
    bad = (err > bar) & ~skip
    assert not bad.any(), (f"{what}: {bad.sum()} velocities above their bar, worst "
                           f"{float(err[bad].max()):.3g} (ill-conditioned: {int((bad & illc).sum())})")
    strict = ~skip & ~illc
    return float(err[strict].max()) if strict.any() else 0.0
