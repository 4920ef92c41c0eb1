"""Pins of the oracle's angular-momentum solve and of its float32 rounding sensitivity.

The angular-momentum-conserving collisions (Eqs. 3-4 for SRD+a; AT+a alike) add
omega x r_ic to each particle, with omega the rotation that restores the cell's angular
momentum about its centre of mass.  Its defining property: after the rotation is
removed, the particles' angular momentum about the centre of mass vanishes,
sum_j r_j x (w_j - omega x r_j) = 0 (n >= 3; for a pair, the component normal to the
pair axis).  That property, and numpy's linear solvers, pin `orc_cell_omega`.

The GPU computes the same solve in float32.  The oracle exports, per particle, a
first-order sensitivity sens_i of the new velocity to float32 rounding (relative unit
u = 2^-24) of the positions, velocities and cell sums; the GPU parity tests widen the
1e-5 velocity bar to 16 u sens_i / scale_i where that is larger.  Here float32
evaluations of the solve (two passes about the centre of mass; one pass of raw sums about
the cell centre for cells of six or more members, as the kernel takes them), over many
member orders, cells and velocity frames (at rest and drifting by 5 sigma), including
near-collinear cells and near-coincident pairs, must stay within u sens_i: the bound
holds without the factor 16, and it is not inflated (its upper tail is reached to within
a factor of ten).  A constant sensitivity in its place would not bound them.
"""
import numpy as np
import pytest

import oracle

U = 2.0**-24
F32 = np.float32


def _grid(x):
    """positions on the fixed-point grid of a 512-cell box (exact in float32)"""
    return np.round(np.asarray(x) * 2.0**22) / 2.0**22


def _adjugate_solve(J, L, n):
    """omega = J^-1 L by the adjugate (n >= 3) or the pair pseudo-inverse (n = 2), in the
    dtype of J"""
    t = J.dtype.type
    if n == 2:
        trM = (J[0, 0] + J[1, 1] + J[2, 2]) * t(0.5)  # J = tr(M) 1 - M, M = sum r r^T
        M = trM * np.eye(3, dtype=J.dtype) - J
        it = t(1) / trM
        return (L - (M @ L) * it) * it
    A = np.empty((3, 3), dtype=J.dtype)
    A[0, 0] = J[1, 1] * J[2, 2] - J[1, 2] * J[1, 2]
    A[0, 1] = J[2, 0] * J[1, 2] - J[0, 1] * J[2, 2]
    A[0, 2] = J[0, 1] * J[1, 2] - J[2, 0] * J[1, 1]
    A[1, 1] = J[0, 0] * J[2, 2] - J[2, 0] * J[2, 0]
    A[1, 2] = J[2, 0] * J[0, 1] - J[0, 0] * J[1, 2]
    A[2, 2] = J[0, 0] * J[1, 1] - J[0, 1] * J[0, 1]
    A[1, 0], A[2, 0], A[2, 1] = A[0, 1], A[0, 2], A[1, 2]
    det = J[0, 0] * A[0, 0] + J[0, 1] * A[0, 1] + J[2, 0] * A[0, 2]
    if not det > 0:
        return np.zeros(3, dtype=J.dtype)
    return (A @ L) / det


def _float32_rotation_term(rho, w, one_pass):
    """omega x r_i evaluated in float32: the sums in member order, the moments either about
    the centre of mass (two passes) or from raw sums about the cell centre (one pass)"""
    n = len(rho)
    r32, w32 = rho.astype(F32), w.astype(F32)
    rc, wm = np.zeros(3, F32), np.zeros(3, F32)
    for k in range(n):
        rc += r32[k]
        wm += w32[k]
    inv = F32(1) / F32(n)
    rc, wm = rc * inv, wm * inv
    M, L = np.zeros((3, 3), F32), np.zeros(3, F32)
    if one_pass:
        for k in range(n):
            M += np.outer(r32[k], r32[k])
            L += np.cross(r32[k], w32[k])
        M -= F32(n) * np.outer(rc, rc)
        L -= F32(n) * np.cross(rc, wm)
    else:
        for k in range(n):
            rr, ww = r32[k] - rc, w32[k] - wm
            M += np.outer(rr, rr)
            L += np.cross(rr, ww)
    J = (M[0, 0] + M[1, 1] + M[2, 2]) * np.eye(3, dtype=F32) - M
    om = _adjugate_solve(J, L, n)
    return np.cross(om, r32 - rc).astype(np.float64)


def _cells(rng):
    for n in (2, 3, 4, 5, 6, 8, 10, 15, 20, 30):
        for _ in range(24):
            yield "uniform", _grid(rng.uniform(-0.5, 0.5, (n, 3)))
    for eps in (0.1, 0.03, 0.01, 0.003, 0.001):
        for n in (3, 4, 6, 10):
            for _ in range(10):
                d = rng.normal(size=3)
                d /= np.linalg.norm(d)
                pts = rng.uniform(-0.4, 0.4, n)[:, None] * d + eps * rng.normal(size=(n, 3))
                yield "near-collinear", _grid(np.clip(pts, -0.5, 0.5 - 2.0**-22))
    for s in (0.3, 0.03, 0.003):
        for _ in range(12):
            c = rng.uniform(-0.4, 0.4, 3)
            d = rng.normal(size=3)
            d *= s / np.linalg.norm(d)
            yield "near pair", _grid(np.clip(np.stack([c, c + d]), -0.5, 0.5 - 2.0**-22))


def test_omega_restores_the_angular_momentum():
    rng = np.random.default_rng(11)
    for n in (2, 3, 4, 7, 12, 40):
        for _ in range(30):
            rho = _grid(rng.uniform(-0.5, 0.5, (n, 3)))
            w = rng.normal(size=(n, 3)) + rng.normal(size=3) * 3.0
            om, rc, sens, fl = oracle.cell_omega(rho, w)
            assert fl & oracle.FLAG_DEGENERATE == 0
            np.testing.assert_allclose(rc, rho.mean(axis=0), rtol=0, atol=1e-15)
            r = rho - rc
            resid = np.cross(r, w - np.cross(om, r)).sum(axis=0)
            scale = np.abs(np.cross(r, w)).sum()
            if n >= 3:
                assert np.abs(resid).max() <= 1e-12 * scale
                J = np.einsum("ka,ka->", r, r) * np.eye(3) - r.T @ r
                np.testing.assert_allclose(om, np.linalg.solve(J, np.cross(r, w).sum(axis=0)),
                                           rtol=1e-9, atol=1e-12 * np.abs(om).max())
            else:
                d = r[0] - r[1]
                # a pair cannot rotate about its own axis: only the normal part is restored,
                # and omega has no component along the axis (the pseudo-inverse)
                assert abs(resid @ d) <= 1e-12 * scale * np.linalg.norm(d) + 1e-300
                resid_perp = resid - d * (resid @ d) / (d @ d)
                assert np.abs(resid_perp).max() <= 1e-12 * scale
                assert abs(om @ d) <= 1e-12 * np.linalg.norm(om) * np.linalg.norm(d)
                J = (r * r).sum() * np.eye(3) - r.T @ r
                np.testing.assert_allclose(om, np.linalg.pinv(J) @ np.cross(r, w).sum(axis=0),
                                           rtol=1e-8, atol=1e-12 * np.abs(om).max())
            assert np.all(np.isfinite(sens)) and np.all(sens > 0)


def test_collinear_cell_is_degenerate():
    rho = _grid(np.array([[-0.25, -0.25, -0.25], [0.0, 0.0, 0.0], [0.25, 0.25, 0.25]]))
    om, _, _, fl = oracle.cell_omega(rho, np.random.default_rng(1).normal(size=(3, 3)))
    assert fl & oracle.FLAG_DEGENERATE and np.all(om == 0.0)


def test_sensitivity_bounds_float32_rounding():
    rng = np.random.default_rng(7)
    per_cell = []      # (kind, max over members and orders of |dv_i| / (u sens_i))
    const_ratio = []   # the same with a constant sensitivity in place of sens_i
    sens_all = []
    for kind, rho in _cells(rng):
        n = len(rho)
        for drift in (0.0, 5.0):
            # w = v - v_ran (AT+a) has variance 2 kT/m per component; a drifting frame
            # adds a uniform velocity
            w = rng.normal(scale=np.sqrt(2.0), size=(n, 3))
            w[:, 0] += drift
            om, rc, sens, fl = oracle.cell_omega(rho, w)
            if fl & oracle.FLAG_DEGENERATE:
                continue
            exact = np.cross(om, rho - rc)
            worst, worst_abs = 0.0, 0.0
            for one_pass in ((False, True) if n >= 6 else (False,)):
                for _ in range(3):
                    o = rng.permutation(n)
                    err = np.linalg.norm(_float32_rotation_term(rho[o], w[o], one_pass) - exact[o],
                                         axis=1)
                    worst = max(worst, float((err / (U * sens[o])).max()))
                    worst_abs = max(worst_abs, float(err.max()))
            per_cell.append((kind, worst))
            const_ratio.append(worst_abs)
            sens_all.append(sens)
    ratios = np.array([r for _, r in per_cell])
    kinds = np.array([k for k, _ in per_cell])
    for k in ("uniform", "near-collinear", "near pair"):
        sel = ratios[kinds == k]
        print(f"{k}: {len(sel)} cells, |dv| / (u sens) max {sel.max():.3f}, "
              f"p90 {np.quantile(sel, 0.9):.3f}, median {np.median(sel):.3f}")
    # an upper bound, without the factor 16 of the parity bar ...
    assert ratios.max() <= 1.0
    # ... that is not inflated: its upper tail is reached to within a factor of ten
    assert np.quantile(ratios, 0.99) >= 0.1
    # a constant sensitivity (the median of the real ones) would not bound the errors
    c = float(np.median(np.concatenate(sens_all)))
    assert (np.array(const_ratio) / (U * c)).max() > 16.0


def test_one_pass_moments_fail_for_tight_pairs():
    """Why the kernel takes the raw-sum (one-pass) moments only for cells of six or more
    members: for a close pair the raw sums cancel catastrophically and the float32 error
    exceeds the sensitivity bound many times; the two-pass form stays within it."""
    rng = np.random.default_rng(5)
    bad_one, bad_two = 0.0, 0.0
    for _ in range(40):
        c = rng.uniform(-0.4, 0.4, 3)
        d = rng.normal(size=3)
        d *= 0.003 / np.linalg.norm(d)
        rho = _grid(np.stack([c, c + d]))
        w = rng.normal(scale=np.sqrt(2.0), size=(2, 3))
        om, rc, sens, _ = oracle.cell_omega(rho, w)
        exact = np.cross(om, rho - rc)
        e1 = np.linalg.norm(_float32_rotation_term(rho, w, True) - exact, axis=1) / (U * sens)
        e2 = np.linalg.norm(_float32_rotation_term(rho, w, False) - exact, axis=1) / (U * sens)
        bad_one, bad_two = max(bad_one, e1.max()), max(bad_two, e2.max())
    assert bad_two <= 1.0 < bad_one
