"""Pins of the oracle's collision step against the invariants the paper states.

* SRD, Eq. (2): the rotation D(alpha) against scipy's Rotation; per-cell conservation of
  momentum and kinetic energy (Sec. II: SRD conserves energy); |v_ic| preserved; the
  angle between v_ic and D v_ic has the closed form cos(theta) = cos(a) + (1 - cos(a))
  (n.v_hat)^2; alpha = 180 deg reduces to the reflection 2 (n.v) n - v.
* MBS thermostat, Eqs. (5)-(7): momentum conserved per cell, and the post-collision
  relative kinetic energy of a cell of n particles is exactly E_k ~ Gamma(3(n-1)/2, kT).
* SRD+a, Eqs. (3)-(4), and MPC-AT+a: per-cell linear and angular momentum conserved.
"""
import numpy as np
import pytest
from scipy import stats
from scipy.spatial.transform import Rotation

import oracle


def test_rotation_matches_scipy():
    rng = np.random.default_rng(3)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        alpha = rng.uniform(0, 2 * np.pi)
        v = rng.normal(size=3)
        ref = Rotation.from_rotvec(alpha * n).apply(v)
        np.testing.assert_allclose(oracle.rotate(n, alpha, v), ref, rtol=0, atol=1e-13)


def test_srd_axis_uniform_on_sphere():
    p = oracle.params(L=16)
    ax = np.array([oracle.srd_axis(p, 3, c) for c in range(4096)])
    np.testing.assert_allclose(np.linalg.norm(ax, axis=1), 1.0, atol=1e-14)
    assert stats.kstest(ax[:, 2], stats.uniform(-1, 2).cdf).pvalue > 1e-3
    phi = np.arctan2(ax[:, 1], ax[:, 0])
    assert stats.kstest(phi, stats.uniform(-np.pi, 2 * np.pi).cdf).pvalue > 1e-3


def _per_cell_sum(cell, values, C):
    out = np.zeros((C,) + values.shape[1:])
    np.add.at(out, cell, values)
    return out


def _rho(p, X, step):
    """positions relative to the collision-cell centre (exact, from the fixed point)"""
    F = oracle.fixed_bits(p)
    S = oracle.shift(p, step).astype(np.int64)
    t = X.astype(np.int64) + S[:, None]
    u = (t & ((1 << F) - 1)) - (1 << (F - 1))
    return (u / 2.0**F).T


def _run_one(p, steps=1, want_state_step=0):
    X, V, ids = oracle.init(p)
    X, V, ids, _ = oracle.run(p, want_state_step, state=(X, V, ids))
    r = oracle.step(p, X, V, ids, want_state_step, cells=True, counts=True, vpre=True,
                    flags=True)
    return r


@pytest.mark.parametrize("alpha", [130.0, 90.0, 180.0, 17.0])
def test_srd_conserves_momentum_energy_and_rotates(alpha):
    p = oracle.params(L=8, n_c=6, alpha_deg=alpha, seed=21)
    r = _run_one(p, want_state_step=2)
    C = oracle.num_cells(p)
    vb, vn, cell = r["vpre"].T, r["V"].T, r["cell"]
    P0, P1 = _per_cell_sum(cell, vb, C), _per_cell_sum(cell, vn, C)
    E0 = _per_cell_sum(cell, (vb**2).sum(1), C)
    E1 = _per_cell_sum(cell, (vn**2).sum(1), C)
    np.testing.assert_allclose(P1, P0, atol=1e-12)
    np.testing.assert_allclose(E1, E0, rtol=1e-12, atol=1e-12)
    n = np.bincount(cell, minlength=C)
    vcm = P0 / np.maximum(n, 1)[:, None]
    rel0 = vb - vcm[cell]
    rel1 = vn - vcm[cell]
    np.testing.assert_allclose(np.linalg.norm(rel1, axis=1), np.linalg.norm(rel0, axis=1),
                               rtol=1e-11, atol=1e-12)
    a = np.deg2rad(alpha)
    axes = np.array([oracle.srd_axis(p, 2, c) for c in range(C)])
    nh = axes[cell]
    norm0 = np.linalg.norm(rel0, axis=1)
    ok = norm0 > 1e-6
    cos_theta = (rel0 * rel1).sum(1)[ok] / norm0[ok] ** 2
    nv = (nh * rel0).sum(1)[ok] / norm0[ok]
    np.testing.assert_allclose(cos_theta, np.cos(a) + (1 - np.cos(a)) * nv**2, atol=1e-11)
    if alpha == 180.0:
        ref = 2 * (nh * rel0).sum(1)[:, None] * nh - rel0
        np.testing.assert_allclose(rel1, ref, atol=1e-12)


def test_single_particle_cells_unchanged():
    p = oracle.params(L=8, n_c=0.3, seed=4)
    r = _run_one(p, want_state_step=0)
    cell, C = r["cell"], oracle.num_cells(p)
    n = np.bincount(cell, minlength=C)
    lone = n[cell] == 1
    assert lone.sum() > 20
    np.testing.assert_array_equal(r["V"].T[lone], r["vpre"].T[lone])


def test_mbs_thermostat_gamma_energy_and_momentum():
    """Eqs. (5)-(7): after scaling, sum_i m v_ic'^2 / 2 = E_k ~ Gamma(f/2, kT), f = 3(n-1)."""
    kT = 1.7
    p = oracle.params(L=12, n_c=10, thermostat=1, kT=kT, seed=8)
    X, V, ids = oracle.init(p)
    samples = {}
    for s in range(4):
        r = oracle.step(p, X, V, ids, s, cells=True, vpre=True)
        C = oracle.num_cells(p)
        vb, vn, cell = r["vpre"].T, r["V"].T, r["cell"]
        np.testing.assert_allclose(_per_cell_sum(cell, vn, C), _per_cell_sum(cell, vb, C),
                                   atol=1e-11)
        n = np.bincount(cell, minlength=C)
        vcm = _per_cell_sum(cell, vn, C) / np.maximum(n, 1)[:, None]
        K = 0.5 * _per_cell_sum(cell, ((vn - vcm[cell]) ** 2).sum(1), C)
        for nc in (6, 10, 14):
            samples.setdefault(nc, []).extend(K[n == nc])
        X, V = r["X"], r["V"]
    for nc, ks in samples.items():
        ks = np.asarray(ks)
        assert ks.size > 200
        assert stats.kstest(ks, stats.gamma(1.5 * (nc - 1), scale=kT).cdf).pvalue > 1e-3, nc


def _angular_momentum_check(p, step_index, tol):
    X, V, ids = oracle.init(p)
    X, V, ids, _ = oracle.run(p, step_index, state=(X, V, ids))
    r = oracle.step(p, X, V, ids, step_index, cells=True, vpre=True, flags=True)
    C = oracle.num_cells(p)
    vb, vn, cell = r["vpre"].T, r["V"].T, r["cell"]
    rho = _rho(p, r["X"], step_index)
    P0, P1 = _per_cell_sum(cell, vb, C), _per_cell_sum(cell, vn, C)
    np.testing.assert_allclose(P1, P0, atol=1e-11)
    L0 = _per_cell_sum(cell, np.cross(rho, vb), C)
    L1 = _per_cell_sum(cell, np.cross(rho, vn), C)
    bad = (r["flags"] & oracle.FLAG_DEGENERATE) != 0
    np.testing.assert_allclose(L1[~bad], L0[~bad], atol=tol)
    return r


@pytest.mark.parametrize("n_c", [3.0, 10.0])
def test_at_a_conserves_linear_and_angular_momentum(n_c):
    p = oracle.params(L=8, n_c=n_c, variant=oracle.AT_A, h=0.05, seed=31)
    r = _angular_momentum_check(p, 1, 1e-9)
    n = np.bincount(r["cell"], minlength=oracle.num_cells(p))
    if n_c == 3.0:
        assert (n == 2).sum() > 20  # the pair (pseudo-inverse) branch is exercised


def test_srd_a_conserves_linear_and_angular_momentum():
    p = oracle.params(L=8, n_c=10, variant=oracle.SRD_A, h=0.1, seed=32)
    _angular_momentum_check(p, 2, 1e-9)


def test_plain_srd_does_not_conserve_angular_momentum():
    """Control for the test above: Eq. (2) alone changes the cell angular momentum
    (Sec. II, 'Angular-momentum conservation')."""
    p = oracle.params(L=8, n_c=10, variant=oracle.SRD, seed=32)
    X, V, ids = oracle.init(p)
    r = oracle.step(p, X, V, ids, 0, cells=True, vpre=True)
    C = oracle.num_cells(p)
    rho = _rho(p, r["X"], 0)
    L0 = _per_cell_sum(r["cell"], np.cross(rho, r["vpre"].T), C)
    L1 = _per_cell_sum(r["cell"], np.cross(rho, r["V"].T), C)
    assert np.abs(L1 - L0).max() > 0.1


def test_at_a_random_part_variance():
    """AT+a draws the relative velocities from N(0, kT/m), so it thermostats by itself:
    the kinetic temperature relaxes to kT within a few collisions."""
    kT = 0.8
    p = oracle.params(L=8, n_c=10, variant=oracle.AT_A, h=0.05, kT=kT, seed=33)
    X, V, ids, obs = oracle.run(p, 30, obs=True)
    T = np.array([o["temperature"] for o in obs[10:]])
    assert abs(T.mean() - kT) < 0.02


def test_min_eigenvalue_matches_numpy():
    """The closed-form smallest eigenvalue (used to scale the float32 parity bound of the
    angular-momentum variants) against LAPACK."""
    rng = np.random.default_rng(9)
    for _ in range(300):
        A = rng.normal(size=(3, 3))
        A = A @ A.T * rng.uniform(1e-4, 10)
        if rng.random() < 0.2:
            A = np.diag(np.diag(A))
        ref = np.linalg.eigvalsh(A)
        assert abs(oracle.min_eigenvalue_sym3(A) - ref[0]) <= 1e-9 * np.abs(A).max()
        assert abs(oracle.max_eigenvalue_sym3(A) - ref[2]) <= 1e-9 * np.abs(A).max()


def test_ill_conditioned_flag_follows_the_eigenvalue_ratio():
    """FLAG_ILL_CONDITIONED marks the cells of three or more members whose inertia tensor
    has lambda_max / lambda_min above COND_FLOAT32 (checked with numpy's eigvalsh on the
    oracle's own collision positions), and no others."""
    p = oracle.params(L=12, n_c=4.0, h=0.05, variant=oracle.AT_A, seed=21)
    X, V, ids = oracle.init(p)
    r = oracle.step(p, X, V, ids, 0, cells=True, counts=True, flags=True)
    F = oracle.fixed_bits(p)
    S = oracle.shift(p, 0).astype(np.int64)
    rho = (((r["X"].astype(np.int64) + S[:, None]) & ((1 << F) - 1)) / 2.0**F - 0.5).T
    flagged, checked = 0, 0
    for c in np.flatnonzero(r["counts"] >= 3):
        m = rho[r["cell"] == c]
        q = m - m.mean(axis=0)
        J = (q * q).sum() * np.eye(3) - q.T @ q
        ev = np.linalg.eigvalsh(J)
        ill = ev[2] > oracle.COND_FLOAT32 * ev[0]
        if abs(ev[2] / ev[0] / oracle.COND_FLOAT32 - 1.0) < 1e-9:
            continue  # on the threshold
        assert bool(r["flags"][c] & oracle.FLAG_ILL_CONDITIONED) == ill, c
        flagged += ill
        checked += 1
    assert checked > 1000 and flagged > 10  # N_c = 4: small cells, often ill-conditioned


def test_tight_clusters_are_flagged():
    """Members within TIGHT_RMS (rms) of their centre of mass are flagged
    FLAG_ILL_CONDITIONED whatever the shape; slightly wider clusters of the same shape
    are not."""
    rng = np.random.default_rng(4)
    for n in (2, 3, 6):
        for _ in range(20):
            shape = rng.normal(size=(n, 3))
            shape -= shape.mean(axis=0)
            shape /= np.sqrt((shape**2).sum() / n)  # rms radius 1
            c = rng.uniform(-0.3, 0.3, 3)
            w = rng.normal(size=(n, 3))
            ev = np.linalg.eigvalsh((shape**2).sum() * np.eye(3) - shape.T @ shape)
            if n >= 3 and ev[2] > 0.5 * oracle.COND_FLOAT32 * ev[0]:
                continue  # keep clear of the conditioning criterion
            for rms, expect in ((0.9 * oracle.TIGHT_RMS, True), (1.1 * oracle.TIGHT_RMS, False)):
                _, _, _, fl = oracle.cell_omega(c + rms * shape, w)
                assert bool(fl & oracle.FLAG_ILL_CONDITIONED) == expect, (n, rms)
