"""Pins of the oracle's phantom particles (Sec. II, "Boundary conditions").

In a collision cell cut by a no-slip wall, the part inside the wall is filled with
virtual particles at the fluid's mean density N_c, with Maxwell-Boltzmann velocities of
variance kT/m about the wall's velocity (the paper's "variance sqrt(kT/m)" is read as
variance kT/m).  An SRD collision sees only their aggregates, which the oracle draws
directly: the count k, the total momentum and K = sum m |v - <v>|^2 about their own mean
(twice their internal kinetic energy).
Pinned here against the definition -- k independent Gaussian particles -- by
distribution tests over many cells:
  * k ~ Poisson(N_c phi) for wall volume fraction phi (chi-square test);
  * total momentum per component ~ m k u_wall + N(0, k m kT) (KS test of the
    standardised values, and a two-sample test against explicit Gaussian particles);
  * K ~ kT chi^2(3(k - 1)) (KS test of the CDF-transformed values, and a two-sample test
    against explicit Gaussian particles).
"""
import numpy as np
import pytest
from scipy import stats

import oracle

M, KT, N_C = 2.0, 1.5, 7.0
U_WALL = (0.3, -0.2)


def _draws(phi, wall, n_cells=4000, steps=(0, 1, 2)):
    p = oracle.params(L=(16, 16, 16), n_c=N_C, kT=KT, m=M, walls_z=1, thermostat=1, seed=31,
                      wall_u=U_WALL)
    out = []
    for s in steps:
        for c in range(n_cells):
            k, P, K, _ = oracle.phantoms(p, s, c, phi, wall)
            out.append((k, P[0], P[1], P[2], K))
    return np.array(out)


@pytest.mark.parametrize("phi", [0.13, 0.5, 0.91])
def test_phantom_count_is_poisson(phi):
    d = _draws(phi, 0)
    k = d[:, 0].astype(int)
    lam = N_C * phi
    kmax = int(stats.poisson(lam).ppf(1 - 1e-4)) + 1
    obs = np.bincount(np.minimum(k, kmax), minlength=kmax + 1)
    pmf = stats.poisson(lam).pmf(np.arange(kmax + 1))
    pmf[-1] = stats.poisson(lam).sf(kmax - 1)
    exp = pmf * len(k)
    keep = exp >= 5
    chi2 = (((obs - exp) ** 2) / exp)[keep].sum() + ((obs[~keep].sum() - exp[~keep].sum()) ** 2
                                                     / max(exp[~keep].sum(), 1e-9))
    dof = keep.sum()
    assert stats.chi2(dof).sf(chi2) > 1e-3
    assert abs(k.mean() - lam) < 4 * np.sqrt(lam / len(k))


@pytest.mark.parametrize("wall", [0, 1])
def test_phantom_momentum_and_internal_energy(wall):
    d = _draws(0.6, wall)
    k, P, K = d[:, 0], d[:, 1:4], d[:, 4]
    has = k >= 1
    # momentum: m k u_wall + N(0, k m kT) per component
    z = (P[has] - np.outer(M * k[has], [U_WALL[wall], 0.0, 0.0])) / np.sqrt(k[has] * M * KT)[:, None]
    for a in range(3):
        assert stats.kstest(z[:, a], "norm").pvalue > 1e-3
    assert np.all(P[~has] == 0.0) and np.all(K[~has] == 0.0)
    # K about the phantoms' own mean: kT chi^2(3(k - 1)); zero for one phantom
    two = k >= 2
    assert np.all(K[k == 1] == 0.0)
    u = stats.chi2.cdf(K[two] / KT, 3 * (k[two] - 1))
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_aggregates_match_explicit_gaussian_particles():
    """The definition: k particles with independent Maxwell-Boltzmann velocities about the
    wall velocity.  Their total momentum and sum m |v - <v>|^2, drawn explicitly (numpy),
    have the same distributions as the oracle's aggregates for the same counts."""
    d = _draws(0.8, 1, n_cells=6000, steps=(4,))
    k = d[:, 0].astype(int)
    rng = np.random.default_rng(2)
    P_ex, K_ex = [], []
    for kk in k:
        v = rng.normal(scale=np.sqrt(KT / M), size=(kk, 3)) + np.array([U_WALL[1], 0.0, 0.0])
        P_ex.append(M * v.sum(axis=0) if kk else np.zeros(3))
        K_ex.append(M * ((v - v.mean(axis=0)) ** 2).sum() if kk else 0.0)  # sum m |v - <v>|^2
    P_ex, K_ex = np.array(P_ex), np.array(K_ex)
    for a in range(3):
        assert stats.ks_2samp(d[:, 1 + a], P_ex[:, a]).pvalue > 1e-3
    assert stats.ks_2samp(d[:, 4], K_ex).pvalue > 1e-3
    assert abs(d[:, 4].mean() - K_ex.mean()) < 0.05 * K_ex.mean()


def test_phantom_particles_fill_the_wall_part():
    """For the angular-momentum-conserving variants the phantoms are drawn one by one:
    uniform positions in the part of the cell beyond the wall (x, y over the whole cell),
    velocities N(u_wall, kT/m) and random velocities N(0, kT/m) per component; their
    number is the count of the aggregate draw."""
    p = oracle.params(L=(16, 16, 16), n_c=N_C, kT=KT, m=M, walls_z=1, variant=oracle.AT_A,
                      seed=33, wall_u=U_WALL)
    F = oracle.fixed_bits(p)
    sig = np.sqrt(KT / M)
    for wall, frac in ((0, 0.37), (1, 0.62)):
        Sz = int(frac * 2**F)
        s = Sz / 2.0**F
        phi = s if wall == 0 else 1.0 - s
        rho, v, vr = [], [], []
        for c in range(3000):
            k = oracle.phantoms(p, 2, c, phi, wall)[0]
            r_, v_, u_ = oracle.phantom_particles(p, 2, c, Sz, wall, k)
            rho.append(r_)
            v.append(v_)
            vr.append(u_)
        rho, v, vr = np.concatenate(rho), np.concatenate(v), np.concatenate(vr)
        lo, hi = (-0.5, s - 0.5) if wall == 0 else (s - 0.5, 0.5)
        assert rho[:, 2].min() >= lo and rho[:, 2].max() < hi
        assert stats.kstest(rho[:, 2], stats.uniform(lo, hi - lo).cdf).pvalue > 1e-3
        for a in (0, 1):
            assert stats.kstest(rho[:, a], stats.uniform(-0.5, 1.0).cdf).pvalue > 1e-3
        assert stats.kstest((v[:, 0] - U_WALL[wall]) / sig, "norm").pvalue > 1e-3
        for a in (1, 2):
            assert stats.kstest(v[:, a] / sig, "norm").pvalue > 1e-3
        for a in range(3):
            assert stats.kstest(vr[:, a] / sig, "norm").pvalue > 1e-3
        assert abs(len(rho) / 3000 - N_C * phi) < 4 * np.sqrt(N_C * phi / 3000)


def _wall_cells_members(p, step, X_after, cell):
    F = oracle.fixed_bits(p)
    S = oracle.shift(p, step).astype(np.int64)
    rho = (((X_after.astype(np.int64) + S[:, None]) & ((1 << F) - 1)) / 2.0**F - 0.5).T
    Lx, Ly, Lz = p.L
    cz = cell // (Lx * Ly)
    return rho, cz, int(S[2])


def _vran_fluid(p, ids, step):
    """AT+a random velocities of fluid particles: Philox(id, step, tag 6) through
    Box-Muller, restated in numpy from the published transform"""
    sig = np.sqrt(p.kT / p.m)
    out = np.zeros((len(ids), 3))
    key = [p.seed & 0xFFFFFFFF, p.seed >> 32]
    for i, pid in enumerate(ids):
        r = oracle.philox([int(pid), step, 6 << 24, p.box], key)
        u = (np.asarray(r, dtype=np.float64) // 512 + 0.5) / 2.0**23
        R0, R1 = np.sqrt(-2 * np.log(u[0])), np.sqrt(-2 * np.log(u[2]))
        out[i] = sig * np.array([R0 * np.cos(2 * np.pi * u[1]), R0 * np.sin(2 * np.pi * u[1]),
                                 R1 * np.cos(2 * np.pi * u[3])])
    return out


@pytest.mark.parametrize("variant", [oracle.AT_A, oracle.SRD_A])
def test_no_slip_wall_cells_conserve_momentum_and_angular_momentum_with_phantoms(variant):
    """In a cell cut by a no-slip wall the collision acts on fluid and phantom particles
    together: recomputing it in numpy from the members (np.linalg.solve for omega), the
    fluid velocities match the oracle's, and the linear and angular momentum of all
    members (the phantoms' post-collision velocities included) are conserved."""
    p = oracle.params(L=(6, 6, 5), n_c=6.0, h=0.1, alpha_deg=120.0, variant=variant,
                      walls_z=1, wall_u=(0.2, -0.1), seed=41)
    X, V, ids = oracle.init(p)
    step = 2
    X, V, ids, _ = oracle.run(p, step, state=(X, V, ids))
    r = oracle.step(p, X, V, ids, step, cells=True, counts=True, vpre=True, flags=True)
    rho, cz, Sz = _wall_cells_members(p, step, r["X"], r["cell"])
    F = oracle.fixed_bits(p)
    s = Sz / 2.0**F
    checked = 0
    for c in np.flatnonzero(r["counts"] > 0):
        czc = c // 36
        if czc not in (0, p.L[2]) or r["flags"][c] & oracle.FLAG_DEGENERATE:
            continue
        wall = 0 if czc == 0 else 1
        phi = s if wall == 0 else 1.0 - s
        k = oracle.phantoms(p, step, int(c), phi, wall)[0]
        if k == 0:
            continue
        rp, vp, up = oracle.phantom_particles(p, step, int(c), Sz, wall, k)
        m_idx = np.flatnonzero(r["cell"] == c)
        R = np.concatenate([rho[m_idx], rp])
        Vb = np.concatenate([r["vpre"][:, m_idx].T, vp])
        vcm = Vb.mean(axis=0)
        rc = R.mean(axis=0)
        q = R - rc
        J = (q * q).sum() * np.eye(3) - q.T @ q
        if variant == oracle.AT_A:
            U = np.concatenate([_vran_fluid(p, ids[m_idx], step), up])
            W = Vb - U
            om = np.linalg.solve(J, np.cross(q, W).sum(axis=0))
            new = vcm + U - U.mean(axis=0) + np.cross(om, q)
        else:
            ax = oracle.srd_axis(p, step, int(c))
            D = np.array([oracle.rotate(ax, np.deg2rad(120.0), e) for e in np.eye(3)]).T
            vic = Vb - vcm
            W = vic - vic @ D.T
            om = np.linalg.solve(J, np.cross(q, W).sum(axis=0))
            new = vcm + vic @ D.T + np.cross(om, q)
        np.testing.assert_allclose(new[: len(m_idx)], r["V"][:, m_idx].T, rtol=0, atol=1e-9)
        np.testing.assert_allclose(new.sum(axis=0), Vb.sum(axis=0), rtol=0, atol=1e-9)
        np.testing.assert_allclose(np.cross(q, new).sum(axis=0), np.cross(q, Vb).sum(axis=0),
                                   rtol=0, atol=1e-9)
        checked += 1
    assert checked > 10
