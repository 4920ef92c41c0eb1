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
