"""Physics pins of the oracle: initial state, equipartition and Maxwell-Boltzmann
statistics, and Poiseuille flow between no-slip walls under gravity (Sec. II:
'External fields' + 'Boundary conditions' + 'Thermostat') against its closed form with
the SRD viscosity closed forms of the transport theory the paper cites (Kikuchi et al.
2003; Noguchi & Gompper 2008):
  eta_kin = N_c kT h [5 N_c / ((N_c - 1 + e^-N_c)(4 - 2 cos a - 2 cos 2a)) - 1/2]
  eta_col = m (N_c - 1 + e^-N_c)(1 - cos a) / (18 h)          (a = m = 1).
"""
import numpy as np
import pytest
from scipy import stats

import oracle


def eta_srd(n_c, h, alpha_deg, kT=1.0):
    a = np.deg2rad(alpha_deg)
    z = n_c - 1 + np.exp(-n_c)
    kin = n_c * kT * h * (5 * n_c / (z * (4 - 2 * np.cos(a) - 2 * np.cos(2 * a))) - 0.5)
    col = z * (1 - np.cos(a)) / (18 * h)
    return kin + col


def test_eta_closed_form_value():
    # N_c = 10, h = 0.1, alpha = 130 deg -> 0.486 + 8.214
    assert abs(eta_srd(10, 0.1, 130) - 8.700) < 2e-3


def test_initial_state():
    p = oracle.params(L=(12, 10, 8), n_c=10, kT=2.0, seed=17)
    X, V, ids = oracle.init(p)
    N = oracle.num_particles(p)
    assert N == 12 * 10 * 8 * 10
    np.testing.assert_array_equal(ids, np.arange(N))
    np.testing.assert_allclose(V.mean(axis=1), 0.0, atol=1e-13)
    F = oracle.fixed_bits(p)
    for ax, L in enumerate((12, 10, 8)):
        assert X[ax].max() < L * 2**F
        counts = np.bincount(X[ax] >> F, minlength=L)
        assert stats.chisquare(counts).pvalue > 1e-3
        assert abs(V[ax].var() - 2.0) < 5 * 2.0 * np.sqrt(2.0 / N)
    assert stats.kstest(V[0] / np.sqrt(2.0), "norm").pvalue > 1e-3


def test_equipartition_and_maxwell_boltzmann_after_srd():
    """SRD is microcanonical: the temperature set at initialisation persists, every
    component carries kT/2, and velocities become Maxwellian (kurtosis 3)."""
    p = oracle.params(L=10, n_c=10, h=0.1, alpha_deg=130, seed=19)
    X, V, ids, obs = oracle.run(p, 100, obs=True)
    N = X.shape[1]
    T = obs[-1]["temperature"]
    assert abs(T - 1.0) < 5 * np.sqrt(2.0 / (3 * N))
    var = V.var(axis=1)
    np.testing.assert_allclose(var, T, rtol=6 * np.sqrt(2.0 / N))
    assert abs(stats.kurtosis(V.ravel(), fisher=False) - 3.0) < 0.06
    assert stats.kstest(V.ravel() / np.sqrt(T), "norm").pvalue > 1e-3
    P = np.array([obs[-1]["px"], obs[-1]["py"], obs[-1]["pz"]])
    assert np.abs(P).max() < 1e-9


def poiseuille_eta(Lz=10, g=0.05, n_c=10.0, seed=5):
    """The oracle's viscosity estimate from a Poiseuille profile: returns (eta, slip,
    profile, z, mean temperature)."""
    p = oracle.params(L=(6, 6, Lz), n_c=n_c, h=0.1, alpha_deg=130, walls_z=1, thermostat=1,
                      g=(g, 0, 0), seed=seed)
    X, V, ids = oracle.init(p)
    F = oracle.fixed_bits(p)
    nb = 2 * Lz
    prof, cnt = np.zeros(nb), np.zeros(nb)
    temps = []
    for s in range(2500):
        r = oracle.step(p, X, V, ids, s, obs=(s % 50 == 0))
        X, V = r["X"], r["V"]
        if s >= 500:
            b = np.minimum((X[2] / 2.0**F / Lz * nb).astype(int), nb - 1)
            np.add.at(prof, b, V[0])
            np.add.at(cnt, b, 1)
            if "obs" in r:
                temps.append(r["obs"]["temperature"])
    z = (np.arange(nb) + 0.5) * Lz / nb
    v = prof / cnt
    M = np.stack([z * (Lz - z), np.ones_like(z)], 1)
    (A, slip), *_ = np.linalg.lstsq(M, v, rcond=None)
    return n_c * g / (2 * A), slip, v, z, float(np.mean(temps))


def test_poiseuille_flow_between_no_slip_walls():
    """Body force g along x, bounce-back walls + phantom particles at z = 0, Lz, MBS
    thermostat: steady profile v_x(z) = (rho g / 2 eta) z (Lz - z) (plus a small slip)."""
    Lz, g, n_c = 10, 0.05, 10.0
    eta, slip, v, z, temp = poiseuille_eta(Lz, g, n_c)
    eta_th = eta_srd(n_c, 0.1, 130)
    assert abs(eta - eta_th) / eta_th < 0.05, eta
    vmax = n_c * g * Lz**2 / (8 * eta_th)
    assert abs(slip) < 0.1 * vmax
    # symmetric about the channel centre, flowing along +x
    np.testing.assert_allclose(v, v[::-1], atol=0.03)
    assert v.min() > 0
    # the thermostat removes the viscous heating (temperature about the flow profile
    # is reported by the kinetic estimator including the mean flow, so allow vmax^2/3)
    assert abs(temp - 1.0) < 0.05 + vmax**2 / 3
