"""Pins of the oracle's slip walls and moving no-slip walls (Sec. II, "Boundary
conditions": specular reflection for slip walls; bounce-back, in the frame of a moving
wall, for no-slip walls, which with moving walls drive shear flow).

Checked against: continuous-time closed forms of the reflections (written as the time of
flight before and after the hit, not as the implementation's rational formula); exact
conservation laws that only hold for the intended boundary (slip walls without phantom
particles conserve the kinetic energy of an SRD fluid and its tangential momentum, so a
body force accelerates the whole fluid uniformly); the linear Couette profile between
walls moving in opposite directions.
"""
from fractions import Fraction

import numpy as np

import oracle


def _round_half_even(fr: Fraction) -> int:
    return int(round(fr))  # Python rounds Fractions half to even


def test_slip_wall_specular_reflection():
    p = oracle.params(L=(8, 8, 8), h=0.1, walls_z=oracle.SLIP)
    F = oracle.fixed_bits(p)
    # bottom wall: z = 0.05, v = (0.3, -0.2, -1.0): the tangential motion continues for the
    # whole step, z is mirrored about the wall, only v_z flips
    x0 = [3 * 2**F, 4 * 2**F, int(0.05 * 2**F)]
    x, v = oracle.stream_one(p, x0, [0.3, -0.2, -1.0])
    assert abs((x[0] - x0[0]) / 2**F - 0.03) < 2 * 2.0**-F
    assert abs((int(x[1]) - x0[1]) / 2**F + 0.02) < 2 * 2.0**-F
    assert abs(x[2] / 2**F - 0.05) < 3 * 2.0**-F
    np.testing.assert_array_equal(v, [0.3, -0.2, 1.0])
    # top wall
    x, v = oracle.stream_one(p, [2**F, 2**F, int(7.98 * 2**F)], [1.0, 0.5, 0.4])
    assert abs(x[0] / 2**F - 1.1) < 2 * 2.0**-F and abs(x[1] / 2**F - 1.05) < 2 * 2.0**-F
    assert abs(x[2] / 2**F - 7.98) < 3 * 2.0**-F
    np.testing.assert_array_equal(v, [1.0, 0.5, -0.4])


def test_moving_no_slip_wall_bounce_back():
    """A wall moving with u along x: the particle flies with v until it meets the wall
    after a time t_w, then with 2u - v for the rest of the step."""
    h, u = 0.1, (0.25, -0.6)
    p = oracle.params(L=(8, 8, 8), h=h, walls_z=oracle.NO_SLIP, wall_u=u)
    F = oracle.fixed_bits(p)
    s = 2**F
    P = 8 * s
    for (z0, vel, top) in (((int(0.02 * s)), (1.0, 0.3, -0.5), 0),
                           ((int(7.97 * s)), (-0.7, 0.1, 0.45), 1),
                           ((int(0.003 * s)), (0.2, 0.0, -1.7), 0)):
        x0 = [3 * s, 2 * s, z0]
        x, v = oracle.stream_one(p, x0, list(vel))
        # fixed-point free displacements (the state contract) and the wall positions
        d = [int(np.rint(np.float32(c) * np.float32(h * s))) for c in vel]
        U = int(np.rint(np.float32(u[top]) * np.float32(h * s)))
        w = Fraction(2 * P - 1, 2) if top else Fraction(-1, 2)
        t_w = (w - z0) / d[2]  # fraction of the step before the hit
        x_exp = x0[0] + d[0] * t_w + (2 * U - d[0]) * (1 - t_w)
        y_exp = x0[1] + d[1] * t_w - d[1] * (1 - t_w)
        z_exp = 2 * w - (z0 + d[2])
        assert x[0] == _round_half_even(x_exp) % P
        assert x[1] == _round_half_even(y_exp) % P
        assert x[2] == z_exp
        np.testing.assert_allclose(v, [2 * u[top] - vel[0], -vel[1], -vel[2]], rtol=0, atol=1e-12)


def test_slip_walls_conserve_energy_and_tangential_momentum():
    """SRD with slip walls and no thermostat: no phantom particles, specular reflection
    preserves |v| and the tangential momentum -- kinetic energy and P_x, P_y are conserved
    exactly; with a body force along x, P_x grows by N m g h per step."""
    p = oracle.params(L=(6, 5, 7), n_c=8.0, h=0.1, walls_z=oracle.SLIP, seed=3)
    X, V, ids, obs = oracle.run(p, 40, obs=True)
    e = np.array([o["ekin"] for o in obs])
    np.testing.assert_allclose(e, e[0], rtol=1e-12)
    px = np.array([o["px"] for o in obs])
    assert np.abs(px).max() < 1e-9 * np.abs(V).sum()
    g = 2e-3
    pg = oracle.params(L=(6, 5, 7), n_c=8.0, h=0.1, walls_z=oracle.SLIP, seed=3, g=(g, 0.0, 0.0))
    X, V, ids, obs = oracle.run(pg, 40, obs=True)
    N = X.shape[1]
    px = np.array([o["px"] for o in obs])
    steps = np.arange(1, 41)
    np.testing.assert_allclose(px - px[0], (steps - 1) * N * np.float32(g * 0.1), rtol=2e-6,
                               atol=1e-9 * N)


def test_no_slip_walls_do_not_conserve_energy():
    """With phantom particles (no-slip walls) the wall cells exchange energy with the
    walls -- the difference from the slip case is real."""
    p = oracle.params(L=(6, 5, 7), n_c=8.0, h=0.1, walls_z=oracle.NO_SLIP, seed=3)
    X, V, ids, obs = oracle.run(p, 20, obs=True)
    e = np.array([o["ekin"] for o in obs])
    assert np.abs(e / e[0] - 1).max() > 1e-6


def test_couette_flow_between_moving_walls():
    """Walls at z = 0 and z = Lz moving with -U/2 and +U/2 along x, MBS thermostat: the
    steady profile is linear, v_x(z) = U (z / Lz - 1/2), up to a small slip."""
    Lz, U = 10, 0.4
    p = oracle.params(L=(6, 6, Lz), n_c=10.0, h=0.1, alpha_deg=130, walls_z=oracle.NO_SLIP,
                      thermostat=1, wall_u=(-U / 2, U / 2), seed=9)
    X, V, ids = oracle.init(p)
    F = oracle.fixed_bits(p)
    nb = 10
    prof, cnt = np.zeros(nb), np.zeros(nb)
    for s in range(1500):
        r = oracle.step(p, X, V, ids, s)
        X, V = r["X"], r["V"]
        if s >= 400:
            b = np.minimum((X[2] / 2.0**F / Lz * nb).astype(int), nb - 1)
            np.add.at(prof, b, V[0])
            np.add.at(cnt, b, 1)
    z = (np.arange(nb) + 0.5) * Lz / nb
    v = prof / cnt
    slope, icept = np.polyfit(z - Lz / 2, v, 1)
    assert abs(slope - U / Lz) < 0.1 * U / Lz, slope
    assert abs(icept) < 0.02 * U
    resid = v - (slope * (z - Lz / 2) + icept)
    assert np.abs(resid).max() < 0.1 * U  # linear
