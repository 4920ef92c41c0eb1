"""Pins of the oracle's streaming (Eq. 1), boundary conditions (Sec. II) and cell
assignment on the randomly shifted lattice (Sec. II; Sec. III.B.2 "the respective
collision cell ... is calculated from the position, the random shift and applicable
boundary conditions").

Cell membership is checked against exact rational interval containment, enumerated
over every cell of 2^3 and 3^3 boxes -- a different computation from the oracle's
integer shift-and-floor.  Streaming is checked against the closed-form ballistic and
bounce-back trajectories.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("L", [2, 3, 4, 7, 16, 100, 128, 512, 1000, 1024])
def test_fixed_point_bits(L):
    """F is the largest number of fraction bits with L * 2^F <= 2^31."""
    F = oracle.fixed_bits(oracle.params(L=L))
    assert L * 2**F <= 2**31 < L * 2 ** (F + 1)


def _brute_cell(Lxyz, walls, X, S, F):
    """Enumerate every cell k of the shifted lattice; cell k of an axis covers
    [k - s, k + 1 - s) (and its periodic image).  Returns (linear cell, rho)."""
    one = 2**F
    ks, rhos = [], []
    for ax in range(3):
        L = Lxyz[ax]
        x = Fraction(int(X[ax]), one)
        s = Fraction(int(S[ax]), one)
        periodic = ax < 2 or not walls
        ncell = L if periodic else L + 1
        hits = []
        for k in range(ncell):
            lo, hi = k - s, k + 1 - s
            images = (x, x + L, x - L) if periodic else (x,)
            for xi in images:
                if lo <= xi < hi:
                    hits.append((k, xi - (lo + Fraction(1, 2))))
        assert len(hits) == 1, (ax, hits)
        ks.append(hits[0][0])
        rhos.append(hits[0][1])
    c = ks[0] + Lxyz[0] * (ks[1] + Lxyz[1] * ks[2])
    return c, rhos


@pytest.mark.parametrize("L,walls", [((2, 2, 2), 0), ((3, 3, 3), 0), ((2, 3, 2), 1),
                                     ((3, 2, 4), 0)])
def test_cell_assignment_matches_rational_enumeration(L, walls):
    p = oracle.params(L=L, walls_z=walls)
    F = oracle.fixed_bits(p)
    rng = np.random.default_rng(1234)
    P = [l * 2**F for l in L]
    for _ in range(400):
        X = [int(rng.integers(0, P[ax])) for ax in range(3)]
        S = [int(rng.integers(0, 2**F)) for ax in range(3)]
        # also land exactly on lattice planes now and then
        if rng.random() < 0.2:
            ax = int(rng.integers(0, 3))
            k = int(rng.integers(0, L[ax]))
            X[ax] = (k * 2**F - S[ax]) % P[ax]
        c, rho = oracle.cell_of(p, X, S)
        cb, rhob = _brute_cell(L, walls, X, S, F)
        assert c == cb
        for ax in range(3):
            assert rho[ax] == float(rhob[ax])


def test_cell_assignment_hand_worked():
    # L = 2, F = 30: x = (0.3, 1.7, 0.9) (rounded to the grid), s = (0.8, 0.2, 0.05):
    # x+s = (1.1, 1.9, 0.95) -> cell (1, 1, 0) -> linear 1 + 2*(1 + 2*0) = 3.
    p = oracle.params(L=2)
    F = oracle.fixed_bits(p)
    assert F == 30
    X = [round(v * 2**F) for v in (0.3, 1.7, 0.9)]
    S = [round(v * 2**F) for v in (0.8, 0.2, 0.05)]
    c, rho = oracle.cell_of(p, X, S)
    assert c == 3
    np.testing.assert_allclose(rho, [1.1 - 1.5, 1.9 - 1.5, 0.95 - 0.5], atol=1e-8)
    # periodic wrap: x + s = 1.7 + 0.6 = 2.3 -> cell 0 along x
    c2, _ = oracle.cell_of(p, [round(1.7 * 2**F), 0, 0], [round(0.6 * 2**F), 0, 0])
    assert c2 == 0


def test_free_flight_is_exact_and_ballistic():
    """Eq. (1) with no collision: r(t + kh) = r(t) + k h v, exactly in the fixed-point
    contract (constant integer displacement), to within 2^-F plus float rounding."""
    p = oracle.params(L=16, h=0.1)
    F = oracle.fixed_bits(p)
    P = 16 * 2**F
    rng = np.random.default_rng(5)
    for _ in range(50):
        x0 = rng.integers(0, P, size=3).astype(np.uint32)
        v0 = rng.normal(size=3).astype(np.float32).astype(np.float64)
        x, v = x0.copy(), v0.copy()
        x1, _ = oracle.stream_one(p, x, v)
        d = (x1.astype(np.int64) - x0.astype(np.int64) + P // 2) % P - P // 2
        assert np.all(np.abs(d / 2**F - v0 * 0.1) <= 2.0**-F + np.abs(v0 * 0.1) * 2.0**-22)
        for k in range(2, 12):
            x, v = oracle.stream_one(p, x, v)
        # ten steps: k * d exactly (mod P)
        xs = x0.copy()
        for k in range(11):
            xs, _ = oracle.stream_one(p, xs, v0)
        assert np.array_equal(xs, (x0.astype(np.int64) + 11 * d) % P)
        assert np.array_equal(v, v0)


def test_periodic_wrap():
    p = oracle.params(L=16, h=0.1)
    F = oracle.fixed_bits(p)
    x, v = oracle.stream_one(p, [int((16 - 0.01) * 2**F), 5, 7 * 2**F], [0.5, 0.0, -0.25])
    assert abs(x[0] / 2**F - 0.04) < 1e-6
    assert abs(x[2] / 2**F - (7 - 0.025)) < 1e-6


def test_bounce_back_closed_form():
    """No-slip wall (Sec. II, Boundary conditions): a particle that would cross z = 0
    during the step is reflected for the rest of the step and its velocity reversed."""
    p = oracle.params(L=(8, 8, 8), h=0.1, walls_z=1)
    F = oracle.fixed_bits(p)
    # lower wall: z = 0.05, v_z = -1 -> hits at t = h/2, comes back to z = 0.05;
    # lateral motion cancels (h/2 forward, h/2 back)
    x, v = oracle.stream_one(p, [3 * 2**F, 4 * 2**F, int(0.05 * 2**F)], [0.3, -0.2, -1.0])
    assert abs(x[2] / 2**F - 0.05) < 3 * 2.0**-F
    assert abs(x[0] / 2**F - 3) < 3 * 2.0**-F and abs(x[1] / 2**F - 4) < 3 * 2.0**-F
    np.testing.assert_array_equal(v, [-0.3, 0.2, 1.0])
    # upper wall: z = 7.98, v_z = 0.4 -> crosses at t = 0.05 (of 0.1), ends at 7.98;
    # lateral: forward 0.05 v, back 0.05 v -> 0
    x, v = oracle.stream_one(p, [2**F, 2**F, int(7.98 * 2**F)], [1.0, 0.5, 0.4])
    assert abs(x[2] / 2**F - 7.98) < 3 * 2.0**-F
    assert abs(x[0] / 2**F - 1.0) < 3 * 2.0**-F
    np.testing.assert_array_equal(v, [-1.0, -0.5, -0.4])
    # asymmetric: z = 0.02, v_z = -0.5: crosses after t = 0.04, travels back 0.06 -> z = 0.03,
    # lateral displacement v_x (0.04 - 0.06) = -0.02 v_x
    x, v = oracle.stream_one(p, [2 * 2**F, 2 * 2**F, int(0.02 * 2**F)], [1.0, 0.0, -0.5])
    assert abs(x[2] / 2**F - 0.03) < 3 * 2.0**-F
    assert abs(x[0] / 2**F - (2 - 0.02)) < 1e-6
    # no crossing: unchanged velocity
    x, v = oracle.stream_one(p, [2**F, 2**F, 2**F], [0.1, 0.2, 0.3])
    np.testing.assert_array_equal(v, [0.1, 0.2, 0.3])


def test_gravity_kick_then_drift():
    """External field (Sec. II): the velocity gains g h before the ballistic move."""
    p = oracle.params(L=8, h=0.1, g=(0.01, 0.0, 0.0))
    F = oracle.fixed_bits(p)
    x0 = [4 * 2**F, 4 * 2**F, 4 * 2**F]
    x, v = oracle.stream_one(p, x0, [0.0, 0.0, 0.0])
    assert abs(v[0] - np.float32(0.001)) < 1e-12
    assert abs((x[0] - x0[0]) / 2**F - 0.0001) < 2 * 2.0**-F


def test_nan_velocity_does_not_move_particle():
    p = oracle.params(L=8, h=0.1)
    F = oracle.fixed_bits(p)
    x, v = oracle.stream_one(p, [2**F, 2**F, 2**F], [np.nan, 0.0, 1e30])
    assert x[0] == 2**F  # NaN displacement contract: 0
    assert x[2] == (2**F + 8 * 2**F - 1) % (8 * 2**F)  # clamped to P - 1
