"""Green-Kubo shear viscosity from a series of off-diagonal stresses (test-side analysis,
shared by the GPU tests and the scripts that write stored oracle values; holds none of
the MPC arithmetic).

eta = (V h / kT) [C(0)/2 + sum_{k=1..K} C(k)], C the autocorrelation of each off-diagonal
stress about its mean, averaged over sigma_xy, sigma_yx, sigma_yz, sigma_zy, sigma_zx,
sigma_xz (the Green-Kubo relation for the MPC stress of the transport theory the paper
cites; the discrete time step gives the trapezoidal C(0)/2).
"""
import numpy as np


def green_kubo(stress, vol, h, kT=1.0, K=20, discard=200):
    """stress: (steps, 6) off-diagonal stresses, one row per step"""
    s = np.asarray(stress, dtype=np.float64)[discard:]
    acc = 0.0
    for c in range(s.shape[1]):
        x = s[:, c] - s[:, c].mean()
        n = len(x)
        f = np.fft.rfft(x, 2 * n)
        ac = np.fft.irfft(f * np.conj(f))[: K + 1] / (n - np.arange(K + 1))
        acc += 0.5 * ac[0] + ac[1:].sum()
    return vol * h / kT * acc / s.shape[1]


def stress_from_oracle_obs(obs):
    """the six off-diagonal stresses from an oracle observables dict"""
    return [obs["skin_xy"] + obs["scol_xy"], obs["skin_xy"] + obs["scol_yx"],
            obs["skin_yz"] + obs["scol_yz"], obs["skin_yz"] + obs["scol_zy"],
            obs["skin_zx"] + obs["scol_zx"], obs["skin_zx"] + obs["scol_xz"]]


def stress_from_rows(rows, vol, h, m=1.0):
    """the six off-diagonal stresses from the library's per-step observables rows (raw
    sums: kinetic xy, yz, zx in columns 4-6, collisional xy, yx, yz, zy, zx, xz in 7-12)"""
    rows = np.asarray(rows, dtype=np.float64)
    kin = {0: 4, 1: 4, 2: 5, 3: 5, 4: 6, 5: 6}
    return np.stack([-(m / vol) * (rows[:, kin[c]] + rows[:, 7 + c] / h) for c in range(6)], axis=1)
