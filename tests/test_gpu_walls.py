"""Slip walls (specular reflection) and moving no-slip walls (bounce-back in the wall
frame, shear flow) on the GPU (Sec. II, Boundary conditions): per-step parity with the
oracle, crafted wall hits, exact energy conservation with slip walls, and the linear
Couette profile between walls moving in opposite directions."""
import numpy as np
import pytest

from tests import _parity as par

pytestmark = pytest.mark.gpu


def _mpc():
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    return mpc


CASES = {
    "slip": dict(L=(10, 8, 12), n_c=10.0, h=0.1, alpha_deg=130.0, walls_z=2, seed=51),
    "slip_mbs_gravity": dict(L=(8, 8, 10), n_c=7.0, h=0.1, alpha_deg=130.0, walls_z=2,
                             thermostat=1, gravity=(5e-3, 0.0, -2e-3), seed=52),
    "couette": dict(L=(8, 6, 10), n_c=10.0, h=0.1, alpha_deg=130.0, walls_z=1, thermostat=1,
                    wall_u=(-0.3, 0.3), seed=53),
    "moving_one_wall_gravity": dict(L=(6, 6, 9), n_c=12.0, h=0.05, alpha_deg=90.0, walls_z=1,
                                    wall_u=(0.0, 0.5), gravity=(0.0, 3e-3, 0.0), seed=54),
    # the angular-momentum-conserving variants: slip walls, and no-slip walls whose cut
    # cells hold phantom particles one by one (positions in the wall part)
    "at_a_slip": dict(L=(8, 8, 10), n_c=10.0, h=0.05, walls_z=2, variant=1, seed=55),
    "at_a_no_slip_moving_gravity": dict(L=(8, 6, 10), n_c=10.0, h=0.05, walls_z=1, variant=1,
                                        wall_u=(-0.3, 0.2), gravity=(4e-3, 0.0, 0.0), seed=56),
    "srd_a_no_slip": dict(L=(8, 8, 9), n_c=8.0, h=0.1, alpha_deg=120.0, walls_z=1, variant=2,
                          wall_u=(0.25, 0.0), seed=57),
    "at_a_no_slip_deterministic": dict(L=(6, 8, 8), n_c=6.0, h=0.05, walls_z=1, variant=1,
                                       wall_u=(0.1, -0.1), seed=58, det=True),
}


@pytest.mark.parametrize("name", list(CASES))
def test_walls_parity_every_step(name):
    import oracle

    mpc = _mpc()
    case = dict(CASES[name])
    det = case.pop("det", False)
    kw = dict(case, flags=mpc.MPC_FLAG_DEBUG_CELLS | (mpc.MPC_FLAG_DETERMINISTIC if det else 0))
    sim = mpc.Simulation(**kw)
    p = par.oracle_params(**kw)
    skip = oracle.FLAG_DEGENERATE | oracle.FLAG_MBS_NEAR_TIE | oracle.FLAG_POISSON_NEAR_TIE
    pre = sim.get_state()[:3]
    for s in range(12):
        sim.step(1)
        X1, V1, id1, step, cell1 = sim.get_state(cells=True)
        par.check_step(p, pre, (X1, V1, id1), s, post_cells=cell1, gpu_counts=sim.cell_counts(),
                       strict_flags=skip, kT=case.get("kT", 1.0))
        pre = (X1, V1, id1)
    sim.close()


@pytest.mark.parametrize("walls,wall_u,variant", [(2, (0.0, 0.0), 0), (1, (0.4, -0.25), 0),
                                                  (1, (0.4, -0.25), 1), (2, (0.0, 0.0), 2)])
def test_crafted_wall_hits(walls, wall_u, variant):
    """Every particle starts within one step of a wall, moving into it."""
    import oracle

    mpc = _mpc()
    kw = dict(L=(6, 6, 8), n_c=6.0, h=0.1, alpha_deg=130.0, walls_z=walls, wall_u=wall_u,
              variant=variant, seed=61, flags=mpc.MPC_FLAG_DEBUG_CELLS)
    sim = mpc.Simulation(**kw)
    X, V, ids, _ = sim.get_state()
    F = sim.info.fixed_bits
    rng = np.random.default_rng(3)
    N = X.shape[1]
    top = rng.random(N) < 0.5
    dist = rng.uniform(0.0, 0.09, N)
    X[2] = np.where(top, (8 - dist) * 2**F, dist * 2**F).astype(np.uint32)
    speed = rng.uniform(0.5, 3.0, N)
    V[2] = np.where(top, speed, -speed).astype(np.float32)
    sim.set_state(X, V, ids, 0)
    pre = sim.get_state()[:3]
    p = par.oracle_params(**kw)
    skip = oracle.FLAG_DEGENERATE | oracle.FLAG_MBS_NEAR_TIE | oracle.FLAG_POISSON_NEAR_TIE
    for s in range(3):
        sim.step(1)
        X1, V1, id1, step, cell1 = sim.get_state(cells=True)
        par.check_step(p, pre, (X1, V1, id1), s, post_cells=cell1, gpu_counts=sim.cell_counts(),
                       strict_flags=skip)
        pre = (X1, V1, id1)
    sim.close()


def test_slip_walls_conserve_energy():
    mpc = _mpc()
    sim = mpc.Simulation(L=(16, 16, 20), n_c=10.0, h=0.1, alpha_deg=130.0, walls_z=2, seed=5,
                         flags=mpc.MPC_FLAG_OBSERVABLES)
    e0 = sim.observables()["ekin"]
    sim.step(300)
    rows = sim.observable_series(300)
    e = 0.5 * rows[:, 3]
    assert np.abs(e / e0 - 1).max() < 2e-5  # float32 rounding only
    p = rows[:, 0:2]
    assert np.abs(p).max() < 1e-4 * np.sqrt(2 * e0)  # tangential momentum stays zero
    sim.close()


def test_couette_profile_is_linear():
    """Walls moving with -U/2 and +U/2 along x, MBS thermostat: v_x(z) = U (z/Lz - 1/2).

    The intercept is the box's mean x velocity, which fluctuates like the centre-of-mass
    velocity of N particles exchanging momentum with the walls: standard deviation
    sqrt(kT / (m N)) per snapshot, relaxing with the slowest shear mode's time
    Lz^2 / (pi^2 nu), nu = eta / (m N_c) with the SRD closed form eta = 8.700.  Its time
    average over T has variance sigma^2 (2 tau / T) (T >> tau); the bar is four of those
    standard errors, and at least 1 % of U.
    """
    mpc = _mpc()
    Lx, Lz, U, h, n_c = 48, 20, 0.4, 0.1, 10.0
    sim = mpc.Simulation(L=(Lx, Lx, Lz), n_c=n_c, h=h, alpha_deg=130.0, walls_z=1,
                         thermostat=1, wall_u=(-U / 2, U / 2), seed=77)
    sim.step(3000)
    F = sim.info.fixed_bits
    nb, snaps, every = 20, 80, 50
    prof, cnt = np.zeros(nb), np.zeros(nb)
    for _ in range(snaps):
        sim.step(every)
        X, V, _, _ = sim.get_state()
        b = np.minimum((X[2] / 2.0**F / Lz * nb).astype(int), nb - 1)
        np.add.at(prof, b, V[0])
        np.add.at(cnt, b, 1)
    N = sim.N
    sim.close()
    z = (np.arange(nb) + 0.5) * Lz / nb
    v = prof / cnt
    slope, icept = np.polyfit(z - Lz / 2, v, 1)
    tau = Lz**2 / (np.pi**2 * (8.700 / n_c))
    T = snaps * every * h
    se = np.sqrt(1.0 / N) * np.sqrt(2 * tau / T)
    print(f"Couette slope {slope:.5f} (U/Lz {U / Lz:.5f}), intercept {icept:.2e} (SE {se:.1e})")
    assert abs(slope - U / Lz) < 0.05 * U / Lz
    assert abs(icept) < max(4 * se, 0.01 * U)
    assert np.abs(v - (slope * (z - Lz / 2) + icept)).max() < 0.05 * U
