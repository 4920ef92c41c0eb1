"""GPU-vs-oracle parity of the MPC step through the C ABI (per-step, from identical
states): positions, collision cells and per-cell counts bit-exact; velocities within
1e-5 relative (|dv| / max(|v|, sqrt(kT/m))); conserved quantities to 1e-6.

Cases: the L=16 SRD box of 100 steps (every step compared), AT+a, SRD + MBS thermostat
with no-slip walls and gravity (phantom particles), ragged boxes (edge bricks cut,
non-integer N_c), sparse cells (n = 0, 1, 2), forced brick-capacity overflow and its
repair, multi-step graph replay, crafted edge states.
"""
import numpy as np
import pytest

import oracle
from tests import _parity as par

pytestmark = pytest.mark.gpu


def _mpc():
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    return mpc


def _sim(**kw):
    mpc = _mpc()
    kw.setdefault("flags", mpc.MPC_FLAG_DEBUG_CELLS)
    return mpc.Simulation(**kw)


def _run_parity(kw, steps, check_every=1, strict_flags=0xFF, log=None):
    sim = _sim(**kw)
    p = par.oracle_params(**kw)
    kT, m = kw.get("kT", 1.0), kw.get("m", 1.0)
    pre = sim.get_state()[:3]
    worst = 0.0
    for s in range(steps):
        sim.step(1)
        if s % check_every:
            pre = sim.get_state()[:3]
            continue
        X1, V1, id1, step, cell1 = sim.get_state(cells=True)
        assert step == s + 1
        counts = sim.cell_counts()
        st = par.check_step(p, pre, (X1, V1, id1), s, kT=kT, m=m, post_cells=cell1,
                            gpu_counts=counts, strict_flags=strict_flags)
        worst = max(worst, st["max_err"])
        if log is not None:
            log.append({k: v for k, v in st.items() if k != "ref"})
        pre = (X1, V1, id1)
    sim.close()
    return worst


def test_init_matches_oracle():
    kw = dict(L=16, n_c=10.0, h=0.1, alpha_deg=130.0, seed=1)
    sim = _sim(**kw)
    X, V, ids, step = sim.get_state()
    assert step == 0
    Xo, Vo, ido = oracle.init(par.oracle_params(**kw))
    X, V, ids = par.by_id(X, V, ids)
    np.testing.assert_array_equal(ids, ido)
    np.testing.assert_array_equal(X, Xo)
    np.testing.assert_allclose(V, Vo, rtol=0, atol=2e-6)
    assert np.abs(V.astype(np.float64).sum(axis=1)).max() < 1e-6 * np.abs(V).sum()
    sim.close()


def test_srd_l16_every_step_100_steps():
    """Plain SRD, L = 16, N_c = 10, h = 0.1, alpha = 130 deg, seed 1, 100 steps: each
    step compared with the oracle from the GPU state before it."""
    log = []
    worst = _run_parity(dict(L=16, n_c=10.0, h=0.1, alpha_deg=130.0, seed=1), 100, log=log)
    assert max(e["widened"] for e in log) == 0.0  # SRD: the 1e-5 bar everywhere
    mism = [e["cell_mismatch"] for e in log]
    print(f"max velocity error {worst:.3g}; cell mismatch fraction per step max {max(mism)}")
    assert worst <= par.VEL_TOL


def test_at_a_per_step():
    """MPC-AT+a, N_c 10, h 0.05: every particle within 1e-5 except in the cells the oracle
    flags ill-conditioned (cond(J) > 10), whose share is reported per step."""
    kw = dict(L=16, n_c=10.0, h=0.05, kT=1.0, variant=1, seed=3)
    log = []
    _run_parity(kw, 20, strict_flags=oracle.FLAG_DEGENERATE, log=log)
    ill = [e["ill_cells"] for e in log]
    print(f"AT+a: ill-conditioned cells per step {min(ill):.2e}..{max(ill):.2e}; particles above "
          f"1e-5 (all in them) {max(e['over_tol'] for e in log):.2e}; max error elsewhere "
          f"{max(e['max_err_strict'] for e in log):.3g}; largest error / (u sens) "
          f"{max(e['k_emp'] for e in log):.3g}")
    assert max(ill) < 1e-2


def _crafted_parity(kw, X, V, steps=1, log=None):
    sim = _sim(**kw)
    p = par.oracle_params(**kw)
    sim.set_state(X.astype(np.uint32), V.astype(np.float32), np.arange(sim.N, dtype=np.uint32), 0)
    pre = sim.get_state()[:3]
    for s in range(steps):
        sim.step(1)
        X1, V1, id1, step, cell1 = sim.get_state(cells=True)
        st = par.check_step(p, pre, (X1, V1, id1), s, post_cells=cell1, gpu_counts=sim.cell_counts(),
                            strict_flags=oracle.FLAG_DEGENERATE)
        if log is not None:
            log.append({k: v for k, v in st.items() if k != "ref"})
        pre = (X1, V1, id1)
    sim.close()


def test_at_a_per_step_drifting_frame():
    """The same box moving with 5 sigma along x (a uniform flow): the cell sums are taken
    about the cell centre, so the drift enters them; results stay within the bar."""
    kw = dict(L=16, n_c=10.0, h=0.05, kT=1.0, variant=1, seed=9)
    p = par.oracle_params(**kw)
    X, V, _ = oracle.init(p)
    V = V.copy()
    V[0] += 5.0
    log = []
    _crafted_parity(kw, X, V, steps=5, log=log)
    print(f"AT+a drifting: max error outside ill-conditioned cells "
          f"{max(e['max_err_strict'] for e in log):.3g}; ill-conditioned cells "
          f"{max(e['ill_cells'] for e in log):.2e}; largest error / (u sens) "
          f"{max(e['k_emp'] for e in log):.3g}")


def test_at_a_tight_clusters_take_the_second_pass():
    """Members packed within 0.002 of a point away from the cell centre: the raw sums about
    the centre cancel there, and such cells take their moments in a second pass about
    the centre of mass.  The oracle flags these cells ill-conditioned (a cluster that
    tight is resolved by float32 positions only to ~100 ulps); the second pass keeps
    their errors well inside the 4 u sens_i bar (below u sens_i), where the raw sums
    would exceed it.
    Clusters of 2, 3 and 6 particles at rest, in a fluid of moving particles."""
    kw = dict(L=8, n_c=4.0, h=0.05, kT=1.0, variant=1, seed=10)
    p = par.oracle_params(**kw)
    X, V, _ = oracle.init(p)
    X, V = X.astype(np.int64), V.copy()
    F = oracle.fixed_bits(p)
    P = 8 << F
    S = oracle.shift(p, 0).astype(np.int64)
    rng = np.random.default_rng(12)
    cells = rng.choice(512, size=60, replace=False)
    k = 0
    for j, c in enumerate(cells):
        size = (2, 3, 6)[j % 3]
        corner = np.array([c % 8, (c // 8) % 8, c // 64])
        centre = corner + 0.5 + rng.uniform(-0.35, 0.35, 3)
        for _ in range(size):
            pos = centre + rng.uniform(-0.002, 0.002, 3)
            # the collision sees X + S: place the particle there, at rest (no streaming)
            X[:, k] = (np.round(pos * 2.0**F).astype(np.int64) - S) % P
            V[:, k] = 0.0
            k += 1
    # the rest of the fluid leaves the clusters' cells (the cells it streams into, as the
    # oracle finds them), one cell along x at a time
    chosen = np.zeros(512, dtype=bool)
    chosen[cells] = True
    ids = np.arange(X.shape[1], dtype=np.uint32)
    for _ in range(16):
        cell = oracle.step(p, X.astype(np.uint32), V, ids, 0, cells=True)["cell"]
        inside = chosen[cell]
        inside[:k] = False
        if not inside.any():
            break
        X[0][inside] = (X[0][inside] + (1 << F)) % P
    assert not inside.any()
    log = []
    _crafted_parity(kw, X, V, steps=1, log=log)
    print(f"AT+a tight clusters: ill-conditioned cells {log[0]['ill_cells']:.3f}; largest "
          f"error / (u sens) there {log[0]['k_emp_ill']:.3g}")
    assert log[0]["ill_cells"] > 0.05 and log[0]["k_emp_ill"] < 1.0


def test_srd_a_per_step():
    """MPC-SRD+a, Eqs. (3)-(4): rotation plus the angular-momentum restoring term."""
    kw = dict(L=16, n_c=10.0, h=0.1, alpha_deg=130.0, variant=2, seed=4)
    log = []
    _run_parity(kw, 12, strict_flags=oracle.FLAG_DEGENERATE, log=log)
    print(f"SRD+a: ill-conditioned cells per step up to {max(e['ill_cells'] for e in log):.2e}; "
          f"max error elsewhere {max(e['max_err_strict'] for e in log):.3g}")


def test_srd_mbs_walls_gravity_per_step():
    kw = dict(L=16, n_c=10.0, h=0.1, alpha_deg=130.0, thermostat=1, walls_z=1,
              gravity=(0.02, 0.0, 0.0), seed=2)
    log = []
    worst = _run_parity(kw, 30, strict_flags=oracle.FLAG_MBS_NEAR_TIE | oracle.FLAG_POISSON_NEAR_TIE,
                        log=log)
    assert worst <= par.VEL_TOL


@pytest.mark.parametrize("variant,h", [(0, 0.1), (1, 0.05), (2, 0.1)])
def test_ragged_box(variant, h):
    kw = dict(L=(12, 10, 7), n_c=3.7, h=h, alpha_deg=90.0, variant=variant, seed=11)
    _run_parity(kw, 6, strict_flags=oracle.FLAG_DEGENERATE)


@pytest.mark.parametrize("variant,h", [(0, 1.0), (1, 0.5)])
def test_ragged_box_default_bricks(variant, h):
    """N_c = 10 takes the compiled-in 4x4x4-cell bricks; 21 and 13 cells leave a last brick
    one cell wide, so a particle that streams a cell and a half past the brick before it
    wraps to cell 0 (the brick-delta shortcut of interior bricks must not apply there).
    Large time steps make such moves common."""
    kw = dict(L=(21, 18, 13), n_c=10.0, h=h, alpha_deg=130.0, variant=variant, seed=14)
    _run_parity(kw, 5, strict_flags=oracle.FLAG_DEGENERATE)


def test_sparse_cells_at_a():
    """N_c = 1.5: many cells hold 0, 1 or 2 particles (pair pseudo-inverse branch)."""
    kw = dict(L=10, n_c=1.5, h=0.05, variant=1, seed=12)
    _run_parity(kw, 6, strict_flags=oracle.FLAG_DEGENERATE)


def test_walls_ragged_and_thermostat_small_cells():
    kw = dict(L=(6, 9, 5), n_c=2.5, h=0.1, alpha_deg=130.0, thermostat=1, walls_z=1,
              gravity=(0.0, 0.05, 0.0), seed=13)
    _run_parity(kw, 8, strict_flags=oracle.FLAG_MBS_NEAR_TIE | oracle.FLAG_POISSON_NEAR_TIE)


def test_capacity_overflow_is_repaired():
    """A brick capacity just above the initial maximum overflows within a few steps; the
    chain stops at a consistent step, the handle rebins with a larger capacity and runs
    the remaining steps -- results still match the oracle every step."""
    mpc = _mpc()
    kw = dict(L=16, n_c=10.0, h=0.1, alpha_deg=130.0, seed=5, capacity=4)
    sim = _sim(**kw)
    cap0 = sim.info.capacity
    p = par.oracle_params(**kw)
    pre = sim.get_state()[:3]
    for s in range(12):
        sim.step(1)
        X1, V1, id1, step, cell1 = sim.get_state(cells=True)
        par.check_step(p, pre, (X1, V1, id1), s, post_cells=cell1, gpu_counts=sim.cell_counts())
        pre = (X1, V1, id1)
    info = mpc.mpc_get_info(sim.handle)
    assert info.recoveries > 0 and info.capacity > cap0
    sim.close()


def test_graph_replay_keeps_step_and_parity():
    """40 steps in one call (16-step graphs + single launches), then a checked step."""
    kw = dict(L=16, n_c=10.0, h=0.1, alpha_deg=130.0, seed=6, graph_steps=16)
    sim = _sim(**kw)
    sim.step(40)
    X0, V0, id0, step = sim.get_state()
    assert step == 40
    sim.step(1)
    X1, V1, id1, step, cell1 = sim.get_state(cells=True)
    par.check_step(par.oracle_params(**kw), (X0, V0, id0), (X1, V1, id1), 40, post_cells=cell1,
                   gpu_counts=sim.cell_counts())
    sim.close()


def test_observables_and_conservation():
    mpc = _mpc()
    kw = dict(L=12, n_c=10.0, h=0.1, alpha_deg=130.0, seed=8,
              flags=mpc.MPC_FLAG_OBSERVABLES | mpc.MPC_FLAG_DEBUG_CELLS)
    sim = _sim(**kw)
    p = par.oracle_params(**kw)
    e0 = sim.observables()["ekin"]
    for s in range(10):
        X0, V0, id0, _ = sim.get_state()
        sim.step(1)
        o = sim.observables()
        X1, V1, id1, _ = sim.get_state()
        ref = par.check_step(p, (X0, V0, id0), (X1, V1, id1), s)["ref"]["obs"]
        scale = np.abs(V1.astype(np.float64)).sum()
        assert np.abs(o["momentum"]).max() <= 1e-6 * scale
        assert abs(o["ekin"] - e0) <= 1e-6 * e0  # SRD without thermostat conserves energy
        assert abs(o["ekin"] - ref["ekin"]) <= 1e-6 * ref["ekin"]
        assert o["has_stress"]
        np.testing.assert_allclose(o["stress_kin"], [ref["skin_xy"], ref["skin_yz"], ref["skin_zx"]],
                                   rtol=1e-4, atol=1e-6)
        col = [ref[k] for k in ("scol_xy", "scol_yx", "scol_yz", "scol_zy", "scol_zx", "scol_xz")]
        np.testing.assert_allclose(o["stress_col"], col, rtol=1e-4, atol=1e-5)
    rows = sim.observable_series(10)
    assert rows.shape == (10, 16)
    np.testing.assert_array_equal(rows[:, 13], np.arange(1, 11))
    sim.close()


def test_crafted_edge_states():
    """Particles on lattice planes and on the walls, velocities that cross a wall exactly
    at the end of the step, a huge velocity that hits the displacement clamp."""
    kw = dict(L=(8, 8, 8), n_c=2.0, h=0.1, alpha_deg=130.0, walls_z=1, thermostat=1, seed=21)
    sim = _sim(**kw)
    p = par.oracle_params(**kw)
    F = oracle.fixed_bits(p)
    P = 8 << F
    N = sim.N
    rng = np.random.default_rng(4)
    X = rng.integers(0, P, size=(3, N), dtype=np.int64)
    V = rng.normal(size=(3, N)).astype(np.float32)
    S = oracle.shift(p, 0).astype(np.int64)
    k = N // 8
    X[0, :k] = (rng.integers(0, 8, size=k) * (1 << F) - S[0]) % P      # on x lattice planes
    X[2, k:2 * k] = 0                                                   # on the lower wall
    X[2, 2 * k:3 * k] = P - 1                                           # just under the upper wall
    V[2, k:2 * k] = -np.abs(V[2, k:2 * k]) - 0.1
    V[2, 2 * k:3 * k] = np.abs(V[2, 2 * k:3 * k]) + 0.1
    V[0, 3 * k] = 1e6                                                   # displacement clamp
    ids = np.arange(N, dtype=np.uint32)
    X = X.astype(np.uint32)
    sim.set_state(X, V, ids, 0)
    pre = sim.get_state()[:3]
    sim.step(1)
    X1, V1, id1, step, cell1 = sim.get_state(cells=True)
    par.check_step(p, pre, (X1, V1, id1), 0, post_cells=cell1, gpu_counts=sim.cell_counts(),
                   strict_flags=oracle.FLAG_MBS_NEAR_TIE | oracle.FLAG_POISSON_NEAR_TIE)
    sim.close()


def test_invalid_inputs_are_rejected():
    mpc = _mpc()
    sim = _sim(L=8, n_c=2.0, seed=1)
    X, V, ids, _ = sim.get_state()
    p = par.oracle_params(L=8)
    X[0, 5] = 8 << oracle.fixed_bits(p)  # outside [0, L << F)
    with pytest.raises(mpc.MpcError) as e:
        sim.set_state(X, V, ids, 3)
    assert e.value.status == mpc.MPC_EINVAL
    # the handle is still usable afterwards
    X[0, 5] = 0
    sim.set_state(X, V, ids, 3)
    sim.step(2)
    assert sim.get_state()[3] == 5
    with pytest.raises(mpc.MpcError):
        mpc.mpc_step(sim.handle, -1)
    sim.close()
