"""Shear viscosity of the GPU fluid from the decay of a transverse shear wave.

A velocity profile v_x = A sin(k z) (k = 2 pi / L) decays as exp(-nu k^2 t) with the
kinematic viscosity nu = eta / rho (rho = N_c m); the estimate is averaged over
independent boxes.  Checked against:
  * SRD (N_c 10, h 0.1, alpha 130 deg): within 2 % of the kinetic + collisional closed
    form of the transport theory the paper cites, eta = 8.700 (0.486 + 8.214), and of the
    oracle's own estimate from a Poiseuille profile between no-slip walls;
  * MPC-SRD+a (N_c 50, h 0.02, alpha 130 deg): within 2 % of the oracle's shear-wave
    estimate, and within 3 % of the value the paper prints for this parameter set in its
    squirmer showcase (Sec. V.B), eta = 111.3 sqrt(m kT)/a^2 (both implementations
    measure ~109);
plus Green-Kubo estimates of served and batched boxes against the SRD closed forms.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def eta_srd(n_c, h, alpha_deg):
    a = np.deg2rad(alpha_deg)
    z = n_c - 1 + np.exp(-n_c)
    kin = n_c * h * (5 * n_c / (z * (4 - 2 * np.cos(a) - 2 * np.cos(2 * a))) - 0.5)
    col = z * (1 - np.cos(a)) / (18 * h)
    return kin + col


def shear_wave_eta(variant, n_c, h, L, steps, samples, A=0.3, seed=11):
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    sim = mpc.Simulation(L=L, n_c=n_c, h=h, alpha_deg=130.0, variant=variant, seed=seed)
    sim.step(20)
    X, V, ids, step = sim.get_state()
    F = sim.info.fixed_bits
    k = 2 * np.pi / L
    z = X[2].astype(np.float64) / 2.0**F
    V[0] += (A * np.sin(k * z)).astype(np.float32)
    sim.set_state(X, V, ids, step)
    t, amp = [], []
    every = steps // samples
    for j in range(samples + 1):
        X, V, _, s = sim.get_state()
        z = X[2].astype(np.float64) / 2.0**F
        amp.append(2.0 * np.mean(V[0] * np.sin(k * z)))
        t.append((s - step) * h)
        if j < samples:
            sim.step(every)
    sim.close()
    t, amp = np.asarray(t), np.asarray(amp)
    rate = -np.polyfit(t, np.log(amp), 1)[0]
    return rate / k**2 * n_c  # eta = rho nu, rho = N_c m


def _mean_eta(variant, n_c, h, L, steps):
    vals = [shear_wave_eta(variant, n_c, h, L, steps, 20, seed=s) for s in (1, 2, 3, 4)]
    return float(np.mean(vals)), float(np.std(vals) / np.sqrt(len(vals)))


def test_srd_viscosity_matches_closed_form_and_oracle():
    from tests.test_oracle_physics import poiseuille_eta

    eta, err = _mean_eta(0, 10.0, 0.1, L=64, steps=2400)
    ref = eta_srd(10, 0.1, 130)
    eta_oracle = poiseuille_eta()[0]
    print(f"SRD shear-wave eta = {eta:.3f} +- {err:.3f}; closed form {ref:.3f}; "
          f"oracle (Poiseuille) {eta_oracle:.3f}")
    assert abs(eta - ref) / ref < 0.02
    assert abs(eta - eta_oracle) / eta_oracle < 0.02


def _oracle_shear_eta(args):
    """The same shear-wave estimate on the oracle (runs in a spawned process)."""
    import oracle

    variant, n_c, h, L, steps, samples, A, seed = args
    p = oracle.params(L=L, n_c=n_c, h=h, alpha_deg=130.0, variant=variant, seed=seed)
    X, V, ids = oracle.init(p)
    F = oracle.fixed_bits(p)
    for s in range(20):
        r = oracle.step(p, X, V, ids, s)
        X, V = r["X"], r["V"]
    k = 2 * np.pi / L
    V = V.copy()
    V[0] += (A * np.sin(k * X[2] / 2.0**F)).astype(np.float32).astype(np.float64)
    t, amp, s = [], [], 20
    for j in range(samples + 1):
        amp.append(2.0 * np.mean(V[0] * np.sin(k * X[2] / 2.0**F)))
        t.append((s - 20) * h)
        if j < samples:
            for _ in range(steps // samples):
                r = oracle.step(p, X, V, ids, s)
                X, V = r["X"], r["V"]
                s += 1
    return -np.polyfit(np.array(t), np.log(np.array(amp)), 1)[0] / k**2 * n_c


def test_srd_a_viscosity_matches_oracle_and_printed_value():
    """MPC-SRD+a, N_c 50, h 0.02: the GPU shear-wave viscosity agrees with the oracle's
    (same estimator, L = 16, independent seeds) within 2 %, and with the value the paper
    prints (111.3, the mean-field closed form) within 3 % at L = 48 -- both
    implementations measure ~109, 2 % below the closed form, a gap of the closed form at
    this density and time step, not of the kernel."""
    import multiprocessing as mp
    import os

    import oracle

    oracle.build()
    jobs = [(2, 50.0, 0.02, 16, 300, 20, 0.3, seed) for seed in range(1, 17)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        ref = np.array(pool.map(_oracle_shear_eta, jobs))
    gpu16 = np.array([shear_wave_eta(2, 50.0, 0.02, 16, 300, 20, seed=100 + s) for s in range(32)])
    eta, err = _mean_eta(2, 50.0, 0.02, L=48, steps=2600)
    print(f"SRD+a: oracle L=16 {ref.mean():.2f} +- {ref.std(ddof=1) / 4:.2f}; GPU L=16 "
          f"{gpu16.mean():.2f} +- {gpu16.std(ddof=1) / np.sqrt(32):.2f}; GPU L=48 {eta:.2f} +- "
          f"{err:.2f}; paper 111.3")
    assert abs(gpu16.mean() - ref.mean()) / ref.mean() < 0.02
    assert abs(eta - 111.3) / 111.3 < 0.03


def test_green_kubo_viscosity_of_served_boxes():
    """The per-job Green-Kubo viscosity the server reports (stress autocorrelation of the
    streaming + collision stress, the estimator used for batched and served viscosity
    jobs, window one time unit) agrees with the SRD closed form within three standard
    errors plus 2 %: eight independent L = 12 boxes, 20,000 steps each, N_c 10, h 0.1,
    alpha 130 deg."""
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    with mpc.Server(8 << 30, chunk_steps=100) as srv:
        ids = [srv.submit(steps=20000, L=12, n_c=10.0, h=0.1, alpha_deg=130.0, variant=0,
                          seed=300 + k) for k in range(8)]
        srv.run(timeout_s=600.0)
        etas = np.array([srv.job(i)["eta_gk"] for i in ids])
    mean, err = etas.mean(), etas.std(ddof=1) / np.sqrt(len(etas))
    ref = eta_srd(10, 0.1, 130)
    print(f"Green-Kubo eta {mean:.3f} +- {err:.3f} (closed form {ref:.3f}); boxes {etas}")
    assert abs(mean - ref) < 3 * err + 0.02 * ref


def _green_kubo(rows, vol, h, kT=1.0, m=1.0, K=None):
    """eta from the library's observables rows by the test-side estimator (tests/_gk.py,
    independent of the server's C++ copy); window one time unit unless K is given"""
    from tests._gk import green_kubo, stress_from_rows

    K = K if K is not None else max(1, int(round(1.0 / h)))
    return green_kubo(stress_from_rows(rows, vol, h, m), vol, h, kT, K=K)


def _golden_at_a():
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "at_a_viscosity.json")) as f:
        return json.load(f)


def test_at_a_green_kubo_viscosity_matches_oracle():
    """MPC-AT+a at the headline workload's physics (N_c 10, h 0.05, kT 1): the Green-Kubo
    viscosity of independent L = 10 GPU machines, stepped together in one batch, agrees with
    the oracle's by the same estimator (tests/golden/at_a_viscosity.json, written by
    tests/golden/make_at_a_viscosity.py from the oracle alone, other seeds) within 2 %,
    each side's standard error below 1 %.  The AT+a viscosity has no closed form in the
    paper: the oracle is the reference."""
    import torch

    import paper_2406_15236_gb300 as mpc
    from tests._gk import green_kubo, stress_from_rows

    torch.cuda.set_device(0)
    gold = _golden_at_a()
    P = gold["params"]
    steps, nbox = gold["steps"], 64
    vol = float(P["L"] ** 3)
    with mpc.Batch(graph_steps=100) as b:
        members = [b.add(L=P["L"], n_c=P["n_c"], h=P["h"], kT=P["kT"], variant=1, seed=40000 + k,
                         box_id=k, flags=mpc.MPC_FLAG_OBSERVABLES, obs_ring=steps)
                   for k in range(nbox)]
        b.step(steps)
        b.synchronize()
        etas = np.array([green_kubo(stress_from_rows(m.observable_series(steps), vol, P["h"]), vol,
                                    P["h"], P["kT"], K=gold["window_steps"],
                                    discard=gold["discard_steps"]) for m in members])
    mean, se = etas.mean(), etas.std(ddof=1) / np.sqrt(nbox)
    print(f"AT+a Green-Kubo eta: GPU {mean:.3f} +- {se:.3f} ({nbox} boxes); oracle "
          f"{gold['mean']:.3f} +- {gold['se']:.3f} ({gold['boxes']} boxes); ratio {mean / gold['mean']:.4f}")
    assert se < 0.01 * mean and gold["se"] < 0.01 * gold["mean"]
    assert abs(mean / gold["mean"] - 1.0) < 0.02


def test_batched_green_kubo_viscosity_against_closed_forms():
    """The batched ensemble's per-box viscosity: SRD boxes of different N_c, h and alpha and
    MPC-AT+a boxes (N_c 10, h 0.05), stepped together in one batch for 20,000 steps, each
    measured by Green-Kubo from its own stress series (window one time unit) and compared
    with the SRD closed form of its parameters, or for AT+a with the oracle's estimate
    (tests/golden/at_a_viscosity.json).  Each parameter set's mean lies within three
    standard errors (the boxes' own scatter) plus 2 % of its reference; all boxes together
    within 2 %."""
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    steps, reps = 20000, 3
    gold = _golden_at_a()
    groups = [dict(n_c=10.0, h=0.1, alpha_deg=130.0, variant=0),
              dict(n_c=10.0, h=0.05, alpha_deg=130.0, variant=0),
              dict(n_c=20.0, h=0.1, alpha_deg=130.0, variant=0),
              dict(n_c=5.0, h=0.1, alpha_deg=130.0, variant=0),
              dict(n_c=10.0, h=0.1, alpha_deg=90.0, variant=0),
              dict(n_c=20.0, h=0.05, alpha_deg=90.0, variant=0),
              dict(n_c=10.0, h=0.05, alpha_deg=130.0, variant=1)]
    boxes = []
    for k, gp in enumerate(groups):
        for rep in range(reps):
            boxes.append(dict(L=10, seed=700 + reps * k + rep, box_id=reps * k + rep, **gp))
    with mpc.Batch(graph_steps=100) as b:
        members = [b.add(flags=mpc.MPC_FLAG_OBSERVABLES, obs_ring=steps, **kw) for kw in boxes]
        b.step(steps)
        b.synchronize()
        ratios = []
        for kw, box in zip(boxes, members):
            eta = _green_kubo(box.observable_series(steps), 1000.0, kw["h"])
            ref = gold["mean"] if kw["variant"] == 1 else eta_srd(kw["n_c"], kw["h"], kw["alpha_deg"])
            ratios.append(eta / ref)
    ratios = np.array(ratios).reshape(len(groups), reps)
    mean = ratios.mean(axis=1)
    se = ratios.std(axis=1, ddof=1).mean() / np.sqrt(reps)  # pooled per-group standard error
    for gp, r in zip(groups, ratios):
        print(f"eta_GK / reference {gp}: {np.round(r, 3)}")
    print(f"per-group mean ratios {np.round(mean, 4)}; pooled standard error {se:.4f}; "
          f"all boxes {ratios.mean():.4f}")
    assert np.all(np.abs(mean - 1.0) < 3 * se + 0.02)
    assert abs(ratios.mean() - 1.0) < 0.02
