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
    jobs) agrees with the SRD closed form: eight independent L = 12 boxes, 20,000 steps
    each, N_c 10, h 0.1, alpha 130 deg."""
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
    assert abs(mean - ref) < max(3 * err, 0.02 * ref) + 0.03 * ref


def _green_kubo(rows, vol, h, kT=1.0, m=1.0, K=50):
    """eta = (V h / kT)[C(0)/2 + sum_k C(k)] over the six off-diagonal stresses (test-side
    restatement of the estimator; independent of the server's C++ copy)."""
    kin = {0: 4, 1: 4, 2: 5, 3: 5, 4: 6, 5: 6}
    col = {0: 7, 1: 8, 2: 9, 3: 10, 4: 11, 5: 12}
    acc = 0.0
    for c in range(6):
        s = -(m / vol) * (rows[:, kin[c]] + rows[:, col[c]] / h)
        s = s - s.mean()
        n = len(s)
        f = np.fft.rfft(s, 2 * n)
        ac = np.fft.irfft(f * np.conj(f))[: K + 1] / (n - np.arange(K + 1))
        acc += 0.5 * ac[0] + ac[1:].sum()
    return vol * h / kT * acc / 6.0


def test_batched_green_kubo_viscosity_against_closed_forms():
    """The batched ensemble's per-box viscosity: SRD boxes of different N_c, h and alpha,
    stepped together in one batch for 20,000 steps, each measured by Green-Kubo from its
    own stress series and compared with the SRD closed form of its parameters."""
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    steps = 20000
    boxes = []
    for k, (n_c, h, alpha) in enumerate([(10.0, 0.1, 130.0), (10.0, 0.05, 130.0),
                                         (20.0, 0.1, 130.0), (5.0, 0.1, 130.0),
                                         (10.0, 0.1, 90.0), (20.0, 0.05, 90.0)]):
        for rep in range(2):
            boxes.append(dict(L=10, n_c=n_c, h=h, alpha_deg=alpha, variant=0,
                              seed=700 + 2 * k + rep, box_id=2 * k + rep))
    with mpc.Batch(graph_steps=100) as b:
        members = [b.add(flags=mpc.MPC_FLAG_OBSERVABLES, obs_ring=steps, **kw) for kw in boxes]
        b.step(steps)
        b.synchronize()
        ratios = []
        for kw, box in zip(boxes, members):
            rows = box.observable_series(steps)
            eta = _green_kubo(rows, 1000.0, kw["h"])
            ratios.append(eta / eta_srd(kw["n_c"], kw["h"], kw["alpha_deg"]))
    ratios = np.array(ratios)
    per_param = ratios.reshape(-1, 2).mean(axis=1)
    print("eta_GK / eta_closed per box:", np.round(ratios, 3))
    # molecular-chaos closed forms run a few per cent high at these h; 20,000 steps give
    # ~3 % noise per box
    assert abs(ratios.mean() - 1.0) < 0.04
    assert np.all(np.abs(per_param - 1.0) < 0.10)
