"""The continuous-batching server through the C ABI.

Jobs arrive over time, are admitted while their device footprint fits the HBM budget,
run together as members of one batch and are retired at their own step counts.  In
deterministic mode (fixed-point sums) each job's per-step observables and final state
are checked to be the same bit for bit alone, in the mix, and on the sequential plain
path; admission waits for memory and refuses a job that cannot fit at all.
"""
import numpy as np
import pytest

from tests import _parity as par

pytestmark = pytest.mark.gpu

TRACE = [
    dict(L=8, n_c=10.0, h=0.1, alpha_deg=130.0, variant=0, seed=11, steps=300, arrival_s=0.0),
    dict(L=(12, 8, 10), n_c=5.0, h=0.05, variant=1, seed=12, steps=500, arrival_s=0.0),
    dict(L=10, n_c=20.0, h=0.02, alpha_deg=90.0, variant=0, seed=13, steps=200, arrival_s=0.001),
    dict(L=16, n_c=10.0, h=0.1, alpha_deg=130.0, variant=2, seed=14, steps=400, arrival_s=0.002),
    dict(L=12, n_c=10.0, h=0.1, alpha_deg=130.0, variant=0, thermostat=1, walls_z=1,
         gravity=(1e-3, 0.0, 0.0), seed=15, steps=250, arrival_s=0.002),
    dict(L=8, n_c=10.0, h=0.05, variant=1, seed=16, steps=700, arrival_s=0.003),
]


def _mpc():
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    return mpc


def _box_kw(job):
    return {k: v for k, v in job.items() if k not in ("steps", "arrival_s")}


def _peak(mpc, job):
    p = mpc.make_params(flags=mpc.MPC_FLAG_OBSERVABLES, obs_ring=job["steps"], **_box_kw(job))
    return mpc.mpc_footprint(p)


def _run(mpc, jobs, budget, **kw):
    with mpc.Server(budget, chunk_steps=64, **kw) as srv:
        ids = [srv.submit(keep_series=True, keep_state=True, **j) for j in jobs]
        srv.run(timeout_s=120.0)
        out = []
        for i in ids:
            r = srv.job(i)
            X, V, idv = srv.state(i) if r["status"] == mpc.MPC_JOB_DONE else (None, None, None)
            out.append((r, srv.series(i) if r["status"] == mpc.MPC_JOB_DONE else None,
                        par.by_id(X, V, idv) if X is not None else None))
        return out


@pytest.mark.parametrize("policy", [{}, {"share_all": True}, {"first_come": True},
                                    {"fill_kparticles": 1}, {"aged": True, "backfill": True},
                                    {"priority_head": True}, {"priority_head": True, "aged": True}])
def test_each_job_same_alone_and_in_the_mix(policy):
    mpc = _mpc()
    peaks = [_peak(mpc, j)[1] for j in TRACE]
    budget = int(2.2 * max(peaks))  # two or three jobs resident at a time
    mixed = _run(mpc, TRACE, budget, deterministic=True, **policy)
    for (r, series, state), job in zip(mixed, TRACE):
        assert r["status"] == mpc.MPC_JOB_DONE, r
        assert r["steps"] == job["steps"] and series.shape == (job["steps"], 16)
        assert np.array_equal(series[:, 13], np.arange(1, job["steps"] + 1))  # step column
        assert r["admit_s"] >= r["arrival_s"] and r["finish_s"] > r["admit_s"]
        assert 0.5 < r["temperature"] < 1.5
    for job, (r_mix, s_mix, st_mix) in zip(TRACE, mixed):
        (r_one, s_one, st_one), = _run(mpc, [dict(job, arrival_s=0.0)], budget, deterministic=True)
        assert np.array_equal(s_one, s_mix), f"observables differ alone vs mixed: {job}"
        for a, b in zip(st_one, st_mix):
            assert np.array_equal(a, b), f"final state differs alone vs mixed: {job}"
        assert r_one["eta_gk"] == r_mix["eta_gk"]


@pytest.mark.parametrize("policy", [{}, {"aged": True}, {"share_all": True},
                                    {"priority_head": True}])
def test_each_job_same_alone_and_in_the_mix_float_mode(policy):
    """Float mode (the default: float cell sums, whose order depends on the other boxes of a
    launch): one step of every job of the trace, alone and in the mix, gives bit-identical
    positions and velocities within the per-step bar of 1e-5 of each other (outside the
    cells the oracle flags ill-conditioned); both runs also pass the oracle's per-step
    check from the job's initial state."""
    import oracle

    mpc = _mpc()
    jobs = [dict(j, steps=1, arrival_s=0.0) for j in TRACE]
    budget = 8 << 30
    mixed = _run(mpc, jobs, budget, **policy)
    skip = oracle.FLAG_DEGENERATE | oracle.FLAG_MBS_NEAR_TIE | oracle.FLAG_POISSON_NEAR_TIE
    worst = 0.0
    for job, (r_mix, _, st_mix) in zip(jobs, mixed):
        assert r_mix["status"] == mpc.MPC_JOB_DONE, r_mix
        (r_one, _, st_one), = _run(mpc, [job], budget)
        X1, V1, id1 = st_one
        X2, V2, id2 = st_mix
        assert np.array_equal(id1, id2) and np.array_equal(X1, X2), f"positions differ: {job}"
        sim = mpc.Simulation(**_box_kw(job))
        pre = sim.get_state()[:3]
        sim.close()
        p = par.oracle_params(**_box_kw(job))
        ref = par.check_step(p, pre, st_one, 0, strict_flags=skip)["ref"]
        par.check_step(p, pre, st_mix, 0, strict_flags=skip)
        loose = (ref["flags"][ref["cell"]] & (skip | oracle.FLAG_ILL_CONDITIONED)) != 0
        scale = np.maximum(np.linalg.norm(V1.astype(np.float64), axis=0), 1.0)
        d = np.linalg.norm(V1.astype(np.float64) - V2, axis=0) / scale
        worst = max(worst, float(d[~loose].max()))
        assert d[~loose].max() <= par.VEL_TOL, f"velocities differ alone vs mixed: {job}"
    print(f"float mode, alone vs mixed, one step: positions bit-identical, largest velocity "
          f"difference {worst:.3g}")


def test_admission_waits_for_memory():
    """With room for one job at a time, each job is admitted only after the previous one
    has been retired, and all finish."""
    mpc = _mpc()
    job = dict(L=16, n_c=10.0, h=0.1, alpha_deg=130.0, variant=0, steps=200, arrival_s=0.0)
    budget = int(1.5 * _peak(mpc, job)[1])
    with mpc.Server(budget, chunk_steps=50) as srv:
        ids = [srv.submit(**dict(job, seed=40 + k)) for k in range(4)]
        srv.run(timeout_s=60.0)
        res = [srv.job(i) for i in ids]
    assert all(r["status"] == mpc.MPC_JOB_DONE for r in res)
    order = sorted(res, key=lambda r: r["admit_s"])
    for prev, nxt in zip(order, order[1:]):
        assert nxt["admit_s"] > prev["admit_s"]
        assert nxt["admit_s"] >= prev["finish_s"] - 0.05  # retired (results pending) first


def test_sequential_plain_path_gives_the_same_results():
    mpc = _mpc()
    peaks = [_peak(mpc, j)[1] for j in TRACE]
    served = _run(mpc, TRACE, int(4 * max(peaks)), deterministic=True)
    plain = _run(mpc, TRACE, int(4 * max(peaks)), deterministic=True, sequential=True)
    for (r1, s1, st1), (r2, s2, st2) in zip(served, plain):
        assert r2["status"] == mpc.MPC_JOB_DONE
        assert np.array_equal(s1, s2)
        for a, b in zip(st1, st2):
            assert np.array_equal(a, b)


def test_job_that_cannot_fit_fails_and_others_finish():
    mpc = _mpc()
    small = [dict(TRACE[0]), dict(TRACE[2])]
    big = dict(L=40, n_c=10.0, h=0.1, variant=0, seed=5, steps=10, arrival_s=0.0)
    budget = int(1.5 * max(_peak(mpc, j)[1] for j in small))
    assert _peak(mpc, big)[1] > budget
    with mpc.Server(budget, chunk_steps=32) as srv:
        ids = [srv.submit(**small[0]), srv.submit(**big), srv.submit(**small[1])]
        srv.run(timeout_s=60.0)
        res = [srv.job(i) for i in ids]
    assert res[1]["status"] == mpc.MPC_JOB_FAILED and res[1]["error"] == mpc.MPC_ENOMEM
    assert res[0]["status"] == mpc.MPC_JOB_DONE and res[2]["status"] == mpc.MPC_JOB_DONE


def test_served_job_matches_oracle_step():
    """A served job's last step matches the oracle from its state one step earlier (the
    server stops the box exactly at its step count; deterministic mode makes the two
    server runs and the replay follow one trajectory)."""
    mpc = _mpc()
    job = dict(L=(10, 8, 12), n_c=10.0, h=0.1, alpha_deg=130.0, variant=0, seed=21)
    budget = 4 * _peak(mpc, dict(job, steps=40, arrival_s=0.0))[1]
    res = {}
    for steps in (39, 40):
        with mpc.Server(budget, chunk_steps=16, deterministic=True) as srv:
            jid = srv.submit(steps=steps, keep_state=True, **job)
            srv.run(timeout_s=60.0)
            assert srv.job(jid)["steps"] == steps
            res[steps] = srv.state(jid)
    # replay the 40th step from the 39-step state on a plain box and compare with the oracle
    sim = mpc.Simulation(flags=mpc.MPC_FLAG_DETERMINISTIC, **job)
    X, V, ids = res[39]
    sim.set_state(X, V, ids, 39)
    sim.step(1)
    X1, V1, id1, step = sim.get_state()
    sim.close()
    par.check_step(par.oracle_params(**job), (X, V, ids), (X1, V1, id1), 39)
    Xs, Vs, ids_s = par.by_id(*res[40])
    Xp, Vp, ids_p = par.by_id(X1, V1, id1)
    assert np.array_equal(Xs, Xp) and np.array_equal(Vs, Vp)
