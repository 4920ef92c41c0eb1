"""Batched stepping and the deterministic (fixed-point) mode through the C ABI.

A batch advances many independent boxes (uneven L, n_c, variant, alpha, h, seeds) with
one persistent launch of the fused step per time step.  Checked here:
  - every member's step matches the oracle (same bar as the single-box parity tests);
  - deterministic mode (Sec. III.B, "Reproducibility": fixed-point summation) matches
    the oracle, and its trajectories are bit-identical whatever the brick tiling, the
    threads per cell, the kernel (single box or batch) or the other boxes in the batch;
  - per-box step limits stop each box at its own step;
  - arena admission refuses boxes that do not fit and reuses released memory;
  - brick-capacity overflow inside a batch is repaired without changing the result;
  - the autotuner returns one of its candidates.
"""
import numpy as np
import pytest

from tests import _parity as par

pytestmark = pytest.mark.gpu

MIX = [
    dict(L=(12, 12, 12), n_c=5.0, h=0.1, alpha_deg=90.0, variant=0, seed=1001),
    dict(L=(16, 8, 12), n_c=10.0, h=0.05, variant=1, seed=1002),
    dict(L=(8, 8, 8), n_c=20.0, h=0.02, alpha_deg=130.0, variant=0, seed=1003),
    dict(L=(20, 12, 16), n_c=10.0, h=0.1, alpha_deg=130.0, variant=2, seed=1004),
    dict(L=(10, 10, 10), n_c=7.5, h=0.1, alpha_deg=130.0, variant=0, thermostat=1, walls_z=1,
         gravity=(1e-3, 0.0, 0.0), seed=1005),
]


def _mpc():
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    return mpc


def _state(box):
    X, V, ids, step = box.get_state()
    return par.by_id(X, V, ids) + (step,)


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_batch_members_match_oracle_every_step():
    mpc = _mpc()
    with mpc.Batch(graph_steps=4) as b:
        boxes = [b.add(**kw) for kw in MIX]
        for s in range(3):
            pre = [bx.get_state()[:3] for bx in boxes]
            b.step(1)
            for kw, bx, p0 in zip(MIX, boxes, pre):
                X1, V1, id1, step = bx.get_state()
                assert step == s + 1
                par.check_step(par.oracle_params(**kw), p0, (X1, V1, id1), s)
        # graph replay (4-step graphs + single launches), then one checked step
        b.step(9)
        pre = [bx.get_state()[:3] for bx in boxes]
        b.step(1)
        for kw, bx, p0 in zip(MIX, boxes, pre):
            X1, V1, id1, step = bx.get_state()
            assert step == 13
            par.check_step(par.oracle_params(**kw), p0, (X1, V1, id1), 12)


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_deterministic_mode_matches_oracle(variant):
    mpc = _mpc()
    kw = dict(L=(12, 10, 8), n_c=10.0, h=0.1, alpha_deg=130.0, variant=variant, seed=77,
              flags=mpc.MPC_FLAG_DETERMINISTIC | mpc.MPC_FLAG_DEBUG_CELLS)
    if variant == 0:
        kw.update(thermostat=1, walls_z=1, gravity=(2e-3, 0.0, 0.0))
    sim = mpc.Simulation(**kw)
    p = par.oracle_params(**kw)
    pre = sim.get_state()[:3]
    for s in range(4):
        sim.step(1)
        X1, V1, id1, step, cell1 = sim.get_state(cells=True)
        par.check_step(p, pre, (X1, V1, id1), s, post_cells=cell1, gpu_counts=sim.cell_counts())
        pre = (X1, V1, id1)
    sim.close()


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_deterministic_trajectory_independent_of_tiling(variant):
    """Fixed-point sums make the trajectory a function of the physics alone: three brick
    tilings / thread splits give bit-identical states and observables after 40 steps,
    while the floating-point mode is allowed to differ."""
    mpc = _mpc()
    flags = mpc.MPC_FLAG_DETERMINISTIC | mpc.MPC_FLAG_OBSERVABLES
    kw = dict(L=(16, 12, 20), n_c=10.0, h=0.1, alpha_deg=130.0, variant=variant, seed=91,
              flags=flags)
    results = []
    for tile, tpc in ((320, 1), (640, 0), (1280, 8)):
        sim = mpc.Simulation(tile_particles=tile, threads_per_cell=tpc, **kw)
        sim.step(40)
        results.append((_state(sim), sim.observable_series(40), tuple(sim.info.brick),
                        sim.info.threads_per_cell))
        sim.close()
    assert len({r[2] for r in results}) == 3  # the tilings really differ
    for r in results[1:]:
        assert _same(r[0], results[0][0])
        assert np.array_equal(r[1], results[0][1])


def test_deterministic_alone_equals_mixed_and_single_box():
    """Each box's trajectory and observables are the same alone in a batch, mixed with
    the others, and stepped by the single-box kernel: bit for bit."""
    mpc = _mpc()
    flags = mpc.MPC_FLAG_OBSERVABLES
    steps = 60
    mixed = {}
    with mpc.Batch(deterministic=True, graph_steps=16) as b:
        boxes = [b.add(flags=flags, **kw) for kw in MIX]
        b.step(steps)
        for k, bx in enumerate(boxes):
            mixed[k] = (_state(bx), bx.observable_series(steps))
    for k, kw in enumerate(MIX):
        with mpc.Batch(deterministic=True, graph_steps=16) as b:
            bx = b.add(flags=flags, **kw)
            b.step(steps)
            alone = (_state(bx), bx.observable_series(steps))
        assert _same(alone[0], mixed[k][0]), f"box {k}: state differs alone vs mixed"
        assert np.array_equal(alone[1], mixed[k][1]), f"box {k}: observables differ"
        sim = mpc.Simulation(flags=flags | mpc.MPC_FLAG_DETERMINISTIC, **kw)
        sim.step(steps)
        single = (_state(sim), sim.observable_series(steps))
        sim.close()
        assert _same(single[0], mixed[k][0]), f"box {k}: single-box kernel differs"
        assert np.array_equal(single[1], mixed[k][1])


def test_step_limits_stop_each_box():
    mpc = _mpc()
    limits = [5, 17, 40]
    with mpc.Batch(deterministic=True, graph_steps=8) as b:
        boxes = [b.add(**MIX[k]) for k in range(3)]
        for bx, lim in zip(boxes, limits):
            bx.set_step_limit(lim)
        b.step(30)
        b.synchronize()
        assert [bx.get_state()[3] for bx in boxes] == [5, 17, 30]
        s5 = _state(boxes[0])
        b.step(25)
        assert [bx.get_state()[3] for bx in boxes] == [5, 17, 40]
        assert _same(_state(boxes[0]), s5)  # untouched after its limit
        with pytest.raises(mpc.MpcError):
            boxes[1].set_step_limit(3)  # before the steps already requested
    with mpc.Batch(deterministic=True) as b:
        bx = b.add(**MIX[0])
        b.step(5)
        assert _same(_state(bx), s5)


def test_arena_admission_and_reuse():
    mpc = _mpc()
    kw = dict(L=24, n_c=10.0, h=0.1, alpha_deg=130.0, seed=3)
    steady, peak = mpc.mpc_footprint(mpc.make_params(**kw))
    assert 0 < steady < peak
    arena = steady + peak + peak // 2  # two boxes, not three
    with mpc.Batch(arena_bytes=arena, graph_steps=4) as b:
        a1 = b.add(**kw)
        assert a1.info.device_bytes <= steady
        a2 = b.add(**dict(kw, seed=4))
        with pytest.raises(mpc.MpcError) as e:
            b.add(**dict(kw, seed=5))
        assert e.value.status == mpc.MPC_ENOMEM
        b.step(6)  # queued steps still read a1 when it is removed
        b.remove(a1)
        a3 = b.add(**dict(kw, seed=5))  # reuses a1's memory once the steps have passed
        b.step(6)
        b.synchronize()
        assert a2.get_state()[3] == 12 and a3.get_state()[3] == 6
        info = b.info()
        assert info.n_boxes == 2 and info.arena_used <= 2 * steady + (1 << 20)
        b.remove(a2)
        b.remove(a3)
        b.synchronize()
        assert b.info().arena_used == 0


def test_overflow_inside_batch_is_repaired_exactly():
    """A member whose brick capacity is too small halts inside the batch, is repaired at
    synchronisation and finishes its steps alone: in deterministic mode its trajectory is
    bit-identical to the same box with ample capacity."""
    mpc = _mpc()
    kw = dict(L=16, n_c=10.0, h=0.1, alpha_deg=130.0, variant=1, seed=12)
    with mpc.Batch(deterministic=True, graph_steps=8) as b:
        tight = b.add(capacity=4, **kw)
        other = b.add(**MIX[0])
        b.step(24)
        b.synchronize()
        assert mpc.mpc_get_info(tight.handle).recoveries > 0
        st_tight = _state(tight)
        assert st_tight[3] == 24 and other.get_state()[3] == 24
    with mpc.Batch(deterministic=True, graph_steps=8) as b:
        ref = b.add(**kw)
        b.step(24)
        assert _same(_state(ref), st_tight)


def test_autotune_picks_a_candidate():
    mpc = _mpc()
    p = mpc.make_params(L=32, n_c=10.0, h=0.1, alpha_deg=130.0, variant=0, seed=2)
    tile, tpc, ns = mpc.mpc_autotune(p)
    assert tile in (320, 640, 1280) and tpc in (1, 2, 4, 8, 16, 32) and ns > 0
    with mpc.Batch(autotune=True) as b:
        b.add(L=12, n_c=10.0, variant=0, seed=1)
        b.add(L=20, n_c=10.0, variant=0, seed=2)
        b.add(L=16, n_c=5.0, variant=1, seed=3)
        assert b.info().tuned_classes == 2
        b.step(3)
        b.synchronize()


def test_boxes_with_different_shared_memory_needs_coexist():
    """Creating a box with a small shared-memory need must not break a box created
    earlier with a larger one (the kernels' shared-memory cap is process-wide)."""
    mpc = _mpc()
    big = mpc.Simulation(L=16, n_c=20.0, variant=1, tile_particles=1280, seed=1)
    small = mpc.Simulation(L=8, n_c=5.0, variant=0, tile_particles=320, seed=2)
    big.step(3)
    small.step(3)
    big.synchronize()
    small.synchronize()
    assert big.get_state()[3] == 3 and small.get_state()[3] == 3
    big.close()
    small.close()


def test_solo_members_match_packed_and_oracle():
    """Members with at least two GPU waves of bricks get their own single-box launch
    inside the batch step; their results are bit-identical to packing them (deterministic
    mode) and match the oracle."""
    mpc = _mpc()
    big = dict(L=48, n_c=20.0, h=0.05, variant=1, seed=2001)
    kws = [big, MIX[0], MIX[3]]
    runs = []
    for pack_all in (False, True):
        with mpc.Batch(deterministic=True, graph_steps=8, pack_all=pack_all) as b:
            boxes = [b.add(**kw) for kw in kws]
            b.step(20)
            runs.append(([_state(bx) for bx in boxes], b.info().solo_boxes))
    assert runs[0][1] == 1 and runs[1][1] == 0
    for a, c in zip(runs[0][0], runs[1][0]):
        assert _same(a, c)
    with mpc.Batch(graph_steps=8) as b:
        boxes = [b.add(**kw) for kw in kws]
        b.step(3)
        pre = [bx.get_state()[:3] for bx in boxes]
        b.step(1)
        for kw, bx, p0 in zip(kws, boxes, pre):
            X1, V1, id1, step = bx.get_state()
            assert step == 4
            par.check_step(par.oracle_params(**kw), p0, (X1, V1, id1), 3)
