"""Checkpoint files through the C ABI on the GPU: the files follow the documented layout
(read back by an independent reader), a box restored from them has the same state and
step, and in deterministic mode continues bit for bit as the original would."""
import numpy as np
import pytest

from tests import _ckpt, _parity as par

pytestmark = pytest.mark.gpu


def _mpc():
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    return mpc


@pytest.mark.parametrize("variant", [0, 1])
def test_checkpoint_round_trip_and_restart(tmp_path, variant):
    mpc = _mpc()
    kw = dict(L=(12, 8, 10), n_c=7.5, h=0.1, alpha_deg=130.0, variant=variant, seed=31,
              flags=mpc.MPC_FLAG_DETERMINISTIC)
    sim = mpc.Simulation(**kw)
    sim.step(17)
    prefix = str(tmp_path / "box")
    sim.checkpoint(prefix)
    X0, V0, id0, step0 = sim.get_state()
    # the layout, read independently
    kv, L, X, V, ids, counts, offsets = _ckpt.read(prefix)
    assert L == (12, 8, 10) and int(kv["step"]) == 17 and int(kv["seed"]) == 31
    F = int(kv["fixed_bits"])
    c = _ckpt.cells_of(X, L, F)
    assert np.all(np.diff(c) >= 0)
    np.testing.assert_array_equal(counts, np.bincount(c, minlength=len(counts)))
    np.testing.assert_array_equal(offsets[1:], np.cumsum(counts)[:-1])
    for a, b in zip(par.by_id(X, V, ids), par.by_id(X0, V0, id0)):
        np.testing.assert_array_equal(a, b)
    # restore, compare, continue
    rest = mpc.Simulation.from_checkpoint(prefix)
    X1, V1, id1, step1 = rest.get_state()
    assert step1 == 17
    for a, b in zip(par.by_id(X1, V1, id1), par.by_id(X0, V0, id0)):
        np.testing.assert_array_equal(a, b)
    sim.step(10)
    rest.step(10)
    for a, b in zip(par.by_id(*sim.get_state()[:3]), par.by_id(*rest.get_state()[:3])):
        np.testing.assert_array_equal(a, b)
    sim.close()
    rest.close()


def test_independently_written_checkpoint_is_read(tmp_path):
    mpc = _mpc()
    L, n_c = (6, 5, 4), 3.0
    F = _ckpt.fixed_bits(L)
    N = int(round(np.prod(L) * n_c))
    rng = np.random.default_rng(4)
    X = np.stack([rng.integers(0, l << F, N, dtype=np.int64) for l in L]).astype(np.uint32)
    V = rng.normal(size=(3, N)).astype(np.float32)
    ids = rng.permutation(N).astype(np.uint32)
    prefix = str(tmp_path / "ext")
    _ckpt.write(prefix, L, n_c, X, V, ids, step=5, seed=9)
    sim = mpc.Simulation.from_checkpoint(prefix)
    X1, V1, id1, step = sim.get_state()
    assert step == 5
    for a, b in zip(par.by_id(X1, V1, id1), par.by_id(X, V, ids)):
        np.testing.assert_array_equal(a, b)
    # one step matches the oracle from the restored state
    sim.step(1)
    X2, V2, id2, _ = sim.get_state()
    par.check_step(par.oracle_params(L=L, n_c=n_c, h=0.1, alpha_deg=130.0, seed=9),
                   (X1, V1, id1), (X2, V2, id2), 5)
    sim.close()


def test_checkpoint_keeps_moving_walls(tmp_path):
    mpc = _mpc()
    kw = dict(L=(6, 6, 8), n_c=8.0, h=0.1, alpha_deg=130.0, walls_z=1, thermostat=1,
              wall_u=(-0.2, 0.35), seed=8, flags=mpc.MPC_FLAG_DETERMINISTIC)
    sim = mpc.Simulation(**kw)
    sim.step(9)
    prefix = str(tmp_path / "walls")
    sim.checkpoint(prefix)
    rest = mpc.Simulation.from_checkpoint(prefix)
    sim.step(6)
    rest.step(6)
    for a, b in zip(par.by_id(*sim.get_state()[:3]), par.by_id(*rest.get_state()[:3])):
        np.testing.assert_array_equal(a, b)
    sim.close()
    rest.close()
