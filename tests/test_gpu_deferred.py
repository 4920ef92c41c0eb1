"""The deferring step kernel of large boxes.

Boxes of 8192 bricks or more step with a kernel whose shared-memory tile holds 736 of a
brick's 864 slots (7 CTAs per SM instead of 6 for MPC-AT+a, 9 instead of 8 for SRD and
MPC-SRD+a); a brick that holds more particles in a step is left to a full-capacity pass
launched right after it.  At uniform density that
is ~7e-5 of the bricks.  Here a 128^3 box (32,768 bricks of 4^3 cells) gets a denser slab
(N_c 11 in x < 32: about a tenth of that slab's bricks exceed the tile in a step, and
none comes near the 864 slots of a brick) by moving particles into it with set_state.  For two consecutive steps, particles of cells sampled
inside the slab and outside it are compared with the oracle (stepped on the neighbourhood
of each sampled cell: the particles that collide in cell c come from unshifted cells
c-2..c+1 per axis); the second step also shows that the list of deferred bricks was
cleared in between.  The whole particle set (count, ids) must survive.  In the
fixed-point mode, where a trajectory does not depend on which kernel processes a brick,
the same dense-slab box stepped with the deferring kernel and with bricks of 320
particles (the generic kernel, full tile) must stay bit-identical.
"""
import numpy as np
import pytest

import oracle
from tests import _parity as par

pytestmark = pytest.mark.gpu

L = 128
KW = dict(L=L, n_c=10.0, h=0.05, kT=1.0, variant=1, seed=11)


def _dense_slab_state(X, ids, F, rng, L=L):
    """moves 5 % of the particles of x >= L/2 (chosen by id, so that the state does not
    depend on the order get_state returns them in) to uniform positions in x < L/4: the
    slab's density becomes 10 (1 + 0.05 * 2) = 11 per cell"""
    by_id = np.argsort(ids)
    src = by_id[(X[0, by_id] >> F) >= L // 2]
    pick = rng.choice(src, size=int(0.05 * src.size), replace=False)
    X = X.copy()
    X[0, pick] = rng.integers(0, (L // 4) << F, size=pick.size, dtype=np.uint64).astype(np.uint32)
    return X


def _neighbourhood(X, F, cells, L=L):
    ucell = (X[0] >> F).astype(np.int64) + L * ((X[1] >> F).astype(np.int64) + L * (X[2] >> F).astype(np.int64))
    mark = np.zeros(L ** 3, dtype=bool)
    offs = np.arange(-2, 2)
    for cx, cy, cz in cells:
        gx, gy, gz = np.meshgrid((cx + offs) % L, (cy + offs) % L, (cz + offs) % L, indexing="ij")
        mark[(gx + L * (gy + L * gz)).ravel()] = True
    return mark[ucell]


# L = 128: a periodic box of power-of-two extent without gravity (the plain kernel body);
# L = 96: the general streaming body with the deferring kernel
@pytest.mark.parametrize("variant,h,L", [(1, 0.05, 128), (0, 0.1, 128), (2, 0.05, 128), (1, 0.05, 96)])
def test_deferred_bricks_match_oracle(variant, h, L):
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    kw = dict(KW, variant=variant, h=h, L=L)
    sim = mpc.Simulation(flags=mpc.MPC_FLAG_OBSERVABLES, **kw)
    N = sim.N
    F = sim.info.fixed_bits
    nb = sim.info.n_bricks
    assert nb[0] * nb[1] * nb[2] >= 8192
    rng = np.random.default_rng(5)
    X, V, ids, s = sim.get_state()
    X = _dense_slab_state(X, ids, F, rng, L)
    sim.set_state(X, V, ids, s)
    # cells inside the dense slab (most of them in deferred bricks) and outside it
    cells = np.concatenate([
        np.stack([rng.integers(2, L // 4 - 2, 40), rng.integers(0, L, 40), rng.integers(0, L, 40)], axis=1),
        np.stack([rng.integers(L // 2, L, 10), rng.integers(0, L, 10), rng.integers(0, L, 10)], axis=1)])
    sampled = set(int(cx + L * (cy + L * cz)) for cx, cy, cz in cells)
    p = par.oracle_params(**kw)
    for k in range(2):
        X0, V0, id0, s0 = sim.get_state()
        assert X0.shape[1] == N and int(id0.astype(np.int64).sum()) == N * (N - 1) // 2
        sel = _neighbourhood(X0, F, cells, L)
        Xs, Vs, idss = X0[:, sel], V0[:, sel], id0[sel]
        sim.step(1)
        X1, V1, id1, s1 = sim.get_state()
        assert s1 == s0 + 1
        assert int(id1.astype(np.int64).sum()) == N * (N - 1) // 2
        idm = np.zeros(N, dtype=bool)
        idm[idss] = True
        sel1 = idm[id1]
        o0 = np.argsort(idss)
        o1 = np.argsort(id1[sel1])
        assert np.array_equal(id1[sel1][o1], idss[o0])
        ref = oracle.step(p, Xs[:, o0], Vs[:, o0].astype(np.float64), idss[o0], s0, cells=True,
                          sens=True, flags=True)
        keep = np.array([c in sampled for c in ref["cell"]])
        in_slab = keep & ((ref["X"][0] >> F) < L // 4)
        assert keep.sum() > 400 and in_slab.sum() > 300
        worst = par.check_subset(ref, X1[:, sel1][:, o1], V1[:, sel1][:, o1], keep,
                                 what=f"step {s0}")
        print(f"step {s0}: {keep.sum()} particles of {len(sampled)} sampled cells "
              f"({in_slab.sum()} in the dense slab), max velocity error {worst:.3g}")
    info = mpc.mpc_get_info(sim.handle)
    assert info.recoveries == 0  # no brick overflowed: the deferral, not the repair, ran
    sim.close()


def test_deterministic_deferred_equals_full_tile():
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    flags = mpc.MPC_FLAG_DETERMINISTIC | mpc.MPC_FLAG_OBSERVABLES
    rng = np.random.default_rng(6)
    results = []
    state0 = None
    for tile in (640, 320):
        sim = mpc.Simulation(flags=flags, tile_particles=tile, **KW)
        nb = sim.info.n_bricks
        if tile == 640:
            assert nb[0] * nb[1] * nb[2] >= 8192 and sim.info.capacity == 864  # deferring kernel
            X, V, ids, s = sim.get_state()
            state0 = (_dense_slab_state(X, ids, sim.info.fixed_bits, rng), V, ids, s)
        else:
            assert sim.info.capacity != 864  # the generic kernel
        sim.set_state(*state0)
        sim.step(6)
        X, V, ids, s = sim.get_state()
        o = np.argsort(ids)
        results.append((X[:, o], V[:, o], s, sim.observable_series(6)))
        assert mpc.mpc_get_info(sim.handle).recoveries == 0
        sim.close()
    assert results[0][2] == results[1][2] == 6
    assert np.array_equal(results[0][0], results[1][0])
    assert np.array_equal(results[0][1].view(np.uint32), results[1][1].view(np.uint32))
    assert np.array_equal(results[0][3], results[1][3])


def test_deferred_solo_member_of_a_batch_equals_packed():
    """A large member of a batch steps alone with the deferring kernel (and its
    full-capacity pass) inside the batch's graph; in the fixed-point mode its trajectory
    must equal the same member packed with the others (the packed kernel, full tile)."""
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    rng = np.random.default_rng(8)
    small = dict(L=12, n_c=10.0, h=0.1, variant=0, seed=31)
    state0 = None
    results = []
    for pack_all in (False, True):
        with mpc.Batch(deterministic=True, graph_steps=4, pack_all=pack_all) as b:
            big = b.add(**KW)
            other = b.add(**small)
            if state0 is None:
                X, V, ids, s = big.get_state()
                state0 = (_dense_slab_state(X, ids, big.info.fixed_bits, rng), V, ids, s)
            big.set_state(*state0)
            b.step(6)
            assert b.info().solo_boxes == (0 if pack_all else 1)
            X, V, ids, s = big.get_state()
            o = np.argsort(ids)
            results.append((X[:, o], V[:, o].view(np.uint32), s, _state_of(other)))
    assert results[0][2] == results[1][2] == 6
    assert np.array_equal(results[0][0], results[1][0])
    assert np.array_equal(results[0][1], results[1][1])
    for a, c in zip(results[0][3], results[1][3]):
        assert np.array_equal(a, c)


def _state_of(box):
    X, V, ids, _ = box.get_state()
    o = np.argsort(ids)
    return X[:, o], V[:, o].view(np.uint32)
