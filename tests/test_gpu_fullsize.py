"""Parity at the benchmark's full size and launch configuration: the MPC-AT+a box of
512^3 cells, N_c = 10 (1,342,177,280 particles), h = 0.05, seed 3, observables on --
exactly what bench.py times.

The oracle cannot step 1.3e9 particles, but a collision is local: the particles that
collide in cell c at step n all come from unshifted cells within c-2..c+1 per axis
(they move less than one cell per step and the shift is below one cell).  The test
gathers those particles from the GPU state for 50 random cells, steps the GPU once,
steps the oracle on the gathered subset, and compares every particle whose collision
cell is one of the sampled cells (positions bit-exact, velocities within the parity
bar).  Whole-box invariants (particle count, id set, momentum) are checked at the same
time.
"""
import numpy as np
import pytest

import oracle
from tests import _parity as par

pytestmark = pytest.mark.gpu

L = 512
KW = dict(L=L, n_c=10.0, h=0.05, kT=1.0, variant=1, seed=3)


def test_fullsize_sampled_cells_match_oracle():
    import torch

    import paper_2406_15236_gb300 as mpc

    torch.cuda.set_device(0)
    free, total = torch.cuda.mem_get_info()
    if free < 200e9:
        pytest.skip(f"needs ~200 GB of free device memory, {free / 1e9:.0f} GB free")
    sim = mpc.Simulation(flags=mpc.MPC_FLAG_OBSERVABLES, **KW)
    N = sim.N
    F = sim.info.fixed_bits
    step0 = 2
    sim.step(step0)
    P0 = sim.observables()["momentum"]

    def state():
        X = torch.empty((3, N), dtype=torch.int32, device="cuda")
        V = torch.empty((3, N), dtype=torch.float32, device="cuda")
        ids = torch.empty(N, dtype=torch.int32, device="cuda")
        s = mpc.mpc_get_state(sim.handle, X, V, ids, device_ptrs=True)
        return X, V, ids, s

    # --- pre-step state and the particles that can reach the sampled cells ---
    X, V, ids, s = state()
    assert s == step0
    rng = np.random.default_rng(7)
    cells = rng.integers(0, L, size=(50, 3))
    mark = torch.zeros(L * L * L, dtype=torch.bool, device="cuda")
    offs = np.arange(-2, 2)
    for cx, cy, cz in cells:
        gx, gy, gz = np.meshgrid((cx + offs) % L, (cy + offs) % L, (cz + offs) % L, indexing="ij")
        lin = torch.as_tensor((gx + L * (gy + L * gz)).ravel(), device="cuda")
        mark[lin] = True
    # canonical positions are below 2^31, so int32 arithmetic is exact here
    ucell = (X[0] >> F) + L * ((X[1] >> F) + L * (X[2] >> F))
    sel = mark[ucell]
    del ucell
    Xs = X[:, sel].cpu().numpy().view(np.uint32)
    Vs = V[:, sel].cpu().numpy()
    idss = ids[sel].cpu().numpy().view(np.uint32)
    # whole-box invariants on the pre-step state
    assert int(torch.sum(ids, dtype=torch.int64).item()) == N * (N - 1) // 2
    assert float(V.abs().max().item()) * KW["h"] < 1.0  # the neighbourhood argument holds
    del X, V, ids, sel
    torch.cuda.empty_cache()

    # --- one GPU step, then the same particles after it ---
    sim.step(1)
    X, V, ids, s = state()
    assert s == step0 + 1
    idmark = torch.zeros(N, dtype=torch.bool, device="cuda")
    idmark[torch.as_tensor(idss.astype(np.int64), device="cuda")] = True
    sel = idmark[ids]
    X1 = X[:, sel].cpu().numpy().view(np.uint32)
    V1 = V[:, sel].cpu().numpy()
    id1 = ids[sel].cpu().numpy().view(np.uint32)
    assert int(torch.sum(ids, dtype=torch.int64).item()) == N * (N - 1) // 2
    del X, V, ids, sel, idmark, mark
    P1 = sim.observables()["momentum"]
    sim.close()
    torch.cuda.empty_cache()

    # momentum is conserved by every AT+a collision: drift below 1e-6 of sum m|v|
    # (sum m|v| ~ 1.6 N at kT = 1)
    assert np.abs(np.asarray(P1) - np.asarray(P0)).max() < 1e-6 * 1.5 * N

    # --- oracle on the subset; compare the particles of the sampled cells ---
    p = par.oracle_params(**KW)
    o0 = np.argsort(idss)
    ref = oracle.step(p, Xs[:, o0], Vs[:, o0].astype(np.float64), idss[o0], step0, cells=True,
                      sens=True, flags=True)
    o1 = np.argsort(id1)
    assert np.array_equal(id1[o1], idss[o0])
    sampled = set(int(cx + L * (cy + L * cz)) for cx, cy, cz in cells)
    # the collision cell index on the shifted lattice equals cx + L(cy + L cz) for periodic boxes
    keep = np.array([c in sampled for c in ref["cell"]])
    assert keep.sum() > 300
    worst = par.check_subset(ref, X1[:, o1], V1[:, o1], keep, what="full size")
    print(f"full size: {keep.sum()} particles in {len(sampled)} sampled cells, "
          f"max velocity error outside ill-conditioned cells {worst:.3g}")
