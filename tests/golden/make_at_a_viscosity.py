"""Writes at_a_viscosity.json: the oracle's Green-Kubo shear viscosity of MPC-AT+a at
N_c = 10, h = 0.05, kT = m = 1 (the headline workload's physics), from independent L = 10
boxes.  Calls only the oracle (FP64 CPU) and the test-side estimator tests/_gk.py.

    python tests/golden/make_at_a_viscosity.py [--boxes 32 --steps 24000 --procs 8]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

PARAMS = dict(L=10, n_c=10.0, h=0.05, kT=1.0, m=1.0)
K = 20          # window: one time unit (the stress autocorrelation has decayed)
DISCARD = 200   # steps of equilibration left out


def one_box(args):
    seed, steps = args
    sys.path.insert(0, ROOT)
    import oracle
    from tests._gk import green_kubo, stress_from_oracle_obs

    p = oracle.params(L=PARAMS["L"], n_c=PARAMS["n_c"], h=PARAMS["h"], kT=PARAMS["kT"],
                      m=PARAMS["m"], variant=oracle.AT_A, seed=seed)
    X, V, ids = oracle.init(p)
    rows = []
    for s in range(steps):
        r = oracle.step(p, X, V, ids, s, obs=True)
        X, V = r["X"], r["V"]
        rows.append(stress_from_oracle_obs(r["obs"]))
    return green_kubo(rows, float(PARAMS["L"] ** 3), PARAMS["h"], PARAMS["kT"], K=K, discard=DISCARD)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--boxes", type=int, default=32)
    ap.add_argument("--steps", type=int, default=24000)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    sys.path.insert(0, ROOT)
    import oracle

    oracle.build()
    seeds = [20000 + b for b in range(a.boxes)]
    with mp.get_context("spawn").Pool(a.procs) as pool:
        etas = pool.map(one_box, [(s, a.steps) for s in seeds])
    etas = np.array(etas)
    out = {"what": "oracle Green-Kubo shear viscosity, MPC-AT+a", "params": PARAMS,
           "window_steps": K, "discard_steps": DISCARD, "boxes": a.boxes, "steps": a.steps,
           "seeds": seeds, "eta": [float(e) for e in etas], "mean": float(etas.mean()),
           "se": float(etas.std(ddof=1) / np.sqrt(len(etas))),
           "written_by": "tests/golden/make_at_a_viscosity.py (oracle only)"}
    with open(os.path.join(HERE, "at_a_viscosity.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(f"eta = {out['mean']:.4f} +- {out['se']:.4f}")


if __name__ == "__main__":
    main()
