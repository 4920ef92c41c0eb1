"""A second, independent writer/reader of the checkpoint file layout documented in
include/mpc.h (test infrastructure): text parameters, particle SoA blocks ordered by
unshifted cell, per-cell counts and offsets."""
import numpy as np


def fixed_bits(L):
    return 31 - int(np.ceil(np.log2(max(L))))


def cells_of(X, L, F):
    cx, cy, cz = (X >> np.uint32(F)).astype(np.int64)
    return cx + L[0] * (cy + L[1] * cz)


def write(prefix, L, n_c, X, V, ids, step, seed=7, h=0.1, alpha_deg=130.0, variant=0):
    L = tuple(int(v) for v in L)
    F = fixed_bits(L)
    N = X.shape[1]
    c = cells_of(X, L, F)
    order = np.argsort(c, kind="stable")
    X, V, ids, c = X[:, order], V[:, order], ids[order], c[order]
    C = L[0] * L[1] * L[2]
    counts = np.bincount(c, minlength=C).astype(np.uint32)
    offsets = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.uint32)
    with open(prefix + ".txt", "w") as f:
        f.write("format = mpc-checkpoint 1\n")
        f.write(f"L = {L[0]} {L[1]} {L[2]}\na = 1\nn_c = {n_c!r}\nh = {h!r}\n")
        f.write(f"alpha_deg = {alpha_deg!r}\nkT = 1\nm = 1\nvariant = {variant}\nthermostat = 0\n")
        f.write(f"walls_z = 0\ngravity = 0 0 0\nseed = {seed}\nbox_id = 0\nflags = 0\n")
        f.write(f"step = {step}\nn_particles = {N}\nfixed_bits = {F}\ncells = {C}\noffset_bytes = 4\n")
    with open(prefix + ".particles", "wb") as f:
        f.write(np.ascontiguousarray(X, dtype="<u4").tobytes())
        f.write(np.ascontiguousarray(V, dtype="<f4").tobytes())
        f.write(np.ascontiguousarray(ids, dtype="<u4").tobytes())
    with open(prefix + ".cells", "wb") as f:
        f.write(counts.astype("<u4").tobytes())
        f.write(offsets.astype("<u4").tobytes())


def read(prefix):
    kv = {}
    for line in open(prefix + ".txt"):
        if "=" in line:
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    L = tuple(int(v) for v in kv["L"].split())
    N = int(kv["n_particles"])
    C = int(kv["cells"])
    raw = np.fromfile(prefix + ".particles", dtype="<u4")
    assert raw.size == 7 * N
    X = raw[: 3 * N].reshape(3, N)
    V = raw[3 * N: 6 * N].view("<f4").reshape(3, N)
    ids = raw[6 * N:]
    cells = np.fromfile(prefix + ".cells", dtype="<u4")
    assert cells.size == 2 * C
    return kv, L, X, V, ids, cells[:C], cells[C:]
