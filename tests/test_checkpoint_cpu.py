"""Checkpoint reading validates the file set on the host before any device work: a
valid set written by an independent writer gets as far as creating the box (which needs
a GPU: MPC_ECUDA here), and broken sets are refused with MPC_EINVAL."""
import numpy as np
import pytest

import paper_2406_15236_gb300 as mpc
from tests import _ckpt

pytestmark = pytest.mark.skipif(
    __import__("torch").cuda.is_available(), reason="checks the host-only failure path")


def _valid(tmp_path, name="ck"):
    L, n_c = (4, 3, 5), 2.0
    F = _ckpt.fixed_bits(L)
    N = int(round(np.prod(L) * n_c))
    rng = np.random.default_rng(0)
    X = np.stack([rng.integers(0, l << F, N, dtype=np.int64) for l in L]).astype(np.uint32)
    V = rng.normal(size=(3, N)).astype(np.float32)
    ids = rng.permutation(N).astype(np.uint32)
    prefix = str(tmp_path / name)
    _ckpt.write(prefix, L, n_c, X, V, ids, step=11)
    return prefix, N


def _status(prefix):
    with pytest.raises(mpc.MpcError) as e:
        mpc.mpc_checkpoint_read(prefix)
    return e.value.status


def test_valid_set_reaches_device_creation(tmp_path):
    prefix, _ = _valid(tmp_path)
    assert _status(prefix) == mpc.MPC_ECUDA


@pytest.mark.parametrize("damage", ["counts", "offsets", "cell", "truncate", "format", "key",
                                    "outside", "n_particles"])
def test_broken_sets_are_refused(tmp_path, damage):
    prefix, N = _valid(tmp_path)
    kv, L, X, V, ids, counts, offsets = _ckpt.read(prefix)
    if damage == "counts":
        counts = counts.copy()
        counts[0] += 1
        counts[-1] -= 1 if counts[-1] else 0
        open(prefix + ".cells", "wb").write(counts.astype("<u4").tobytes() + offsets.astype("<u4").tobytes())
    elif damage == "offsets":
        offsets = offsets.copy()
        offsets[1] += 1
        open(prefix + ".cells", "wb").write(counts.astype("<u4").tobytes() + offsets.astype("<u4").tobytes())
    elif damage in ("cell", "outside"):
        X = X.copy()
        F = int(kv["fixed_bits"])
        X[0, 0] = (np.uint32(L[0]) << np.uint32(F)) + 5 if damage == "outside" else X[0, -1]
        raw = np.concatenate([X.ravel(), V.view("<u4").ravel(), ids]).astype("<u4")
        if damage == "cell" and _ckpt.cells_of(X, L, F)[0] == _ckpt.cells_of(X, L, F)[-1]:
            pytest.skip("first and last particle share a cell")
        open(prefix + ".particles", "wb").write(raw.tobytes())
    elif damage == "truncate":
        data = open(prefix + ".particles", "rb").read()
        open(prefix + ".particles", "wb").write(data[:-4])
    else:
        text = open(prefix + ".txt").read()
        if damage == "format":
            text = text.replace("mpc-checkpoint 1", "mpc-checkpoint 9")
        elif damage == "key":
            text = text.replace("seed = 7\n", "")
        else:
            text = text.replace(f"n_particles = {N}", f"n_particles = {N + 1}")
        open(prefix + ".txt", "w").write(text)
    assert _status(prefix) == mpc.MPC_EINVAL
    assert "checkpoint" in mpc.mpc_last_error()
