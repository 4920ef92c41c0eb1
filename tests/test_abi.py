"""The C-ABI library builds, loads and exports every entry point include/mpc.h declares;
struct layouts of the Python mirror match the header; argument checks run before any
device access (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2406_15236_gb300 as mpc
from paper_2406_15236_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpc_[a-z_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    _build.build()
    lib = ctypes.CDLL(_build.LIB)
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), f"{n} declared in mpc.h but not exported"


def test_version_and_error_text():
    assert "sm_103a" in mpc.mpc_version()


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mpc.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mpc_params),'
                   ' sizeof(mpc_allocator), sizeof(mpc_obs), sizeof(mpc_info),'
                   ' offsetof(mpc_params, seed), offsetof(mpc_params, graph_steps),'
                   ' offsetof(mpc_obs, step));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(mpc.mpc_params), ctypes.sizeof(mpc.mpc_allocator),
            ctypes.sizeof(mpc.mpc_obs), ctypes.sizeof(mpc.mpc_info),
            mpc.mpc_params.seed.offset, mpc.mpc_params.graph_steps.offset, mpc.mpc_obs.step.offset]
    assert got == want


@pytest.mark.parametrize("bad", [dict(L=1), dict(L=(8, 8, 2000)), dict(h=0.0), dict(kT=-1.0),
                                 dict(n_c=0.0), dict(variant=7), dict(variant=1, thermostat=1),
                                 dict(variant=1, walls_z=1), dict(capacity=-3),
                                 dict(gravity=(float("nan"), 0.0, 0.0))])
def test_invalid_parameters_rejected_without_device(bad):
    p = mpc.make_params(**bad)
    with pytest.raises(mpc.MpcError) as e:
        mpc.mpc_create(p)
    assert e.value.status == mpc.MPC_EINVAL
    assert mpc.mpc_last_error()


def test_only_a_equals_one():
    p = mpc.make_params()
    p.a = 2.0
    with pytest.raises(mpc.MpcError) as e:
        mpc.mpc_create(p)
    assert e.value.status == mpc.MPC_EINVAL


def test_null_handle_calls_fail_cleanly():
    lib = mpc.lib()
    assert lib.mpc_step(None, 1) == mpc.MPC_EINVAL
    assert lib.mpc_synchronize(None) == mpc.MPC_EINVAL
    assert lib.mpc_destroy(None) == mpc.MPC_OK
