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


LAYOUT = [
    ("sizeof(mpc_params)", lambda: ctypes.sizeof(mpc.mpc_params)),
    ("sizeof(mpc_allocator)", lambda: ctypes.sizeof(mpc.mpc_allocator)),
    ("sizeof(mpc_obs)", lambda: ctypes.sizeof(mpc.mpc_obs)),
    ("sizeof(mpc_info)", lambda: ctypes.sizeof(mpc.mpc_info)),
    ("sizeof(mpc_batch_config)", lambda: ctypes.sizeof(mpc.mpc_batch_config)),
    ("sizeof(mpc_batch_info)", lambda: ctypes.sizeof(mpc.mpc_batch_info)),
    ("offsetof(mpc_params, seed)", lambda: mpc.mpc_params.seed.offset),
    ("offsetof(mpc_params, graph_steps)", lambda: mpc.mpc_params.graph_steps.offset),
    ("offsetof(mpc_params, tile_particles)", lambda: mpc.mpc_params.tile_particles.offset),
    ("offsetof(mpc_params, obs_ring)", lambda: mpc.mpc_params.obs_ring.offset),
    ("offsetof(mpc_params, wall_u)", lambda: mpc.mpc_params.wall_u.offset),
    ("offsetof(mpc_obs, step)", lambda: mpc.mpc_obs.step.offset),
    ("offsetof(mpc_info, threads_per_cell)", lambda: mpc.mpc_info.threads_per_cell.offset),
    ("offsetof(mpc_batch_config, flags)", lambda: mpc.mpc_batch_config.flags.offset),
    ("offsetof(mpc_batch_info, grid)", lambda: mpc.mpc_batch_info.grid.offset),
    ("offsetof(mpc_batch_info, tuned_classes)", lambda: mpc.mpc_batch_info.tuned_classes.offset),
    ("offsetof(mpc_batch_info, solo_boxes)", lambda: mpc.mpc_batch_info.solo_boxes.offset),
    ("offsetof(mpc_batch_info, packed_launches)",
     lambda: mpc.mpc_batch_info.packed_launches.offset),
    ("offsetof(mpc_batch_info, plan_ms)", lambda: mpc.mpc_batch_info.plan_ms.offset),
    ("sizeof(mpc_server_config)", lambda: ctypes.sizeof(mpc.mpc_server_config)),
    ("sizeof(mpc_job)", lambda: ctypes.sizeof(mpc.mpc_job)),
    ("sizeof(mpc_job_result)", lambda: ctypes.sizeof(mpc.mpc_job_result)),
    ("offsetof(mpc_job, steps)", lambda: mpc.mpc_job.steps.offset),
    ("offsetof(mpc_job, keep)", lambda: mpc.mpc_job.keep.offset),
    ("offsetof(mpc_job_result, eta_gk)", lambda: mpc.mpc_job_result.eta_gk.offset),
    ("offsetof(mpc_server_config, flags)", lambda: mpc.mpc_server_config.flags.offset),
    ("offsetof(mpc_server_config, fill_kparticles)",
     lambda: mpc.mpc_server_config.fill_kparticles.offset),
    ("sizeof(mpc_server_stats)", lambda: ctypes.sizeof(mpc.mpc_server_stats)),
    ("offsetof(mpc_server_stats, plan_ms)", lambda: mpc.mpc_server_stats.plan_ms.offset),
]


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    body = "".join(f'printf("%zu\\n", (size_t){expr});' for expr, _ in LAYOUT)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mpc.h"\n'
                   'int main(void){' + body + 'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [f() for _, f in LAYOUT]
    assert got == want, list(zip([e for e, _ in LAYOUT], got, want))


@pytest.mark.parametrize("bad", [dict(L=1), dict(L=(8, 8, 2000)), dict(h=0.0), dict(kT=-1.0),
                                 dict(n_c=0.0), dict(variant=7), dict(variant=1, thermostat=1),
                                 dict(variant=2, thermostat=1, walls_z=1), dict(capacity=-3),
                                 dict(gravity=(float("nan"), 0.0, 0.0)),
                                 dict(tile_particles=-1), dict(tile_particles=20000),
                                 dict(threads_per_cell=3), dict(threads_per_cell=64),
                                 dict(obs_ring=-1), dict(flags=64), dict(walls_z=3),
                                 dict(wall_u=(0.1, 0.0)),
                                 dict(walls_z=2, wall_u=(0.0, -0.1)),
                                 dict(walls_z=1, wall_u=(float("inf"), 0.0))])
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


def test_reserved_field_must_be_zero():
    p = mpc.make_params()
    p.reserved = 1
    with pytest.raises(mpc.MpcError) as e:
        mpc.mpc_create(p)
    assert e.value.status == mpc.MPC_EINVAL


def test_null_batch_calls_fail_cleanly():
    lib = mpc.lib()
    assert lib.mpc_batch_step(None, 1) == mpc.MPC_EINVAL
    assert lib.mpc_batch_synchronize(None) == mpc.MPC_EINVAL
    assert lib.mpc_batch_remove(None, None) == mpc.MPC_EINVAL
    assert lib.mpc_batch_destroy(None) == mpc.MPC_OK
    assert lib.mpc_set_step_limit(None, 5) == mpc.MPC_EINVAL


def test_invalid_batch_config_rejected_without_device():
    cfg = mpc.mpc_batch_config()
    cfg.max_boxes = 100000
    with pytest.raises(mpc.MpcError) as e:
        mpc.mpc_batch_create(cfg)
    assert e.value.status == mpc.MPC_EINVAL
    assert mpc.mpc_batch_last_error()


def test_invalid_server_config_rejected_without_device():
    cfg = mpc.mpc_server_config()
    cfg.hbm_budget_bytes = 0
    with pytest.raises(mpc.MpcError) as e:
        mpc.mpc_server_create(cfg)
    assert e.value.status == mpc.MPC_EINVAL
    assert mpc.mpc_server_last_error()
    lib = mpc.lib()
    assert lib.mpc_server_run(None, 1.0) == mpc.MPC_EINVAL
    assert lib.mpc_server_destroy(None) == mpc.MPC_OK
