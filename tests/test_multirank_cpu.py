"""The multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1) agree on the
max-over-ranks time and pass the barrier; the reference arm does no work on rank > 0."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_env()
    m = bench.max_over_ranks(10.0 + 3.0 * r, w)
    bench.barrier(w)
    ref = None
    if r == 1:
        ref = bench.run_reference(bench.parse_args(["--impl", "reference", "--gpus", "2"]))
    q.put((r, w, local, m, ref))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_max_time_and_barrier():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == 13.0 for o in out)  # max over ranks of 10 + 3 r
    assert out[1][4] == 0  # rank 1 of the reference arm exits 0 without work
