"""The benchmark's multi-process path on CPU: two gloo ranks (127.0.0.1)
run as independent replicas and agree on the maximum of their timings; the
whole-job work is the sum over ranks (weak scaling, no data exchange)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, tdist = bench.dist_init(world)
    val = bench.barrier_max(tdist, 10.0 + r, "cpu")
    tdist.barrier()
    q.put((r, w, val, bench.replica_units(5.0, w)))
    tdist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(o[0] for o in out) == [0, 1]
    assert all(o[1] == world and o[2] == 11.0 and o[3] == 10.0 for o in out)
