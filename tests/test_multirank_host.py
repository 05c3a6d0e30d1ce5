"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank runs its own
copy of the independent domains (no data-path collective); the reported time is the max
over ranks and the value counts the nodes of all ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    specs = bench.rank_domains(synth.batched_domains(8), rank, world)
    cells = sum(s["nx"] * s["ny"] for s in specs)
    ms_local = 100.0 + 50.0 * rank  # rank 1 is the slow one
    ms, value = bench.aggregate(ms_local, cells, 1000, world)
    out.put((rank, cells, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, c0, ms0, v0), (r1, c1, ms1, v1) = res
    assert c0 == c1  # weak scaling: the same per-rank work
    assert ms0 == ms1 == 150.0  # max over ranks
    assert v0 == pytest.approx(c0 * 2 * 1000 / 0.150 / 1e9)
