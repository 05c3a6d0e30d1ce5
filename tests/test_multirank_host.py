"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2). The domains are
independent, so the ranks exchange no data: each rank advances a disjoint, cell-balanced
shard of the set (or, in copy mode, its own full copy); the reported time is the max over
ranks and the value counts the nodes of all ranks."""
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


def _worker(rank, world, port, mode, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    specs = bench.rank_domains(synth.batched_domains(64), rank, world, mode)
    cells = sum(s["nx"] * s["ny"] for s in specs)
    names = sorted(s["name"] for s in specs)
    ms_local = 100.0 + 50.0 * rank  # rank 1 is the slow one
    ms, value, total = bench.aggregate(ms_local, cells, 1000, world)
    out.put((rank, cells, names, ms, value, total))
    dist.barrier()
    dist.destroy_process_group()


def _run(mode, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_two_rank_shards_are_disjoint_balanced_and_aggregate():
    import synth
    every = synth.batched_domains(64)
    all_cells = sum(s["nx"] * s["ny"] for s in every)
    (r0, c0, n0, ms0, v0, t0), (r1, c1, n1, ms1, v1, t1) = _run("shard")
    assert not set(n0) & set(n1)                        # disjoint
    assert sorted(n0 + n1) == sorted(s["name"] for s in every)  # the whole set
    assert c0 + c1 == all_cells
    assert abs(c0 - c1) <= max(s["nx"] * s["ny"] for s in every)  # balanced within a domain
    assert ms0 == ms1 == 150.0                          # max over ranks
    assert t0 == t1 == all_cells                        # nodes summed over ranks
    assert v0 == pytest.approx(all_cells * 1000 / 0.150 / 1e9)


def test_two_rank_copies_aggregate_weak_scaling():
    (r0, c0, n0, ms0, v0, t0), (r1, c1, n1, ms1, v1, t1) = _run("copy")
    assert c0 == c1 and n0 == n1  # the same per-rank work
    assert ms0 == ms1 == 150.0
    assert v0 == pytest.approx(c0 * 2 * 1000 / 0.150 / 1e9)


def test_shard_of_one_rank_is_the_whole_set():
    import bench
    import synth
    every = synth.batched_domains(64)
    assert bench.rank_domains(every, 0, 1) == every
    four = [bench.rank_domains(every, r, 4) for r in range(4)]
    assert sorted(s["name"] for part in four for s in part) == sorted(s["name"] for s in every)
    loads = [sum(s["nx"] * s["ny"] for s in part) for part in four]
    assert max(loads) - min(loads) <= max(s["nx"] * s["ny"] for s in every)


def test_halo_topology_of_slabs_over_ranks():
    from paper_1901_08766_gb300 import slabs
    owner, peers = slabs.halo_topology(4, 2, periodic=True)
    assert owner == [0, 0, 1, 1] and peers == [(1, 1), (0, 0)]
    owner, peers = slabs.halo_topology(4, 2, periodic=False)
    assert peers == [(None, 1), (0, None)]
    owner, peers = slabs.halo_topology(6, 3, periodic=True)
    assert owner == [0, 0, 1, 1, 2, 2] and peers == [(2, 1), (0, 2), (1, 0)]
    owner, peers = slabs.halo_topology(3, 1, periodic=True)
    assert peers == [(None, None)]  # every cut inside the one rank
    with pytest.raises(ValueError):
        slabs.halo_topology(3, 2, periodic=True)
