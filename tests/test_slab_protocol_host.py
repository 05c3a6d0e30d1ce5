"""The halo protocol of the slab decomposition (paper_1901_08766_gb300.slabs) on CPU
ranks (gloo, world size 2): each rank holds one slab of a periodic grid and steps it with
the FP64 oracle on the slab widened by one halo column per side; before every step the
ranks exchange, across each cut, only the populations that cross it (e_x = +1 eastward,
e_x = -1 westward) of their edge column. The gathered slabs equal the undivided oracle
run bit for bit, and the slab forces add up to the undivided forces."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

NX, NY, W0, STEPS = 64, 40, 28, 30


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _grid():
    import synth
    # dyadic centres: the slab-local centre (c - x0) is exact
    shapes = [synth._circle(1, 26.5, 20.25, 6.0), synth._circle(2, 50.25, 14.5, 5.0)]
    bodies = [synth._body(26.5, 20.25, 12.0, omega=1e-3), synth._body(50.25, 14.5, 10.0, vx=0.01)]
    return synth._spec("protocol", NX, NY, 0.05, shapes, bodies, 0, 0.02, synth._edges(),
                       u0=(0.02, 0.0))


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import oracle
    import synth
    from paper_1901_08766_gb300 import slabs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = _grid()
    widths = [W0, NX - W0]
    sp = slabs.split_spec(spec, widths)[rank]
    x0, w = sp["x_origin"], sp["nx"]
    mask_full = oracle.rasterize(spec)
    g_full = synth.random_populations(9, NX, NY, 0.05)
    g = g_full[:, :, x0:x0 + w].copy()
    # the slab widened by one halo column per side; halo nodes are fluid and their own
    # update is discarded, so they add nothing to the forces
    ext = dict(spec, nx=w + 2)
    ext["bodies"] = [dict(b, cx=b["cx"] - (x0 - 1)) for b in spec["bodies"]]
    mask = np.zeros((NY, w + 2), dtype=np.uint8)
    mask[:, 1:w + 1] = mask_full[:, x0:x0 + w]
    east, west = (rank + 1) % world, (rank - 1) % world
    forces = []
    for _ in range(STEPS):
        halo_w = np.repeat(g[:, :, :1], 1, axis=2).copy()  # placeholders for non-crossing directions
        halo_e = np.repeat(g[:, :, -1:], 1, axis=2).copy()
        send_e = torch.from_numpy(np.ascontiguousarray(g[list(slabs.CROSS_EAST), :, -1]))
        send_w = torch.from_numpy(np.ascontiguousarray(g[list(slabs.CROSS_WEST), :, 0]))
        recv_w = torch.empty_like(send_e)  # from the west neighbour: its eastward crossers
        recv_e = torch.empty_like(send_w)  # from the east neighbour: its westward crossers
        reqs = [dist.isend(send_e, east), dist.isend(send_w, west),
                dist.irecv(recv_w, west), dist.irecv(recv_e, east)]
        for r in reqs:
            r.wait()
        halo_w[list(slabs.CROSS_EAST), :, 0] = recv_w.numpy()
        halo_e[list(slabs.CROSS_WEST), :, 0] = recv_e.numpy()
        d = oracle.Domain(ext, mask=mask, g=np.concatenate([halo_w, g, halo_e], axis=2))
        _, fb = d.step_once()
        g = d.g[:, :, 1:w + 1].copy()
        forces.append(fb)
    out.put((rank, x0, g, np.array(forces)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_halo_exchange_reproduces_the_undivided_grid():
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    spec = _grid()
    ref = oracle.Domain(spec, g=synth.random_populations(9, NX, NY, 0.05))
    f_ref = ref.run(STEPS)
    g = np.concatenate([r[2] for r in res], axis=2)
    assert np.array_equal(g, ref.g)
    f = res[0][3] + res[1][3]
    assert np.abs(f - f_ref).max() <= 1e-13 * np.abs(f_ref).max()
