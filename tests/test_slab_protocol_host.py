"""The halo protocol of the slab decomposition (paper_1901_08766_gb300.slabs) on CPU
ranks (gloo, world size 2), with the exchange code the device path uses (slabs.exchange)
and its buffer layout ([9][ny], the crossing planes only). Each rank holds one slab of a
grid and steps it with the FP64 oracle on the slab widened by one halo column on each side
that has a neighbour. Before every step the ranks exchange, across each cut, only the
populations that cross it (e_x = +1 eastward, e_x = -1 westward) of their edge column. For
a periodic ring of two ranks both neighbours are the same rank, which checks that the
transfers are matched in order. The gathered slabs equal the undivided oracle run bit for
bit, and the slab forces add up to the undivided forces."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

NX, NY, W0, STEPS = 64, 40, 32, 30


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _grid(kind):
    import synth
    # dyadic centres: the slab-local centre (c - x0) is exact
    shapes = [synth._circle(1, 26.5, 20.25, 6.0), synth._circle(2, 50.25, 14.5, 5.0)]
    bodies = [synth._body(26.5, 20.25, 12.0, omega=1e-3), synth._body(50.25, 14.5, 10.0, vx=0.01)]
    edges = synth._edges() if kind == "periodic" else synth._edges("inlet", "outflow", "free_slip", "free_slip")
    return synth._spec("protocol", NX, NY, 0.05, shapes, bodies, 0, 0.02, edges,
                       u_in=(0.02, 0.0), u0=(0.02, 0.0))


def _worker(rank, world, port, kind, out):
    import torch
    import torch.distributed as dist
    import oracle
    import synth
    from paper_1901_08766_gb300 import slabs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = _grid(kind)
    widths = [W0, NX - W0]
    sp = slabs.split_spec(spec, widths)[rank]
    x0, w = sp["x_origin"], sp["nx"]
    periodic = kind == "periodic"
    # ranks across the west and east edges (None: the grid's own edge)
    west = (rank - 1) % world if (periodic or rank > 0) else None
    east = (rank + 1) % world if (periodic or rank < world - 1) else None
    hw, he = int(west is not None), int(east is not None)
    mask_full = oracle.rasterize(spec)
    g_full = synth.random_populations(9, NX, NY, 0.05)
    g = g_full[:, :, x0:x0 + w].copy()
    # the slab widened by one halo column per neighbour; halo nodes are fluid and their
    # own update is discarded, so they add nothing to the forces
    ext = dict(spec, nx=w + hw + he)
    ext["bodies"] = [dict(b, cx=b["cx"] - (x0 - hw)) for b in spec["bodies"]]
    mask = np.zeros((NY, w + hw + he), dtype=np.uint8)
    mask[:, hw:hw + w] = mask_full[:, x0:x0 + w]
    bufs = {k: torch.zeros((9, NY), dtype=torch.float64) for k in ("sw", "se", "rw", "re")}
    forces = []
    for _ in range(STEPS):
        # pack: this slab's outgoing crossing planes at its edge columns
        bufs["sw"][list(slabs.LEAVE_WEST)] = torch.from_numpy(g[list(slabs.LEAVE_WEST), :, 0])
        bufs["se"][list(slabs.LEAVE_EAST)] = torch.from_numpy(g[list(slabs.LEAVE_EAST), :, -1])
        slabs.exchange(bufs["sw"], bufs["se"], bufs["rw"], bufs["re"], west, east)
        cols = [g]
        if hw:
            halo_w = g[:, :, :1].copy()  # placeholders for the planes that do not cross
            halo_w[list(slabs.LEAVE_EAST), :, 0] = bufs["rw"][list(slabs.LEAVE_EAST)].numpy()
            cols.insert(0, halo_w)
        if he:
            halo_e = g[:, :, -1:].copy()
            halo_e[list(slabs.LEAVE_WEST), :, 0] = bufs["re"][list(slabs.LEAVE_WEST)].numpy()
            cols.append(halo_e)
        d = oracle.Domain(ext, mask=mask, g=np.concatenate(cols, axis=2))
        _, fb = d.step_once()
        g = d.g[:, :, hw:hw + w].copy()
        forces.append(fb)
    out.put((rank, x0, g, np.array(forces)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["periodic", "channel"])
def test_two_rank_halo_exchange_reproduces_the_undivided_grid(kind):
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, kind, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    spec = _grid(kind)
    ref = oracle.Domain(spec, g=synth.random_populations(9, NX, NY, 0.05))
    f_ref = ref.run(STEPS)
    g = np.concatenate([r[2] for r in res], axis=2)
    assert np.array_equal(g, ref.g)
    f = res[0][3] + res[1][3]
    assert np.abs(f - f_ref).max() <= 1e-13 * np.abs(f_ref).max()
