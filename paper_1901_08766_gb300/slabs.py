"""Slab decomposition of one grid along x.

A grid too large for one device, or one that should spread over several, is cut into
slabs of whole columns. Each slab is a domain of its own whose `x_origin` is its first
global column (so shapes are rasterised, and obstacle velocities evaluated, at global
positions) and whose x edges at the cuts are linked: streaming across a cut (Eq.
streaming) pulls the adjacent column of the neighbouring slab at the same time level.
On one GPU the slabs can be domains of one batch linked to each other (`Batch.link_x`).
Across devices the cuts are halo edges (`HaloGrid`, lbm_batch_set_halo): every step each
cut exchanges the three populations that cross it (e_x = +1: directions 1, 5, 8 eastward;
e_x = -1: 3, 6, 7 westward) of one column each way, packed on the device, moved by a
device copy, NCCL or gloo.

`split_spec` builds the slab specs, `admit_split` admits and links them, and
`gather_populations` / `scatter_populations` move a whole-grid population array to and
from the slabs. The force on a body is the sum of the slabs' forces.
"""
from __future__ import annotations

import numpy as np

# directions whose populations cross a cut eastward / westward (e_x = +1 / -1)
CROSS_EAST = (1, 5, 8)
CROSS_WEST = (3, 6, 7)


def split_spec(spec, widths):
    """Slab specs of `spec` cut into consecutive column ranges of the given widths.

    The first slab keeps the grid's west edge and the last its east edge; the edges at
    the cuts are linked by `admit_split` (their values in the specs are placeholders
    that the library accepts: an inflow/outflow pair in a channel, periodic otherwise).
    With 16-bit storage every cut must fall on a multiple of 8 columns (the rounding bits
    are keyed by global 8-column groups); the library rejects other origins.
    """
    widths = [int(w) for w in widths]
    if sum(widths) != spec["nx"] or min(widths) < 3:
        raise ValueError(f"widths {widths} must be >= 3 and add up to nx = {spec['nx']}")
    e = spec["edges"]
    periodic = e["west"] == "periodic"
    out, x0 = [], 0
    for k, w in enumerate(widths):
        edges = dict(e)
        if not periodic:
            edges["west"], edges["east"] = "inlet", "outflow"
        sp = dict(spec, nx=w, x_origin=x0 + int(spec.get("x_origin", 0)), edges=edges,
                  name=f"{spec['name']}_slab{k}")
        out.append(sp)
        x0 += w
    return out


def admit_split(batch, spec, widths, nsteps, **kw):
    """Admit the slabs of `spec` into `batch` and link them; returns their slots (west to
    east). A periodic grid is closed into a ring."""
    slabs = split_spec(spec, widths)
    slots = [batch.admit(sp, nsteps=nsteps, **kw) for sp in slabs]
    for a, b in zip(slots, slots[1:]):
        batch.link_x(a, b)
    if spec["edges"]["west"] == "periodic":
        batch.link_x(slots[-1], slots[0])
    return slots


def gather_populations(batch, slots):
    """The whole grid's populations [9, ny, nx] from its slabs."""
    return np.concatenate([batch.get_populations(k) for k in slots], axis=2)


def scatter_populations(batch, slots, arr):
    """Set the slabs' populations from a whole-grid array [9, ny, nx]."""
    x0 = 0
    for k in slots:
        w = batch.mask(k).shape[1]
        batch.set_populations(k, np.ascontiguousarray(arr[:, :, x0:x0 + w]))
        x0 += w


# ---- slabs on several devices: halo edges ----------------------------------------------

# plane indices that leave a slab through its west / east edge (and arrive in the
# neighbour's recv buffer at the same plane indices)
LEAVE_WEST = CROSS_WEST
LEAVE_EAST = CROSS_EAST


def exchange(send_west, send_east, recv_west, recv_east, west, east, group=None):
    """One halo exchange of this rank across its two cuts (torch.distributed point to
    point; CUDA tensors over NCCL, host tensors over gloo). send_west goes to rank `west`,
    which receives it as its east halo; send_east to rank `east`; recv_west / recv_east
    receive the neighbours' buffers. A side whose rank is None is skipped (the grid's own
    edge).

    Every rank posts the eastward transfer (send east, receive from the west) before the
    westward one: transfers between the same two ranks are matched in posting order, and
    in a ring of two ranks both neighbours are the same rank. Over NCCL the four
    transfers form one group (no send waits on a send); all are posted before any is
    waited on."""
    import torch.distributed as dist
    ops = []
    if east is not None:
        ops.append((dist.isend, send_east, east))
    if west is not None:
        ops.append((dist.irecv, recv_west, west))
        ops.append((dist.isend, send_west, west))
    if east is not None:
        ops.append((dist.irecv, recv_east, east))
    if not ops:
        return
    if dist.get_backend(group) == "nccl":
        works = dist.batch_isend_irecv([dist.P2POp(op, t, peer, group) for op, t, peer in ops])
    else:
        works = [op(t, peer, group=group) for op, t, peer in ops]
    for w in works:
        w.wait()


def halo_topology(k, world, periodic):
    """Which rank holds each of k slabs (consecutive blocks of k / world), and for every
    rank the ranks across its westmost and eastmost cuts (None: the grid's own edge or
    a cut inside the rank). A periodic grid closes into a ring."""
    if k % world:
        raise ValueError(f"{k} slabs do not divide over {world} ranks")
    owner = [i * world // k for i in range(k)]

    def nb(i, side):
        j = i - 1 if side == 0 else i + 1
        if 0 <= j < k:
            return j
        return (j % k) if periodic else None

    peers = []
    for r in range(world):
        mine = [i for i in range(k) if owner[i] == r]
        wj, ej = nb(mine[0], 0), nb(mine[-1], 1)
        peers.append((owner[wj] if wj is not None and owner[wj] != r else None,
                      owner[ej] if ej is not None and owner[ej] != r else None))
    return owner, peers


class HaloGrid:
    """One grid as slabs whose cuts are halo edges (lbm_batch_set_halo), this rank's
    share in one batch. slab k of the grid (widths in order, west to east) lives on rank
    k * world // len(widths); before every step the batch packs its halo edges, cuts to
    other ranks exchange by `exchange`, then one step runs. At a cut between two slabs of
    this rank each side reads the other side's send buffer as its recv buffer, so the
    packing is all the exchange there is. A periodic grid is closed into a ring. The
    result is the undivided grid's, bit for bit."""

    def __init__(self, spec, widths, storage="f16s", rank=0, world=1, nsteps=None,
                 force_every=1, force_capacity=8192, graph_steps=0, stream=None):
        import torch
        from . import Batch
        self.spec, self.storage, self.rank, self.world = spec, storage, rank, world
        self.slabs = split_spec(spec, widths)
        k = len(self.slabs)
        self.periodic = spec["edges"]["west"] == "periodic"
        self.owner, peers = halo_topology(k, world, self.periodic)
        self.west_rank, self.east_rank = peers[rank]
        self.mine = [i for i in range(k) if self.owner[i] == rank]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.batch = Batch(storage, max_domains=len(self.mine), graph_steps=graph_steps,
                           stream=self.stream)
        n = spec["steps"] if nsteps is None else int(nsteps)
        self.slots = self.batch.admit_many([self.slabs[i] for i in self.mine], nsteps=n,
                                           force_every=force_every, force_capacity=force_capacity)
        dt = {"f64": torch.float64, "f32": torch.float32}.get(storage, torch.int16)
        ny = spec["ny"]
        # a send buffer per halo edge; a cut inside this rank needs no copy (each side's
        # recv buffer is the other side's send buffer), a cut to another rank a recv buffer
        send = {}
        for i in self.mine:
            for side in (0, 1):
                if self._neighbour(i, side) is not None:
                    send[(i, side)] = torch.zeros((9, ny), dtype=dt, device="cuda")
        self.buf = {}  # (slab, side) -> (recv, send)
        for i, slot in zip(self.mine, self.slots):
            for side in (0, 1):
                j = self._neighbour(i, side)
                if j is None:
                    continue
                local = self.owner[j] == rank
                recv = send[(j, 1 - side)] if local else torch.zeros((9, ny), dtype=dt, device="cuda")
                self.buf[(i, side)] = (recv, send[(i, side)])
                self.batch.set_halo(slot, side, recv, send[(i, side)])

    def _neighbour(self, i, side):
        """The slab across side `side` of slab i, or None at the grid's own edge."""
        k = len(self.slabs)
        j = i - 1 if side == 0 else i + 1
        if 0 <= j < k:
            return j
        return (j % k) if self.periodic else None

    def step(self, n=1):
        import torch
        with torch.cuda.stream(self.stream):
            for _ in range(int(n)):
                self.batch.pack_halos()
                with torch.cuda.nvtx.range("slabs.exchange"):
                    self._exchange()
                self.batch.run(1)

    def _exchange(self):
        # cuts inside this rank read the neighbour's send buffer directly: nothing to move.
        # cuts to other ranks: this rank's westmost and eastmost slabs
        first, last = self.mine[0], self.mine[-1]
        west, east = self.west_rank, self.east_rank
        if west is None and east is None:
            return
        rw, sw = self.buf.get((first, 0), (None, None))
        re_, se = self.buf.get((last, 1), (None, None))
        exchange(sw, se, rw, re_, west, east)

    def populations(self):
        """This rank's slabs' populations side by side [9, ny, sum of widths]."""
        return np.concatenate([self.batch.get_populations(k) for k in self.slots], axis=2)

    def forces(self):
        """The sum over this rank's slabs of the force series drained so far."""
        out = [f for f, _ in self.batch.poll_many(self.slots)]
        return sum(out)

    def close(self):
        self.batch.close()
