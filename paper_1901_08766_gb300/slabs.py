"""Slab decomposition of one grid along x.

A grid too large for one device, or one that should spread over several, is cut into
slabs of whole columns. Each slab is a domain of its own whose `x_origin` is its first
global column (so shapes are rasterised, and obstacle velocities evaluated, at global
positions) and whose x edges at the cuts are linked: streaming across a cut (Eq.
streaming) pulls the adjacent column of the neighbouring slab at the same time level.
Here the slabs are domains of one batch on one GPU (`Batch.link_x`); on several devices
the same cut exchanges, every step, the three populations that cross it (e_x = +1:
directions 1, 5, 8 eastward; e_x = -1: 3, 6, 7 westward) of one column each way.

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
