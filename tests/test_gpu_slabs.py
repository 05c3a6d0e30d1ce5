"""Slab decomposition of one grid on the GPU (paper_1901_08766_gb300.slabs): the grid run
as linked slabs of one batch (each slab a domain whose cut edges pull the adjacent
column of its neighbour) reproduces the undivided grid bit for bit, for every storage,
uneven widths (different row pitches), every row pipeline, moving bodies crossing a cut,
and a periodic ring of three slabs. The same with every cut a halo edge fed from device
buffers (the form slabs on several GPUs take), exchanged by device copies."""
import numpy as np
import pytest

import codec
import oracle
import synth
from paper_1901_08766_gb300 import slabs

pytestmark = pytest.mark.gpu


def _grid(edges, moving=False):
    e = synth._edges() if edges == "periodic" else synth._edges("inlet", "outflow", "free_slip", "free_slip")
    shapes = [synth._circle(1, 95.3, 30.7, 9.0),  # crosses the cut at column 96
              {"kind": "naca4", "body": 2, "cx": 170.0, "cy": 34.0, "chord": 40.0,
               "thickness": 0.12, "aoa_rad": 0.15}]
    bodies = [synth._body(95.3, 30.7, 18.0, omega=2e-3, vx=0.04 if moving else 0.0),
              synth._body(170.0, 34.0, 40.0, vy=0.01 if moving else 0.0)]
    sp = synth._spec("slabgrid", 250, 64, 0.04, shapes, bodies, 0, 0.03, e, u_in=(0.03, 0.0),
                     u0=(0.03, 0.0))
    sp["moving"] = moving
    return sp


def _run_whole(lbm, spec, storage, g0, steps, tile):
    b = lbm.Batch(storage, max_domains=1, graph_steps=16)
    k = b.admit(spec, nsteps=steps)
    b.set_tile(*tile)
    b.set_populations(k, g0)
    while b.run(steps):
        pass
    f, _ = b.poll(k)
    out = (b.get_populations(k), f, b.mask(k))
    b.close()
    return out


def _run_split(lbm, spec, storage, g0, steps, tile, widths):
    b = lbm.Batch(storage, max_domains=len(widths), graph_steps=16)
    ks = slabs.admit_split(b, spec, widths, nsteps=steps)
    b.set_tile(*tile)
    slabs.scatter_populations(b, ks, g0)
    while b.run(steps):
        pass
    f = sum(b.poll(k)[0] for k in ks)
    out = (slabs.gather_populations(b, ks), f, np.concatenate([b.mask(k) for k in ks], axis=1))
    b.close()
    return out


@pytest.mark.parametrize("storage", ["f64", "f16s"])
@pytest.mark.parametrize("edges", ["periodic", "channel"])
@pytest.mark.parametrize("tile", [(8, 8, 2, 0), (4, 4, 3, 1), (8, 4, 2, 2), (8, 12, 4, 4)],
                         ids=["direct", "tma", "prefetch", "direct24"])
def test_two_slabs_reproduce_the_grid(lbm, storage, edges, tile):
    vec = tile[0] if storage != "f64" else tile[0] // 4
    tile = (vec,) + tile[1:]
    spec = _grid(edges)
    g0 = codec.encode(synth.random_populations(31, 250, 64, 0.05), storage)
    steps = 40
    whole = _run_whole(lbm, spec, storage, g0, steps, tile)
    split = _run_split(lbm, spec, storage, g0, steps, tile, [96, 154])  # pitches 128 and 192
    assert np.array_equal(split[2], whole[2])
    assert np.array_equal(split[0].view(np.uint8), whole[0].view(np.uint8))
    # forces: each slab sums its part of a body; only the summation order differs
    assert np.abs(split[1] - whole[1]).max() <= 1e-12 * np.abs(whole[1]).max()
    if storage == "f64":
        ora = oracle.Domain(spec, g=g0)
        ora.run(steps)
        assert np.max(np.abs(split[0] - ora.g) / np.abs(ora.g)) <= 1e-13


def test_three_slab_ring_with_moving_bodies(lbm):
    spec = _grid("periodic", moving=True)
    g0 = codec.encode(synth.random_populations(32, 250, 64, 0.05), "f16s")
    whole = _run_whole(lbm, spec, "f16s", g0, 60, (8, 8, 2, 0))
    split = _run_split(lbm, spec, "f16s", g0, 60, (8, 8, 2, 0), [80, 88, 82])
    assert np.array_equal(split[2], whole[2])
    assert np.array_equal(split[2], oracle.rasterize(spec, 60))
    assert np.array_equal(split[0].view(np.uint16), whole[0].view(np.uint16))
    assert np.abs(split[1] - whole[1]).max() <= 1e-12 * np.abs(whole[1]).max()


def test_three_slab_ring_with_turning_shapes(lbm):
    # shapes turned with their bodies (moving = 2) across the cuts: the NACA section turns
    # about a centre 6 cells behind its quarter chord and the circle orbits its body's
    # centre, both placed at global columns; the slabs equal the undivided grid bit for bit
    spec = _grid("periodic", moving=True)
    spec["moving"] = 2
    spec["shapes"] = [synth._circle(1, 95.3, 30.7, 9.0), synth._circle(1, 82.0, 30.7, 3.0), spec["shapes"][1]]
    spec["bodies"] = [dict(spec["bodies"][0], omega=0.02),
                      dict(spec["bodies"][1], cx=176.0, omega=-0.008)]
    g0 = codec.encode(synth.random_populations(33, 250, 64, 0.05), "f16s")
    whole = _run_whole(lbm, spec, "f16s", g0, 60, (8, 8, 2, 0))
    split = _run_split(lbm, spec, "f16s", g0, 60, (8, 8, 2, 0), [80, 88, 82])
    assert np.array_equal(split[2], whole[2])
    assert np.array_equal(split[2], oracle.rasterize(spec, 60))
    assert not np.array_equal(whole[2], oracle.rasterize(dict(spec, moving=True), 60))
    assert np.array_equal(split[0].view(np.uint16), whole[0].view(np.uint16))
    assert np.abs(split[1] - whole[1]).max() <= 1e-12 * np.abs(whole[1]).max()
    # pulsating domains are not linked
    pulse = dict(spec, bodies=[dict(spec["bodies"][0], deform={"amplitude": 0.1, "rate": 0.01}), spec["bodies"][1]])
    b = lbm.Batch("f16s", max_domains=3, graph_steps=16)
    with pytest.raises(lbm.LbmError):
        slabs.admit_split(b, pulse, [80, 88, 82], nsteps=10)
    b.close()


def test_16bit_origin_must_be_a_multiple_of_8(lbm):
    spec = dict(_grid("channel"), nx=100, x_origin=97)
    b = lbm.Batch("f16s", max_domains=1, graph_steps=0)
    with pytest.raises(lbm.LbmError):
        b.admit(spec, nsteps=1)
    b.close()


def test_link_checks_and_evict_unlinks(lbm):
    spec = _grid("channel")
    a_spec, b_spec = slabs.split_spec(spec, [120, 130])
    b = lbm.Batch("f32", max_domains=3, graph_steps=0)
    ka = b.admit(a_spec, nsteps=10)
    kb = b.admit(dict(b_spec, ny=40), nsteps=10)
    with pytest.raises(lbm.LbmError):
        b.link_x(ka, kb)  # different ny
    b.evict(kb)
    kb = b.admit(b_spec, nsteps=20)
    with pytest.raises(lbm.LbmError):
        b.link_x(ka, kb)  # different step counts
    b.evict(kb)
    kb = b.admit(b_spec, nsteps=10)
    b.link_x(ka, kb)
    with pytest.raises(lbm.LbmError):
        b.link_x(ka, kb)  # linked already
    b.evict(kb)  # ka's east edge is its own outflow again
    b.run(10)
    f, done = b.poll(ka)
    assert done and np.isfinite(f).all()
    b.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
@pytest.mark.parametrize("edges", ["periodic", "channel"])
def test_halo_edges_reproduce_the_grid(lbm, storage, edges):
    # every cut a halo edge fed from device buffers (lbm_batch_set_halo), packed on the
    # device before each step; inside one batch each side reads the other's packed
    # buffer (ranks on several GPUs move the same buffers by NCCL)
    from paper_1901_08766_gb300 import slabs as sl
    spec = _grid(edges)
    g0 = codec.encode(synth.random_populations(37, 250, 64, 0.05), storage)
    steps = 40
    whole = _run_whole(lbm, spec, storage, g0, steps, {"f64": (2, 8, 2, 0), "f32": (4, 8, 2, 0)}.get(storage, (8, 8, 2, 0)))
    hg = sl.HaloGrid(spec, [96, 64, 90], storage=storage, nsteps=steps, force_capacity=64)
    x0 = 0
    for k, w in zip(hg.slots, (96, 64, 90)):
        hg.batch.set_populations(k, np.ascontiguousarray(g0[:, :, x0:x0 + w]))
        x0 += w
    hg.step(steps)
    got = hg.populations()
    f = hg.forces()
    masks = np.concatenate([hg.batch.mask(k) for k in hg.slots], axis=1)
    hg.close()
    assert np.array_equal(masks, whole[2])
    assert np.array_equal(got.view(np.uint8), whole[0].view(np.uint8))
    assert np.abs(f - whole[1]).max() <= 1e-12 * np.abs(whole[1]).max()
