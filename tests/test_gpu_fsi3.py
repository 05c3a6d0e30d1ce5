"""Coupled bodies in 3D on the GPU (rigid bodies on springs and dampers that move in
response to their force, semi-implicit Euler of the two-step mean force after every step):
FP64 against the oracle on both lattices (populations, forces, body states, masks), the
infinitely heavy limit bit for bit equal to the prescribed motion, checkpoint and resume
bit for bit, FP32 storage following FP64, and the API's guards."""
import math

import numpy as np
import pytest

import synth
from oracle import d3 as ora3

pytestmark = pytest.mark.gpu


def dynamics3(mass, stiffness=(0.0, 0.0, 0.0), damping=(0.0, 0.0, 0.0), free=(1, 1, 1)):
    return {"mass": float(mass), "stiffness": tuple(float(v) for v in stiffness),
            "damping": tuple(float(v) for v in damping), "free": tuple(int(v) for v in free)}


def _coupled3(edges, q, nx=70):
    # a spring-mounted sphere (coupled, launched across the stream) and a prescribed
    # z-cylinder; both stay clear of the walls and of each other over 400 steps
    r = 4.1
    c1, c2 = (20.3, 10.6, 9.7), (44.6, 9.2, 0.0)
    M = 8.0 * 4.0 / 3.0 * math.pi * r ** 3
    b1 = synth.body3(c1, 2 * r, v=(0.0, 0.02, -0.016), w=(0.001, -0.0015, 0.002))
    b1["dynamics"] = dynamics3(M, (0.5, 4.0, 3.0), (0.0, 2.0, 0.0))
    b2 = synth.body3(c2, 5.8, v=(0.02, 0.006, 0.0), w=(0.0, 0.0, 0.003))
    sp = synth.spec3("coupled3", nx, 20, 20, 0.05, [synth.sphere(1, c1, r), synth.cylinder_z(2, c2[0], c2[1], 2.9)],
                     [b1, b2], 0, 0.03, edges, u_in=(0.03, 0.0, 0.0), u0=(0.01, 0.0, 0.0), lattice=q)
    sp["moving"] = True
    return sp


def _start(lbm, spec, storage, seed):
    q = spec.get("lattice", 19)
    g0 = synth.random_populations3(seed, spec["nx"], spec["ny"], spec["nz"], 0.05, q=q)
    dom = lbm.Domain3(spec, storage=storage)
    if storage == "f64":
        dom.set_populations(g0)
    return dom, g0


@pytest.mark.parametrize("q", [19, 15])
@pytest.mark.parametrize("edges", ["periodic", "channel"])
def test_fp64_3d_coupled_matches_oracle(lbm, edges, q):
    e = synth.edges3() if edges == "periodic" else synth.channel_edges3()
    spec = _coupled3(e, q)
    dom, g0 = _start(lbm, spec, "f64", 29)
    ora = ora3.Domain(spec, g=g0)
    fg, fo = [], []
    b2 = spec["bodies"][1]
    for chunk in (1, 99, 300):  # states and masks compared after each chunk
        fg.append(dom.run(chunk))
        fo.append(ora.run(chunk))
        n = ora.steps_done
        st, cs = dom.body_state(), dom.coupled_state()
        assert np.abs(cs[0] - ora.state[0]).max() <= 1e-11 * max(1.0, np.abs(ora.state[0]).max()), \
            f"coupled state after {n} steps"
        assert np.array_equal(st[0, 0:6], cs[0, 0:6]) and np.array_equal(st[0, 6:9], spec["bodies"][0]["w"])
        assert (cs[1] == 0.0).all()
        for d in range(3):  # prescribed body: c + V n
            assert st[1, d] == b2["c"][d] + b2["v"][d] * n
        assert np.array_equal(dom.mask(), ora.mask), f"mask differs after {n} steps"
    assert ((ora.mask == 1) != (ora3.rasterize(spec) == 1)).any()  # the coupled body moved across nodes
    assert np.abs(ora.state[0, 0:3] - np.array(spec["bodies"][0]["c"])).max() > 0.1
    raw = dom.get_populations()
    dom.close()
    rel = np.abs(raw - ora.g) / np.abs(ora.g)
    assert rel.max() <= 1e-12, f"max relative population difference {rel.max():.3e}"
    fg, fo = np.concatenate(fg), np.concatenate(fo)
    assert fg.shape == (400, 2, 3)
    assert np.abs(fg - fo).max() <= 1e-10 * np.abs(fo).max() + 1e-14


@pytest.mark.parametrize("q", [19, 15])
def test_3d_heavy_coupled_body_is_the_prescribed_motion(lbm, q):
    # M = 1e300 launched with V: the velocity never changes and the centre advances by V
    # each step; no node lies within rounding of the shapes here, so the masks and U_O of
    # every step equal the prescribed motion's: the same bits (FP64, same device path)
    V = (0.11, -0.071, 0.053)
    cen = (9.4, 8.2, 7.7)
    shapes = [synth.sphere(1, cen, 3.3), synth.sphere(1, (cen[0] + 2.1, cen[1], cen[2]), 2.2)]
    b = synth.body3(cen, 7.0, v=V)
    pres = synth.spec3("p3", 20, 17, 15, 0.05, shapes, [dict(b)], 0, 0.02, synth.edges3(), lattice=q)
    pres["moving"] = True
    hb = dict(b)
    hb["dynamics"] = dynamics3(1e300)
    heavy = dict(pres, bodies=[hb])
    g0 = synth.random_populations3(23, 20, 17, 15, q=q)
    out = []
    for sp in (pres, heavy):
        d = lbm.Domain3(sp, storage="f64")
        d.set_populations(g0)
        f = d.run(40)
        out.append((d.get_populations(), f, d.mask(), d.body_state()))
        d.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])
    assert np.abs(out[1][3][0, :3] - (np.array(cen) + 40 * np.array(V))).max() < 1e-12


@pytest.mark.parametrize("storage", ["f16s", "f32"])
def test_3d_coupled_checkpoint_resume_is_bit_identical(lbm, storage):
    spec = _coupled3(synth.channel_edges3(), 19)
    a = lbm.Domain3(spec, storage=storage)
    fa = a.run(160)
    b = lbm.Domain3(spec, storage=storage)
    fb1 = b.run(70)
    snap, st = b.get_populations(), b.coupled_state()
    b.close()
    c = lbm.Domain3(spec, storage=storage)
    c.set_populations(snap)
    c.restore_coupled(70, st)
    assert np.array_equal(c.coupled_state(), st)
    fb2 = c.run(90)
    assert np.array_equal(c.get_populations().view(np.uint8), a.get_populations().view(np.uint8))
    assert np.array_equal(np.concatenate([fb1, fb2]), fa)
    assert np.array_equal(c.mask(), a.mask())
    assert np.array_equal(c.body_state(), a.body_state())
    a.close()
    c.close()


def test_3d_coupled_f32_follows_f64(lbm):
    # the spring-mounted sphere in the channel: FP32 storage tracks the FP64 trajectory
    spec = _coupled3(synth.channel_edges3(), 19)
    traj = {}
    for storage in ("f64", "f32"):
        d = lbm.Domain3(spec, storage=storage)
        ys = []
        for _ in range(12):
            d.run(50)
            ys.append(d.body_state()[0, :3].copy())
        traj[storage] = np.array(ys)
        d.close()
    c0 = np.array(spec["bodies"][0]["c"])
    amp = np.abs(traj["f64"] - c0).max()
    err = np.abs(traj["f32"] - traj["f64"]).max()
    assert amp > 0.3 and err < 0.02 * amp, f"amplitude {amp:.4f}, FP32 deviation {err:.3e}"


def test_3d_coupled_guards(lbm):
    spec = _coupled3(synth.edges3(), 19)
    with pytest.raises(lbm.LbmError):  # not moving
        lbm.Domain3(dict(spec, moving=False), storage="f32")
    with pytest.raises(lbm.LbmError):  # forces not recorded every step
        lbm.Domain3(spec, storage="f32", force_every=2)
    bad = dict(spec, bodies=[dict(spec["bodies"][0], dynamics=dynamics3(-1.0)), spec["bodies"][1]])
    with pytest.raises(lbm.LbmError):
        lbm.Domain3(bad, storage="f32")
    d = lbm.Domain3(spec, storage="f32")
    d.run(3)
    with pytest.raises(lbm.LbmError):  # the step index changes only through restore_coupled
        d.set_steps_done(1)
    d.set_steps_done(3)  # the same index is allowed
    with pytest.raises(ValueError):
        d.restore_coupled(3, np.zeros((1, 9)))
    d.close()
    plain = dict(spec, bodies=[dict(b) for b in spec["bodies"]])
    plain["bodies"][0].pop("dynamics")
    p = lbm.Domain3(plain, storage="f32")
    with pytest.raises(lbm.LbmError):
        p.coupled_state()
    p.close()
