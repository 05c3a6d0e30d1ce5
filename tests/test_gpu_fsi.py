"""Coupled bodies on the GPU (fluid-structure coupling: rigid bodies on springs and
dampers that move in response to their force, semi-implicit Euler after every step): the
FP64 mode against the oracle (populations, forces, body states, masks), the infinitely
heavy limits bit for bit equal to fixed and prescribed motion, batches, and the API's
guards."""
import math

import numpy as np
import pytest

import codec
import oracle
import synth

pytestmark = pytest.mark.gpu


def _coupled_spec(edges="periodic", nx=97, ny=61):
    e = synth._edges() if edges == "periodic" else synth._edges("inlet", "outflow", "free_slip", "free_slip")
    r1, r2 = 7.0, 5.5
    b1 = synth._body(30.3, 28.7, 2 * r1, vx=0.0, vy=0.01, omega=1e-3)
    b1["dynamics"] = synth.dynamics(15.0 * math.pi * r1 * r1, (0.02, 0.4), (0.0, 0.5), free=(1, 1))
    b2 = synth._body(66.0, 33.0, 2 * r2, vx=-0.012, vy=0.004)  # prescribed motion
    shapes = [synth._circle(1, 30.3, 28.7, r1), synth._circle(2, 66.0, 33.0, r2)]
    sp = synth._spec("coupled", nx, ny, 0.04, shapes, [b1, b2], 0, 0.03, e, u_in=(0.03, 0.0),
                     u0=(0.01, 0.0))
    sp["moving"] = True
    return sp


@pytest.mark.parametrize("edges", ["periodic", "channel"])
def test_coupled_fp64_matches_oracle(lbm, edges):
    spec = _coupled_spec(edges)
    g0 = synth.random_populations(31, spec["nx"], spec["ny"], 0.05)
    dom = lbm.Domain(spec, storage="f64")
    dom.set_populations(g0)
    ora = oracle.Domain(spec, g=g0)
    f_gpu, f_ora = [], []
    for chunk in (1, 199, 800):  # states and masks compared after each chunk
        f_gpu.append(dom.run(chunk))
        f_ora.append(ora.run(chunk))
        st = dom.body_state()
        # coupled body: the integrated state; prescribed body: c + V n
        assert np.abs(st[0, :4] - ora.state[0, :4]).max() <= 1e-11, f"body state after {ora.steps_done} steps"
        b2 = spec["bodies"][1]
        n = ora.steps_done
        assert st[1, 0] == b2["cx"] + b2["vx"] * n and st[1, 1] == b2["cy"] + b2["vy"] * n
        assert np.array_equal(dom.mask(), ora.mask), f"mask differs after {ora.steps_done} steps"
    # the coupled body has moved across nodes
    assert ((ora.mask == 1) != (oracle.rasterize(spec) == 1)).any()
    raw = dom.get_populations()
    rel = np.abs(raw - ora.g) / np.abs(ora.g)
    assert rel.max() <= 1e-12, f"max relative population difference {rel.max():.3e}"
    fg, fo = np.concatenate(f_gpu), np.concatenate(f_ora)
    assert fg.shape == (1000, 2, 2)
    assert np.abs(fg - fo).max() <= 1e-10 * np.abs(fo).max() + 1e-14
    dom.close()


def test_heavy_coupled_body_is_fixed_and_prescribed_motion(lbm):
    # M = 1e300: at rest it is the fixed body, launched with V it is the prescribed
    # motion c + V n, bit for bit (FP64, same device path for both)
    for V in ((0.0, 0.0), (0.013, -0.0071)):
        b = synth._body(22.4, 19.7, 10.0, vx=V[0], vy=V[1])
        pres = synth._spec("p", 64, 48, 0.05, [synth._circle(1, 22.4, 19.7, 5.1)], [dict(b)], 0, 0.02,
                           synth._edges())
        pres["moving"] = True
        hb = dict(b)
        hb["dynamics"] = synth.dynamics(1e300)
        heavy = dict(pres, bodies=[hb])
        g0 = synth.random_populations(23, 64, 48)
        out = []
        for sp in (pres, heavy):
            d = lbm.Domain(sp, storage="f64")
            d.set_populations(g0)
            f = d.run(400)
            out.append((d.get_populations(), f, d.mask(), d.body_state()))
            d.close()
        assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
        assert np.array_equal(out[0][2], out[1][2])
        assert np.abs(out[1][3][0, :2] - (np.array([22.4, 19.7]) + 400 * np.array(V))).max() < 1e-12


def test_coupled_domain_alone_equals_in_a_mixed_batch(lbm):
    # FP16-shifted: the same bits alone and batched with fixed and prescribed-moving
    # domains, with and without CUDA graphs
    spec = _coupled_spec("channel")
    fixed = synth.parity_case("channel_97x61")
    moving = dict(_coupled_spec("channel"))
    moving["bodies"] = [dict(b) for b in moving["bodies"]]
    moving["bodies"][0].pop("dynamics")
    g0 = codec.encode(synth.random_populations(5, spec["nx"], spec["ny"], 0.05), "f16s")
    out = []
    for others, graph in [(0, 0), (2, 16), (1, 7)]:
        b = lbm.Batch("f16s", max_domains=4, graph_steps=graph)
        ks = [b.admit(fixed if q % 2 == 0 else moving, nsteps=90) for q in range(others)]
        k = b.admit(spec, nsteps=90)
        b.set_populations(k, g0)
        while b.run(40):
            pass
        f, done = b.poll(k)
        assert done
        out.append((b.get_populations(k).view(np.uint16).copy(), f, b.mask(k), b.body_state(k)))
        for q in ks:
            b.poll(q)
        b.close()
    for o in out[1:]:
        for x, y in zip(o, out[0]):
            assert np.array_equal(x, y)


def test_coupled_fp16s_follows_fp64(lbm):
    # a spring-mounted cylinder in a channel released with a transverse velocity: the
    # 16-bit storage tracks the FP64 trajectory over 3000 steps
    spec = _coupled_spec("channel", nx=160, ny=80)
    traj = {}
    for st in ("f64", "f16s"):
        d = lbm.Domain(spec, storage=st)
        ys = []
        for _ in range(30):
            d.run(100)
            ys.append(d.body_state()[0, 1])
        traj[st] = np.array(ys)
        d.close()
    amp = np.abs(traj["f64"] - 28.7).max()
    assert amp > 0.3
    assert np.abs(traj["f16s"] - traj["f64"]).max() < 0.02 * amp


def test_coupled_api_guards(lbm):
    spec = _coupled_spec()
    fixed = dict(spec, moving=False)
    with pytest.raises(lbm.LbmError):  # not a moving domain
        lbm.Domain(fixed, storage="f32")
    with pytest.raises(lbm.LbmError):  # forces not recorded every step
        lbm.Domain(spec, storage="f32", force_every=2)
    bad = dict(spec, bodies=[dict(spec["bodies"][0], dynamics=synth.dynamics(-1.0)), spec["bodies"][1]])
    with pytest.raises(lbm.LbmError):
        lbm.Domain(bad, storage="f32")
    d = lbm.Domain(spec, storage="f32")
    d.run(5)
    from paper_1901_08766_gb300 import _native
    import ctypes as C
    dyn = _native.dynamics_from(synth.dynamics(100.0))
    assert lbm.load().lbm_set_dynamics(d._handle(), 1, C.byref(dyn)) == _native.LBM_EINVAL  # after stepping
    with pytest.raises(lbm.LbmError):
        d.set_steps_done(2)  # the geometry is state
    d.set_steps_done(5)  # the current index is accepted
    assert d.steps_done() == 5
    d.close()
    b = lbm.Batch("f32", max_domains=2)
    k1 = b.admit(spec, nsteps=10)
    k2 = b.admit(dict(spec, bodies=[dict(x) for x in spec["bodies"]]), nsteps=10)
    with pytest.raises(lbm.LbmError):
        b.link_x(k1, k2)
    b.close()


@pytest.mark.parametrize("storage", ["f64", "f16s"])
def test_coupled_checkpoint_resume_is_bit_identical(lbm, storage):
    # populations, step index and coupled state saved after 50 steps: the resumed run
    # repeats the uninterrupted one bit for bit (states, masks, forces, populations)
    spec = _coupled_spec("channel")
    a = lbm.Domain(spec, storage=storage)
    fa = a.run(120)
    b = lbm.Domain(spec, storage=storage)
    fb1 = b.run(50)
    pops, state = b.get_populations(), b.coupled_state()
    b.close()
    assert state[1].tolist() == [0.0] * 6  # the prescribed body has no coupled state
    c = lbm.Domain(spec, storage=storage)
    c.set_populations(pops)
    c.restore_coupled(50, state)
    fb2 = c.run(70)
    assert c.steps_done() == 120
    assert np.array_equal(c.get_populations().view(np.uint8), a.get_populations().view(np.uint8))
    assert np.array_equal(np.concatenate([fb1, fb2]), fa)
    assert np.array_equal(c.body_state(), a.body_state())
    assert np.array_equal(c.mask(), a.mask())
    with pytest.raises(lbm.LbmError):
        c.restore_coupled(-1, state)  # not a step index
    a.close()
    c.close()
