"""Pulsating bodies in 3D on the GPU (shapes scaled about the body centre by
s(n) = 1 + a sin(nu n), U_O with the dilation velocity kappa (x - c)): FP64 against the
oracle on both lattices with masks bit for bit at every checked step, checkpoint and
resume bit for bit, and the guards."""
import numpy as np
import pytest

import synth
from oracle import d3 as ora3

pytestmark = pytest.mark.gpu


def _pulsing3(edges, q):
    # a sphere with a smaller one riding beside it, pulsating by 8 %, a sphere pulsating by
    # -6 %, and a rigid z-cylinder (a pulsating body is made of spheres); all translate and
    # stay clear of the walls and of each other. The penalized interior follows the
    # dilation, so its density varies as s^-3: at 25 % it falls below zero within 400 steps
    # (on the oracle and the GPU alike), which the GPU's status check reports
    c1, c2, c3 = (20.3, 10.6, 9.7), (40.6, 9.2, 10.3), (55.0, 10.0, 0.0)
    sp = synth.spec3("pulsing3", 70, 20, 20, 0.05,
                     [synth.sphere(1, c1, 4.1), synth.sphere(1, (26.0, 10.6, 9.7), 1.8),
                      synth.sphere(2, c2, 3.4), synth.cylinder_z(3, c3[0], c3[1], 2.5)],
                     [dict(synth.body3(c1, 8.2, v=(0.02, -0.004, 0.003), w=(0.001, -0.0015, 0.002)),
                           deform={"amplitude": 0.08, "rate": 0.021}),
                      dict(synth.body3(c2, 6.8, v=(0.015, 0.004, 0.0)), deform={"amplitude": -0.06, "rate": 0.033}),
                      synth.body3(c3, 5.0, v=(0.01, 0.0, 0.0))],
                     0, 0.03, edges, u_in=(0.03, 0.0, 0.0), u0=(0.01, 0.0, 0.0), lattice=q)
    sp["moving"] = True
    return sp


@pytest.mark.parametrize("q", [19, 15])
@pytest.mark.parametrize("edges", ["periodic", "channel"])
def test_fp64_3d_pulsating_matches_oracle(lbm, edges, q):
    e = synth.edges3() if edges == "periodic" else synth.channel_edges3()
    spec = _pulsing3(e, q)
    g0 = synth.random_populations3(37, spec["nx"], spec["ny"], spec["nz"], 0.05, q=q)
    dom = lbm.Domain3(spec, storage="f64")
    dom.set_populations(g0)
    ora = ora3.Domain(spec, g=g0)
    assert np.array_equal(dom.mask(), ora.mask)
    fg, fo = [], []
    for chunk in (1, 99, 300):
        fg.append(dom.run(chunk))
        fo.append(ora.run(chunk))
        assert np.array_equal(dom.mask(), ora.mask), f"mask differs after {ora.steps_done} steps"
    assert (ora.mask == 1).sum() != (ora3.rasterize(spec, 0) == 1).sum()  # it does pulsate
    raw = dom.get_populations()
    rel = np.abs(raw - ora.g) / np.abs(ora.g)
    assert rel.max() <= 1e-12, f"max relative population difference {rel.max():.3e}"
    fg, fo = np.concatenate(fg), np.concatenate(fo)
    assert np.abs(fg - fo).max() <= 1e-10 * np.abs(fo).max() + 1e-14
    mg, mo = dom.moments(), ora.moments()
    for a, b in zip(mg[1:], mo[1:]):
        assert np.allclose(a, b, rtol=0, atol=1e-13)
    dom.close()


@pytest.mark.parametrize("storage", ["f16s", "f32"])
def test_3d_pulsating_resume_is_bit_identical(lbm, storage):
    spec = _pulsing3(synth.channel_edges3(), 19)
    a = lbm.Domain3(spec, storage=storage)
    fa = a.run(150)
    b = lbm.Domain3(spec, storage=storage)
    fb1 = b.run(60)
    snap = b.get_populations()
    b.close()
    c = lbm.Domain3(spec, storage=storage)
    c.set_populations(snap)
    c.set_steps_done(60)
    assert np.array_equal(c.mask(), ora3.rasterize(spec, 60))
    fb2 = c.run(90)
    assert np.array_equal(c.get_populations().view(np.uint8), a.get_populations().view(np.uint8))
    assert np.array_equal(np.concatenate([fb1, fb2]), fa)
    assert np.array_equal(c.mask(), a.mask())
    a.close()
    c.close()


def test_3d_pulsating_guards(lbm):
    spec = _pulsing3(synth.edges3(), 19)
    with pytest.raises(lbm.LbmError):  # a fixed mask does not pulsate
        lbm.Domain3(dict(spec, moving=False), storage="f32")
    big = dict(spec, bodies=[dict(spec["bodies"][0], deform={"amplitude": 1.0, "rate": 0.01})] + spec["bodies"][1:])
    with pytest.raises(lbm.LbmError):
        lbm.Domain3(big, storage="f32")
    cyl = dict(spec, bodies=spec["bodies"][:2] + [dict(spec["bodies"][2], deform={"amplitude": 0.1, "rate": 0.01})])
    with pytest.raises(lbm.LbmError):  # a pulsating body is made of spheres
        lbm.Domain3(cyl, storage="f32")
    dyn = {"mass": 1e4, "stiffness": (0.0, 0.0, 0.0), "damping": (0.0, 0.0, 0.0), "free": (1, 1, 1)}
    cpl = dict(spec, bodies=[dict(spec["bodies"][0], dynamics=dyn)] + spec["bodies"][1:])
    with pytest.raises(lbm.LbmError):  # coupled bodies do not deform
        lbm.Domain3(cpl, storage="f32")
