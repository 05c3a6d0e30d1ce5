"""3D GPU path (D3Q19 and D3Q15) vs the FP64 3D oracle, element by element, through the
C ABI.

FP64 storage must match the oracle to 1e-12 relative per population after 1000 steps
(every edge rule, moving and rotating bodies, several strips per row and a ragged
tail); the reduced storages are checked one step at a time within one unit of the
stored type (the rest population also carries the rounding residuals of the moving
ones); the sphere/cylinder mask must be bit-exact.
"""
import numpy as np
import pytest

import codec
import synth
from oracle import d3 as ora3

pytestmark = pytest.mark.gpu


def _case(name, q=19):
    sp = _case19(name)
    sp["lattice"] = q
    return sp


def _case19(name):
    if name == "sphere_channel_150x20x12":
        c = (40.3, 9.6, 5.7)
        return synth.spec3(name, 150, 20, 12, 0.04, [synth.sphere(1, c, 4.3)], [synth.body3(c, 8.6)],
                           0, 0.05, synth.channel_edges3(), u_in=(0.05, 0.0, 0.0), u0=(0.05, 0.0, 0.0))
    if name == "periodic_bodies_97x18x14":
        c1, c2 = (30.2, 8.7, 6.4), (70.6, 9.3, 0.0)
        return synth.spec3(name, 97, 18, 14, 0.1,
                           [synth.sphere(1, c1, 4.6), synth.cylinder_z(2, c2[0], c2[1], 3.2)],
                           [synth.body3(c1, 9.2, v=(0.01, -0.005, 0.003), w=(0.001, -0.002, 0.0015)),
                            synth.body3(c2, 6.4, v=(-0.004, 0.002, 0.0), w=(0.0, 0.0, 0.003))],
                           0, 0.01, synth.edges3(), magic_lambda=0.25)
    if name == "slip_y_periodic_z_70x16x22":
        c = (20.5, 7.5, 0.0)
        e = synth.edges3("periodic", "periodic", "free_slip", "free_slip", "periodic", "periodic")
        return synth.spec3(name, 70, 16, 22, 0.02, [synth.cylinder_z(1, c[0], c[1], 3.7)],
                           [synth.body3(c, 7.4)], 0, 0.02, e, u0=(0.02, 0.0, 0.01))
    if name == "inlet_periodic_y_slip_z_261x10x9":
        c = (60.4, 5.2, 4.1)
        e = synth.edges3("inlet", "outflow", "periodic", "periodic", "free_slip", "free_slip")
        return synth.spec3(name, 261, 10, 9, 0.05, [synth.sphere(1, c, 3.1)], [synth.body3(c, 6.2)], 0,
                           0.04, e, u_in=(0.04, 0.003, -0.002), u0=(0.04, 0.0, 0.0), eta=1e-6)
    raise KeyError(name)


CASES = ["sphere_channel_150x20x12", "periodic_bodies_97x18x14", "slip_y_periodic_z_70x16x22",
         "inlet_periodic_y_slip_z_261x10x9"]


def _start(lbm, spec, storage, seed):
    g0 = synth.random_populations3(seed, spec["nx"], spec["ny"], spec["nz"], 0.1, q=ora3.nq(spec))
    raw0 = codec.encode(g0, storage)
    dom = lbm.Domain3(spec, storage=storage)
    dom.set_populations(raw0)
    return dom, codec.decode(raw0, storage)


@pytest.mark.parametrize("q", [19, 15])
@pytest.mark.parametrize("case", CASES)
def test_fp64_3d_matches_oracle_1000_steps(lbm, case, q):
    spec = _case(case, q)
    dom, g0 = _start(lbm, spec, "f64", 11)
    f_gpu = dom.run(1000)
    raw = dom.get_populations()
    dom.close()
    ora = ora3.Domain(spec, g=g0)
    f_ora = ora.run(1000)
    rel = np.abs(raw - ora.g) / np.abs(ora.g)
    assert rel.max() <= 1e-12, f"max relative population difference {rel.max():.3e}"
    assert f_gpu.shape == f_ora.shape == (1000, len(spec["bodies"]), 3)
    scale = np.abs(f_ora).max()
    assert np.abs(f_gpu - f_ora).max() <= 1e-10 * scale + 1e-14


@pytest.mark.parametrize("case", CASES)
def test_3d_mask_bit_exact(lbm, case):
    spec = _case(case)
    dom = lbm.Domain3(spec, storage="f32")
    m = dom.mask()
    dom.close()
    want = ora3.rasterize(spec)
    assert m.sum() > 0
    np.testing.assert_array_equal(m, want)


def test_3d_initial_state_and_moments(lbm):
    spec = _case("periodic_bodies_97x18x14")
    dom, g0 = _start(lbm, spec, "f64", 5)
    dom.step(3)
    rho, ux, uy, uz = dom.moments()
    raw = dom.get_populations()
    dom.close()
    ora = ora3.Domain(spec, g=g0)
    ora.run(3, want_forces=False)
    np.testing.assert_allclose(raw, ora.g, rtol=1e-13, atol=0)
    for a, b in zip((rho, ux, uy, uz), ora.moments()):
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-15)
    # a fresh domain starts from f^eq(rho0, u0)
    spec = _case("slip_y_periodic_z_70x16x22")
    dom = lbm.Domain3(spec, storage="f64")
    g = dom.get_populations()
    dom.close()
    np.testing.assert_allclose(g, ora3.Domain(spec).g, rtol=1e-15, atol=0)


@pytest.mark.parametrize("q", [19, 15])
@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("case", ["sphere_channel_150x20x12", "periodic_bodies_97x18x14"])
def test_reduced_storage_one_step(lbm, storage, case, q):
    spec = _case(case, q)
    dom, g0 = _start(lbm, spec, storage, 3)
    dom.step(1)
    got = codec.decode(dom.get_populations(), storage)
    dom.close()
    ora = ora3.Domain(spec, g=g0)
    ora.step_once()
    tol = codec.step_tol(ora.g, storage, spec)
    err = np.abs(got - ora.g)
    assert (err <= tol).all(), f"worst excess {(err - tol).max():.3e} at {np.unravel_index(np.argmax(err - tol), err.shape)}"


@pytest.mark.parametrize("q", [19, 15])
@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_reduced_storage_200_steps_drift(lbm, storage, q):
    # over many steps the reduced storages stay close to the FP64 oracle: bound the
    # velocity error at 1 percent of the inflow speed and the density error at 1e-4
    spec = _case("sphere_channel_150x20x12", q)
    dom, g0 = _start(lbm, spec, storage, 9)
    dom.step(200)
    rho, ux, uy, uz = dom.moments()
    dom.close()
    ora = ora3.Domain(spec, g=g0)
    ora.run(200, want_forces=False)
    r, x, y, z = ora.moments()
    assert np.abs(rho - r).max() < 1e-4
    for a, b in ((ux, x), (uy, y), (uz, z)):
        assert np.abs(a - b).max() < 0.01 * spec["U"]


def test_3d_divergence_reported(lbm):
    spec = _case("periodic_bodies_97x18x14", 15)
    dom = lbm.Domain3(spec, storage="f64")
    dom.set_populations(np.zeros((15, spec["nz"], spec["ny"], spec["nx"])))
    dom.step(1)
    with pytest.raises(lbm.LbmError) as e:
        dom.forces()
    assert e.value.status == 4
    dom.close()


def test_3d_force_ring_and_steps(lbm):
    spec = _case("sphere_channel_150x20x12")
    dom = lbm.Domain3(spec, storage="f32", force_every=2, force_capacity=4)
    dom.step(8)
    with pytest.raises(lbm.LbmError) as e:
        dom.step(2)  # a fifth undrained entry
    assert e.value.status == 6
    f = dom.forces()
    assert f.shape == (4, 1, 3) and np.isfinite(f).all()
    assert dom.steps_done() == 8
    assert f[-1, 0, 0] != 0.0
    dom.close()


@pytest.mark.parametrize("q", [19, 15])
@pytest.mark.parametrize("shape,edges", [
    ((3, 3, 3), synth.edges3()),
    ((5, 4, 3), synth.edges3("periodic", "periodic", "free_slip", "free_slip", "free_slip", "free_slip")),
    ((7, 3, 5), synth.channel_edges3()),
    ((129, 3, 4), synth.edges3("inlet", "outflow", "periodic", "periodic", "free_slip", "free_slip")),
])
def test_fp64_3d_degenerate_sizes(lbm, shape, edges, q):
    # smallest grids (one strip, both x edges in one lane, y/z of three cells, a strip of
    # one node past a whole strip) with a sphere covering part of the box
    nx, ny, nz = shape
    c = (nx / 2.0 - 0.3, ny / 2.0 - 0.2, nz / 2.0 + 0.1)
    spec = synth.spec3("tiny", nx, ny, nz, 0.05, [synth.sphere(1, c, 1.3)],
                       [synth.body3(c, 2.6, v=(0.01, 0.0, 0.0), w=(0.0, 0.002, 0.0))], 0, 0.02, edges,
                       u_in=(0.02, 0.0, 0.0), u0=(0.02, 0.0, 0.0), lattice=q)
    dom, g0 = _start(lbm, spec, "f64", 21)
    f_gpu = dom.run(200)
    raw = dom.get_populations()
    dom.close()
    ora = ora3.Domain(spec, g=g0)
    f_ora = ora.run(200)
    np.testing.assert_array_equal(ora.mask, ora3.rasterize(spec))
    rel = np.abs(raw - ora.g) / np.abs(ora.g)
    assert rel.max() <= 1e-12
    assert np.abs(f_gpu - f_ora).max() <= 1e-10 * max(np.abs(f_ora).max(), 1e-30) + 1e-14


@pytest.mark.parametrize("q", [19, 15])
def test_3d_empty_geometry_and_no_forces(lbm, q):
    # no shapes and no bodies: a force-free periodic box; no force entries recorded
    spec = synth.spec3("empty", 40, 6, 5, 0.1, [], [], 0, 0.01, synth.edges3(), u0=(0.01, 0.0, 0.0), lattice=q)
    dom, g0 = _start(lbm, spec, "f64", 4)
    f = dom.run(50)
    raw = dom.get_populations()
    assert dom.mask().sum() == 0
    dom.close()
    assert f.shape == (50, 0, 3)
    ora = ora3.Domain(spec, g=g0)
    ora.run(50, want_forces=False)
    assert (np.abs(raw - ora.g) / np.abs(ora.g)).max() <= 1e-12


@pytest.mark.parametrize("storage,q", [("f16s", 19), ("bf16s", 19), ("f32", 19), ("f16s", 15)])
def test_3d_checkpoint_resume_is_bit_identical(lbm, storage, q):
    # a run interrupted after 30 steps and resumed from its populations and step index
    # repeats the uninterrupted run bit for bit (the 16-bit rounding bits follow the step)
    spec = _case("sphere_channel_150x20x12", q)
    a = lbm.Domain3(spec, storage=storage)
    fa = a.run(70)
    b = lbm.Domain3(spec, storage=storage)
    fb1 = b.run(30)
    snap = b.get_populations()
    b.close()
    c = lbm.Domain3(spec, storage=storage)
    c.set_populations(snap)
    c.set_steps_done(30)
    fb2 = c.run(40)
    assert c.steps_done() == 70
    assert np.array_equal(c.get_populations().view(np.uint8), a.get_populations().view(np.uint8))
    assert np.array_equal(np.concatenate([fb1, fb2]), fa)
    a.close()
    c.close()


@pytest.mark.parametrize("q", [19, 15])
@pytest.mark.parametrize("storage", ["f16s", "bf16s", "f32"])
def test_3d_register_budgets_give_the_same_bits(lbm, storage, q):
    # every register budget (16, 20, 24 resident warps for 16-bit storage) and the autotuner
    # step the same bits, bodies and ragged strips included; the autotuner leaves the
    # state as it was
    spec = _case("periodic_bodies_97x18x14", q)
    pipes = [0, 3, 4] if storage != "f32" else [0]
    g0 = codec.encode(synth.random_populations3(17, spec["nx"], spec["ny"], spec["nz"], 0.05, q=q), storage)
    out = []
    for pipe in pipes + ["auto"]:
        d = lbm.Domain3(spec, storage=storage)
        d.set_populations(g0)
        if pipe == "auto":
            before = d.get_populations().view(np.uint8).copy()
            us = d.autotune(reps=2)
            assert us > 0 and d.get_tile() in pipes
            assert np.array_equal(d.get_populations().view(np.uint8), before)
        else:
            d.set_tile(pipe)
            assert d.get_tile() == pipe
        f = d.run(60)
        out.append((d.get_populations().view(np.uint8).copy(), f))
        d.close()
    for x, fx in out[1:]:
        assert np.array_equal(x, out[0][0]) and np.array_equal(fx, out[0][1])
    d = lbm.Domain3(spec, storage=storage)
    assert d.get_tile() == (3 if storage != "f32" and q == 15 else 0)  # the measured default
    with pytest.raises(lbm.LbmError):
        d.set_tile(2)
    if storage == "f32":
        with pytest.raises(lbm.LbmError):
            d.set_tile(4)
    d.close()


def _moving3(edges, q):
    # bodies stay clear of the domain edges and of each other over 400 steps (a body pushed
    # into a wall or across a periodic edge, or two bodies overlapping, is outside the
    # model: positions are not wrapped and rigid bodies do not collide)
    c1, c2 = (20.3, 10.6, 9.7), (44.6, 9.2, 0.0)
    sp = synth.spec3("moving3", 70, 20, 20, 0.05,
                     [synth.sphere(1, c1, 4.1), synth.cylinder_z(2, c2[0], c2[1], 2.9)],
                     [synth.body3(c1, 8.2, v=(0.035, -0.006, 0.005), w=(0.001, -0.0015, 0.002)),
                      synth.body3(c2, 5.8, v=(0.02, 0.006, 0.0), w=(0.0, 0.0, 0.003))],
                     0, 0.03, edges, u_in=(0.03, 0.0, 0.0), u0=(0.01, 0.0, 0.0), lattice=q)
    sp["moving"] = True
    return sp


@pytest.mark.parametrize("q", [19, 15])
@pytest.mark.parametrize("edges", ["periodic", "channel"])
def test_fp64_3d_moving_matches_oracle(lbm, edges, q):
    e = synth.edges3() if edges == "periodic" else synth.channel_edges3()
    spec = _moving3(e, q)
    dom, g0 = _start(lbm, spec, "f64", 17)
    ora = ora3.Domain(spec, g=g0)
    fg, fo = [], []
    for chunk in (1, 99, 300):  # masks compared after each chunk
        fg.append(dom.run(chunk))
        fo.append(ora.run(chunk))
        assert np.array_equal(dom.mask(), ora.mask), f"mask differs after {ora.steps_done} steps"
    assert not np.array_equal(ora.mask, ora3.rasterize(spec))  # the bodies have moved
    raw = dom.get_populations()
    dom.close()
    rel = np.abs(raw - ora.g) / np.abs(ora.g)
    assert rel.max() <= 1e-12, f"max relative population difference {rel.max():.3e}"
    fg, fo = np.concatenate(fg), np.concatenate(fo)
    assert fg.shape == (400, 2, 3)
    assert np.abs(fg - fo).max() <= 1e-10 * np.abs(fo).max() + 1e-14


@pytest.mark.parametrize("storage", ["f16s", "f32"])
def test_3d_moving_checkpoint_resume_is_bit_identical(lbm, storage):
    spec = _moving3(synth.channel_edges3(), 19)
    a = lbm.Domain3(spec, storage=storage)
    fa = a.run(90)
    b = lbm.Domain3(spec, storage=storage)
    fb1 = b.run(40)
    snap = b.get_populations()
    b.close()
    c = lbm.Domain3(spec, storage=storage)
    c.set_populations(snap)
    c.set_steps_done(40)  # also the mask and centres of index 40
    assert np.array_equal(c.mask(), ora3.rasterize(spec, 40))
    fb2 = c.run(50)
    assert np.array_equal(c.get_populations().view(np.uint8), a.get_populations().view(np.uint8))
    assert np.array_equal(np.concatenate([fb1, fb2]), fa)
    assert np.array_equal(c.mask(), a.mask())
    a.close()
    c.close()


def test_3d_moving_rejects_fast_or_too_many_bodies(lbm):
    spec = _moving3(synth.edges3(), 19)
    fast = dict(spec, bodies=[dict(spec["bodies"][0], v=(1.5, 0.0, 0.0)), spec["bodies"][1]])
    with pytest.raises(lbm.LbmError):
        lbm.Domain3(fast, storage="f32")
    many = dict(spec, bodies=[spec["bodies"][0]] * 9)
    with pytest.raises(lbm.LbmError):
        lbm.Domain3(many, storage="f32")
