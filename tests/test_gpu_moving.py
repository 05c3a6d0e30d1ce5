"""Moving obstacles on the GPU (prescribed translation, Sec. 2.2: chi(x, t), U_O(x, t)):
the FP64 mode against the oracle, masks bit for bit at every checked step, batches with
moving and fixed domains, checkpoint resume with the step index."""
import numpy as np
import pytest

import codec
import oracle
import synth

pytestmark = pytest.mark.gpu


def _moving_spec(nx=97, ny=61, edges=None):
    e = edges or synth._edges()
    shapes = [synth._circle(1, 30.3, 28.7, 7.0),
              {"kind": "naca4", "body": 2, "cx": 62.0, "cy": 35.0, "chord": 22.0,
               "thickness": 0.12, "aoa_rad": 0.12}]
    bodies = [synth._body(30.3, 28.7, 14.0, vx=0.037, vy=-0.013, omega=1.5e-3),
              synth._body(62.0, 35.0, 22.0, vx=-0.021, vy=0.008)]
    sp = synth._spec("moving", nx, ny, 0.04, shapes, bodies, 0, 0.03, e, u_in=(0.03, 0.0),
                     u0=(0.01, 0.0))
    sp["moving"] = True
    return sp


@pytest.mark.parametrize("edges", ["periodic", "channel"])
def test_moving_fp64_matches_oracle(lbm, edges):
    e = synth._edges() if edges == "periodic" else synth._edges("inlet", "outflow", "free_slip", "free_slip")
    spec = _moving_spec(edges=e)
    g0 = synth.random_populations(21, spec["nx"], spec["ny"], 0.05)
    dom = lbm.Domain(spec, storage="f64")
    dom.set_populations(g0)
    ora = oracle.Domain(spec, g=g0)
    f_gpu, f_ora = [], []
    for chunk in (1, 99, 300):  # the mask is compared after each chunk
        f_gpu.append(dom.run(chunk))
        f_ora.append(ora.run(chunk))
        assert np.array_equal(dom.mask(), ora.mask), f"mask differs after {ora.steps_done} steps"
    assert not np.array_equal(ora.mask, oracle.rasterize(spec))  # the bodies have moved
    raw = dom.get_populations()
    rel = np.abs(raw - ora.g) / np.abs(ora.g)
    assert rel.max() <= 1e-12, f"max relative population difference {rel.max():.3e}"
    fg, fo = np.concatenate(f_gpu), np.concatenate(f_ora)
    assert np.abs(fg - fo).max() <= 1e-10 * np.abs(fo).max() + 1e-14
    r_g, ux_g, uy_g = dom.moments()
    r_o, ux_o, uy_o = ora.moments()
    assert np.allclose(ux_g, ux_o, rtol=0, atol=1e-13) and np.allclose(uy_g, uy_o, rtol=0, atol=1e-13)
    dom.close()


def test_moving_domain_alone_equals_in_a_mixed_batch(lbm):
    # FP16-shifted: a moving domain gives the same bits alone and batched with fixed
    # domains, for two tile shapes and with CUDA graphs
    moving = _moving_spec()
    fixed = synth.parity_case("channel_97x61")
    g0 = codec.encode(synth.random_populations(5, moving["nx"], moving["ny"], 0.05), "f16s")
    out = []
    for others, tile, graph in [(0, (8, 8, 2, 0), 0), (2, (4, 4, 3, 0), 16), (1, (8, 16, 1, 0), 7), (1, (8, 12, 4, 4), 16), (0, (4, 5, 2, 3), 0)]:
        b = lbm.Batch("f16s", max_domains=4, graph_steps=graph)
        ks = [b.admit(fixed, nsteps=90) for _ in range(others)]
        k = b.admit(moving, nsteps=90)
        b.set_tile(*tile)
        b.set_populations(k, g0)
        while b.run(40):
            pass
        f, done = b.poll(k)
        assert done
        out.append((b.get_populations(k).view(np.uint16).copy(), f, b.mask(k)))
        for q in ks:
            b.poll(q)
        b.close()
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0]) and np.array_equal(o[1], out[0][1])
        assert np.array_equal(o[2], out[0][2])
    assert np.array_equal(out[0][2], oracle.rasterize(moving, 90))


def test_moving_checkpoint_resume(lbm):
    spec = _moving_spec()
    a = lbm.Domain(spec, storage="f16s")
    fa = a.run(120)
    b = lbm.Domain(spec, storage="f16s")
    fb1 = b.run(50)
    snap = b.get_populations()
    b.close()
    c = lbm.Domain(spec, storage="f16s")
    c.set_populations(snap)
    c.set_steps_done(50)  # also moves the bodies and the mask to step index 50
    assert np.array_equal(c.mask(), oracle.rasterize(spec, 50))
    fb2 = c.run(70)
    assert np.array_equal(c.get_populations().view(np.uint16), a.get_populations().view(np.uint16))
    assert np.array_equal(np.concatenate([fb1, fb2]), fa)
    a.close()
    c.close()


def test_moving_rejects_host_mask_and_too_many_bodies(lbm):
    spec = _moving_spec()
    with pytest.raises(lbm.LbmError):
        lbm.Domain(spec, storage="f32", mask=oracle.rasterize(spec))
    many = dict(spec, bodies=[synth._body(10 + 5 * k, 10, 2.0) for k in range(9)],
                shapes=[synth._circle(k + 1, 10 + 5 * k, 10, 1.5) for k in range(9)])
    with pytest.raises(lbm.LbmError):
        lbm.Domain(many, storage="f32")


def test_towing_tank_equals_wind_tunnel(lbm):
    # Galilean equivalence (periodic box, no driving force): a cylinder towed at -U
    # through fluid at rest feels the drag of a fixed cylinder in a uniform stream U. The
    # continuous problems are the same; the lattice (D2Q9, O(u^3) Galilean error, the
    # staircase mask moving by 0.05 cell per step) keeps the mean drag over steps
    # 1000..3000 within 2 % (measured 0.3 %).
    U, D, re = 0.05, 20.0, 100.0
    nu = U * D / re
    e = synth._edges()
    fixed = synth._spec("tunnel", 320, 160, nu, [synth._circle(1, 90.0, 80.5, D / 2)],
                        [synth._body(90.0, 80.5, D)], 0, U, e, u0=(U, 0.0))
    towed = synth._spec("tank", 320, 160, nu, [synth._circle(1, 240.0, 80.5, D / 2)],
                        [synth._body(240.0, 80.5, D, vx=-U)], 0, U, e, u0=(0.0, 0.0))
    towed["moving"] = True
    drag = {}
    for name, sp in (("fixed", fixed), ("towed", towed)):
        dom = lbm.Domain(sp, storage="f32")
        f = dom.run(3000)[:, 0]
        dom.close()
        drag[name] = f[1000:, 0].mean()
    print(f"mean drag: fixed {drag['fixed']:.6f}, towed {drag['towed']:.6f}")
    assert drag["fixed"] > 0 and drag["towed"] > 0
    assert abs(drag["towed"] - drag["fixed"]) / drag["fixed"] < 0.02
