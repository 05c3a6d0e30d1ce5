"""Pins of the 3D oracle's deforming bodies (a body pulsates about its centre: at step
index n its shapes are scaled by s(n) = 1 + a sin(nu n), offsets included, and U_O adds
kappa(n) (x - c), kappa = s'/s), on both lattices, each against something other than the
oracle: the mask against a brute-force numpy rasterisation of the scaled shapes, the
sphere's node count against its volume, the corrected velocity inside a penalized body
against the analytic dilation velocity, zero amplitude bit for bit equal to translation,
and the exact mass and momentum balance."""
import math

import numpy as np
import pytest

import synth
from oracle import d3 as d3

LATTICES = [19, 15]


def _spec(n, shapes, bodies, q=19, eta=1e-4, nu=0.05, lam=3 / 16):
    sp = synth.spec3("deform3_pin", n[0], n[1], n[2], nu, list(shapes), list(bodies), 0, 0.02, synth.edges3(),
                     eta=eta, magic_lambda=lam, lattice=q)
    sp["moving"] = True
    return sp


def _pulsing(body, amplitude, rate):
    return dict(body, deform={"amplitude": float(amplitude), "rate": float(rate)})


def _scale(b, n):
    d = b.get("deform")
    if not d:
        return 1.0, 0.0
    s = 1.0 + d["amplitude"] * math.sin(d["rate"] * n)
    return s, d["amplitude"] * d["rate"] * math.cos(d["rate"] * n) / s


def _brute(spec, n, margin=1e-9):
    nx, ny, nz = spec["nx"], spec["ny"], spec["nz"]
    Z, Y, X = np.meshgrid(np.arange(nz, dtype=float), np.arange(ny, dtype=float), np.arange(nx, dtype=float),
                          indexing="ij")
    ids = np.zeros((nz, ny, nx), dtype=np.uint8)
    near = np.zeros_like(ids, dtype=bool)
    for s in spec["shapes"]:
        b = spec["bodies"][s["body"] - 1]
        sc, _ = _scale(b, n)
        c = [b["c"][d] + b["v"][d] * n + sc * (s["c"][d] - b["c"][d]) for d in range(3)]
        r = sc * s["radius"]
        g = (X - c[0]) ** 2 + (Y - c[1]) ** 2 - r * r
        if s["kind"] == "sphere":
            g = g + (Z - c[2]) ** 2
        ids[g < 0] = s["body"]
        near |= np.abs(g) < margin * r
    return ids, near


@pytest.mark.parametrize("q", LATTICES)
def test_pulsating_mask_is_the_brute_force_mask(q):
    shapes = [synth.sphere(1, (14.3, 12.2, 11.6), 5.0), synth.sphere(1, (21.3, 12.2, 11.6), 2.5),
              synth.sphere(2, (36.0, 13.0, 12.1), 3.5), synth.cylinder_z(3, 44.0, 6.0, 2.0)]
    bodies = [_pulsing(synth.body3((15.3, 12.2, 11.6), 10.0, v=(0.03, -0.01, 0.02)), 0.3, 0.05),
              _pulsing(synth.body3((36.0, 13.0, 12.1), 7.0, v=(-0.02, 0.0, 0.0)), -0.25, 0.08),
              synth.body3((44.0, 6.0, 0.0), 4.0, v=(0.0, 0.01, 0.0))]
    sp = _spec((48, 26, 24), shapes, bodies, q=q)
    for n in (0, 9, 31, 200):
        got = d3.rasterize(sp, n)
        want, near = _brute(sp, n)
        assert np.array_equal(got[~near], want[~near]) and np.array_equal(got, want), f"step {n}"
    assert (d3.rasterize(sp, 31) == 1).sum() > 1.5 * (d3.rasterize(sp, 0) == 1).sum()


def test_pulsating_sphere_volume():
    a, nu = 0.3, 2 * math.pi / 300
    c = (20.25, 19.6, 20.4)
    sp = _spec((40, 40, 40), [synth.sphere(1, c, 10.0)], [_pulsing(synth.body3(c, 20.0), a, nu)])
    for n in range(0, 300, 37):
        r = 10.0 * (1.0 + a * math.sin(nu * n))
        cnt = (d3.rasterize(sp, n) == 1).sum()
        assert abs(cnt - 4.0 / 3.0 * math.pi * r ** 3) <= 0.05 * 4.0 / 3.0 * math.pi * r ** 3


@pytest.mark.parametrize("q", LATTICES)
def test_penalized_interior_moves_with_the_dilation(q):
    a, nu = 0.2, 2 * math.pi / 400
    c = (16.3, 15.6, 14.8)
    b = _pulsing(synth.body3(c, 16.0, v=(0.01, 0.0, 0.0)), a, nu)
    sp = _spec((32, 30, 30), [synth.sphere(1, c, 8.0)], [b], q=q, eta=1e-6)
    dom = d3.Domain(sp, g=synth.random_populations3(3, 32, 30, 30, 0.02, q=q))
    dom.run(57, want_forces=False)
    n = dom.steps_done
    _, kap = _scale(b, n)
    cen = (c[0] + 0.01 * n, c[1], c[2])
    rho, ux, uy, uz = dom.moments()
    K, J, I = np.nonzero(dom.mask == 1)
    assert len(K) > 1000 and abs(kap) > 1e-3
    for u, want in ((ux, 0.01 + kap * (I - cen[0])), (uy, kap * (J - cen[1])), (uz, kap * (K - cen[2]))):
        assert np.abs(u[K, J, I] - want).max() < 1e-6
    assert np.abs(kap * (K - cen[2])).max() > 0.01


@pytest.mark.parametrize("q", LATTICES)
def test_zero_amplitude_is_translation_bit_for_bit(q):
    shapes = [synth.sphere(1, (10.3, 9.2, 8.7), 4.0), synth.cylinder_z(2, 24.0, 10.0, 3.0)]
    rigid = [synth.body3((10.3, 9.2, 8.7), 8.0, v=(0.05, 0.02, -0.03)), synth.body3((24.0, 10.0, 0.0), 6.0, v=(-0.04, 0.0, 0.0))]
    flat = [_pulsing(rigid[0], 0.0, 0.05), rigid[1]]
    g0 = synth.random_populations3(7, 32, 20, 18, q=q)
    a = d3.Domain(_spec((32, 20, 18), shapes, rigid, q=q), g=g0)
    b = d3.Domain(_spec((32, 20, 18), shapes, flat, q=q), g=g0)
    fa, fb = a.run(25), b.run(25)
    assert np.array_equal(a.g, b.g) and np.array_equal(fa, fb) and np.array_equal(a.mask, b.mask)


@pytest.mark.parametrize("q", LATTICES)
def test_pulsating_bodies_conserve_mass_and_balance_momentum(q):
    shapes = [synth.sphere(1, (8.2, 9.1, 7.3), 3.5), synth.sphere(2, (19.5, 8.0, 7.6), 2.5)]
    bodies = [_pulsing(synth.body3((8.2, 9.1, 7.3), 7.0, v=(0.03, 0.01, -0.02)), 0.3, 0.07),
              _pulsing(synth.body3((19.5, 8.0, 7.6), 5.0, w=(0.0, 0.0, 0.02)), -0.3, 0.11)]
    sp = _spec((26, 17, 15), shapes, bodies, q=q, lam=0.25)
    d = d3.Domain(sp, g=synth.random_populations3(5, 26, 17, 15, q=q))
    ex, ey, ez, _, _ = d3.lattice(q)
    E = [np.asarray(e, dtype=float) for e in (ex, ey, ez)]
    m0 = d.g.sum()
    for _ in range(25):
        j0 = [float(np.tensordot(e, d.g, axes=(0, 0)).sum()) for e in E]
        fb = d.run(1)[0]
        j1 = [float(np.tensordot(e, d.g, axes=(0, 0)).sum()) for e in E]
        net = fb.sum(axis=0)
        for c in range(3):
            assert abs((j1[c] - j0[c]) + net[c]) < 1e-14 * d.g[0].size
    assert abs(d.g.sum() - m0) < 1e-12 * m0
    assert (d.mask == 1).sum() != (d3.rasterize(sp, 0) == 1).sum()


def test_oracle_rejects_pulsating_cylinders_and_coupled_pulsation():
    cyl = _spec((20, 16, 12), [synth.cylinder_z(1, 10.0, 8.0, 3.0)],
                [_pulsing(synth.body3((10.0, 8.0, 0.0), 6.0), 0.1, 0.05)])
    with pytest.raises(ValueError):  # isotropic dilation: spheres only
        d3.Domain(cyl)
    b = _pulsing(synth.body3((10.0, 8.0, 6.0), 6.0), 0.1, 0.05)
    b["dynamics"] = {"mass": 1e3, "stiffness": (0.0, 0.0, 0.0), "damping": (0.0, 0.0, 0.0), "free": (1, 1, 1)}
    with pytest.raises(ValueError):  # coupled bodies do not deform
        d3.Domain(_spec((20, 16, 12), [synth.sphere(1, (10.0, 8.0, 6.0), 3.0)], [b]))
    fixed = dict(_spec((20, 16, 12), [synth.sphere(1, (10.0, 8.0, 6.0), 3.0)],
                       [_pulsing(synth.body3((10.0, 8.0, 6.0), 6.0), 0.1, 0.05)]), moving=False)
    with pytest.raises(ValueError):  # a fixed mask does not pulsate
        d3.Domain(fixed)


def test_sincos_against_the_c_library_and_the_2d_oracle():
    import oracle
    for t in np.concatenate([np.linspace(-2e4, 2e4, 40001), np.linspace(-6.5, 6.5, 13001)]):
        s, c = d3.sincos(float(t))
        for mine, ref in ((s, math.sin(t)), (c, math.cos(t))):
            assert abs(mine - ref) <= 2.0 * math.ulp(max(abs(ref), 2.0 ** -60)), (t, mine, ref)
        assert (s, c) == oracle.sincos(float(t))  # the same published method, the same bits
