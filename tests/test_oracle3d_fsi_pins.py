"""Pins of the 3D oracle's fluid-structure coupling (a body that moves in response to its
force: semi-implicit Euler of M dv/dt = F - k (x - x0) - c v per free axis after every
step, F the mean of the last two steps' forces), each against something other than the
oracle: the exact momentum invariant of fluid plus body in a closed box, the closed-form
discrete damped oscillator when the fluid force vanishes, bit-identity with the fixed and
the prescribed motion for an infinitely heavy body, and boundedness for a light body."""
import math

import numpy as np
import pytest

import synth
from oracle import d3 as d3

LATTICES = [19, 15]


def dynamics3(mass, stiffness=(0.0, 0.0, 0.0), damping=(0.0, 0.0, 0.0), free=(1, 1, 1)):
    return {"mass": float(mass), "stiffness": tuple(float(v) for v in stiffness),
            "damping": tuple(float(v) for v in damping), "free": tuple(int(v) for v in free)}


def _box(n, body, shapes, eta=1e-4, nu=0.05, q=19):
    sp = synth.spec3("fsi3_pin", n[0], n[1], n[2], nu, shapes, [body], 0, 0.02, synth.edges3(),
                     eta=eta, lattice=q)
    sp["moving"] = True
    return sp


def _momentum(g):
    ex, ey, ez, _, _ = d3.lattice(g.shape[0])
    return [float(np.tensordot(np.asarray(e, dtype=float), g, axes=(0, 0)).sum()) for e in (ex, ey, ez)]


@pytest.mark.parametrize("q", LATTICES)
def test_fluid_plus_body_momentum_is_conserved(q):
    # closed periodic box: the fluid gains -F_n in step n and a free body without springs
    # gains M dv = (F_n + F_{n-1}) / 2, so P_fluid + M v + F_{n-1} / 2 is invariant on
    # every axis (telescoping). A sign error, a lost force memory or an unfiltered force
    # breaks it.
    r = 3.6
    M = 3.0 * 4.0 / 3.0 * math.pi * r ** 3
    c = (11.3, 9.6, 8.7)
    b = synth.body3(c, 2 * r, v=(0.004, -0.003, 0.002))
    b["dynamics"] = dynamics3(M)
    sp = _box((22, 19, 17), b, [synth.sphere(1, c, r)], q=q)
    d = d3.Domain(sp, g=synth.random_populations3(17, 22, 19, 17, q=q))

    def inv():
        p = _momentum(d.g)
        return [p[a] + M * d.state[0, 3 + a] + 0.5 * d.state[0, 6 + a] for a in range(3)]

    q0 = inv()
    for _ in range(40):
        f = d.run(1)
        qn = inv()
        assert max(abs(qn[a] - q0[a]) for a in range(3)) < 1e-11
        assert np.abs(f).max() > 1e-5
        assert np.array_equal(d.state[0, 6:9], f[0, 0])  # the force memory is this step's force
    assert np.abs(d.state[0, 0:3] - np.array(c)).max() > 0.05


@pytest.mark.parametrize("zeta_c", [0.0, 0.5])
def test_negligible_fluid_force_gives_the_discrete_oscillator(zeta_c):
    # eta = 1e12: F_VP ~ 1e-14, the body is a discrete oscillator on z. Semi-implicit Euler
    # with u = z - z0: u_{m+1} = (2 - c/M - k/M) u_m - (1 - c/M) u_{m-1}, u_0 = 0,
    # u_1 = v0 (1 - c/M): u_m = A r^m sin(m theta), r^2 = 1 - c/M,
    # 2 r cos(theta) = 2 - c/M - k/M. The x and y axes are not free: they keep their
    # initial velocities (here 0.01 and 0).
    M, k, c, v0 = 60.0, 1.5, zeta_c, 0.02
    cen = (12.0, 10.0, 10.0)
    b = synth.body3(cen, 6.0, v=(0.01, 0.0, v0))
    b["dynamics"] = dynamics3(M, (0.0, 0.0, k), (0.0, 0.0, c), free=(0, 0, 1))
    sp = _box((24, 20, 20), b, [synth.sphere(1, cen, 3.0)], eta=1e12)
    d = d3.Domain(sp)
    n = 120
    track = np.zeros((n, 1, 6))
    d.run(n, track=track)
    rr = math.sqrt(1.0 - c / M)
    theta = math.acos((2.0 - c / M - k / M) / (2.0 * rr))
    A = v0 * (1.0 - c / M) / (rr * math.sin(theta))
    m = np.arange(n)
    want = A * rr ** m * np.sin(m * theta)
    u = track[:, 0, 2] - cen[2]
    assert np.abs(u - want).max() < 1e-8
    assert np.abs(u).max() > 0.05
    assert np.abs(track[:, 0, 0] - (cen[0] + 0.01 * m)).max() < 1e-12
    assert (track[:, 0, 1] == cen[1]).all() and (track[:, 0, 3] == 0.01).all() and (track[:, 0, 4] == 0.0).all()


@pytest.mark.parametrize("q", LATTICES)
def test_infinitely_heavy_body_at_rest_is_the_fixed_body(q):
    # M = 1e300, v0 = 0: velocity increments of ~1e-301 vanish against the centre and
    # against u*, so every step equals the fixed body's, bit for bit
    cen = (9.4, 8.2, 7.7)
    b = synth.body3(cen, 7.0)
    fixed = _box((20, 17, 15), dict(b), [synth.sphere(1, cen, 3.5)], q=q)
    hb = dict(b)
    hb["dynamics"] = dynamics3(1e300)
    heavy = _box((20, 17, 15), hb, [synth.sphere(1, cen, 3.5)], q=q)
    g0 = synth.random_populations3(5, 20, 17, 15, q=q)
    a, h = d3.Domain(fixed, g=g0), d3.Domain(heavy, g=g0)
    fa, fh = a.run(30), h.run(30)
    assert np.array_equal(a.g, h.g) and np.array_equal(fa, fh)
    assert tuple(h.state[0, 0:3]) == cen


@pytest.mark.parametrize("q", LATTICES)
def test_infinitely_heavy_moving_body_is_the_prescribed_motion(q):
    # M = 1e300 launched with velocity V: the velocity never changes and the centre
    # advances by V every step, so each step sees the mask and U_O of the prescribed motion
    # c + V n (no node lies within rounding of the sphere here): identical populations and
    # forces. Using the state after the update for a step, or not moving the shapes, would
    # differ from the first step on.
    V = (0.11, -0.071, 0.053)
    cen = (9.4, 8.2, 7.7)
    b = synth.body3(cen, 7.0, v=V)
    shapes = [synth.sphere(1, cen, 3.3), synth.sphere(1, (cen[0] + 2.1, cen[1], cen[2]), 2.2)]
    pres = _box((20, 17, 15), dict(b), shapes, q=q)
    hb = dict(b)
    hb["dynamics"] = dynamics3(1e300)
    heavy = _box((20, 17, 15), hb, shapes, q=q)
    g0 = synth.random_populations3(23, 20, 17, 15, q=q)
    a, h = d3.Domain(pres, g=g0), d3.Domain(heavy, g=g0)
    fa, fh = a.run(40), h.run(40)
    assert np.array_equal(a.g, h.g) and np.array_equal(fa, fh)
    for d in range(3):
        assert abs(h.state[0, d] - (cen[d] + 40 * V[d])) < 1e-12
    assert np.array_equal(a.mask, h.mask) and not np.array_equal(h.mask, d3.rasterize(heavy))


def test_light_body_stays_bounded():
    # the two-step mean removes the alternating component of the penalized interior's
    # force: a sphere 1.5 times heavier than the fluid it displaces, launched in a closed
    # box, comes to rest with the fluid
    r = 3.6
    M = 1.5 * 4.0 / 3.0 * math.pi * r ** 3
    cen = (9.3, 8.6, 8.2)
    b = synth.body3(cen, 2 * r, v=(0.004, -0.003, 0.002))
    b["dynamics"] = dynamics3(M)
    sp = _box((18, 17, 16), b, [synth.sphere(1, cen, r)], q=15)
    d = d3.Domain(sp, g=synth.random_populations3(17, 18, 17, 16, q=15))
    f = d.run(500)
    assert np.isfinite(f).all() and np.abs(f[-50:]).max() < 0.02 * np.abs(f[:10]).max()
    assert np.abs(d.state[0, 3:6]).max() < 0.002
