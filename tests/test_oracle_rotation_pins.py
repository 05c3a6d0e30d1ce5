"""Pins of the oracle's rotating obstacles (a body turns its shapes with its angular
velocity: at step index n by theta = omega n about its centre c + V n, a NACA section's
angle of attack decreasing by theta), each against something other than the oracle: its
own sin/cos against the C library, the mask against a brute-force numpy rasterisation of
the analytically turned shapes, the zero-rotation limit bit for bit equal to pure
translation, a half turn of a symmetric section, and the exact mass and momentum balance
with a turning mask."""
import math

import numpy as np
import pytest

import oracle
import synth

EX, EY = oracle.EX, oracle.EY


def _spec(nx, ny, shapes, bodies, nu=0.05, lam=3 / 16, moving=2, u0=(0.0, 0.0)):
    sp = synth._spec("rot_pin", nx, ny, nu, list(shapes), list(bodies), 0, 0.02, synth._edges(),
                     u0=u0, magic_lambda=lam)
    sp["moving"] = moving
    return sp


def _naca(body, cx, cy, chord, aoa, t=0.12):
    return {"kind": "naca4", "body": body, "cx": float(cx), "cy": float(cy), "chord": float(chord),
            "thickness": float(t), "aoa_rad": float(aoa)}


def test_sincos_against_the_c_library():
    ts = np.concatenate([np.linspace(-3e4, 3e4, 60001), np.linspace(-6.5, 6.5, 26001),
                         np.arange(-64, 65) * (math.pi / 4)])
    for t in ts:
        s, c = oracle.sincos(float(t))
        for mine, ref in ((s, math.sin(t)), (c, math.cos(t))):
            assert abs(mine - ref) <= 2.0 * math.ulp(max(abs(ref), 2.0 ** -60)), (t, mine, ref)
        assert abs(s * s + c * c - 1.0) < 5e-16
    assert oracle.sincos(0.0) == (0.0, 1.0)


def _brute_mask(spec, n, margin=1e-9):
    """Body ids of the turned shapes at step n from numpy (libm sin/cos), and the nodes
    closer than `margin` to some shape's boundary (where libm and the oracle's own sin/cos
    may decide differently)."""
    nx, ny = spec["nx"], spec["ny"]
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    ids = np.zeros((ny, nx), dtype=np.uint8)
    near = np.zeros((ny, nx), dtype=bool)
    for s in spec["shapes"]:
        b = spec["bodies"][s["body"] - 1]
        th = b["omega"] * n
        dx0, dy0 = s["cx"] - b["cx"], s["cy"] - b["cy"]
        px = b["cx"] + b["vx"] * n + math.cos(th) * dx0 - math.sin(th) * dy0
        py = b["cy"] + b["vy"] * n + math.sin(th) * dx0 + math.cos(th) * dy0
        if s["kind"] == "circle":
            g = (X - px) ** 2 + (Y - py) ** 2 - s["radius"] ** 2
            inside = g < 0
            near |= np.abs(g) < margin * s["radius"]
        else:
            a = s["aoa_rad"] - th
            ca, sa = math.cos(a), math.sin(a)
            q = 0.25 * s["chord"]
            lex, ley = px - q * ca, py + q * sa
            xp = (X - lex) * ca - (Y - ley) * sa
            yp = (X - lex) * sa + (Y - ley) * ca
            xc = np.clip(xp / s["chord"], 0.0, 1.0)
            yt = 5 * s["thickness"] * s["chord"] * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc ** 2
                                                     + 0.2843 * xc ** 3 - 0.1015 * xc ** 4)
            inside = (xp >= 0) & (xp <= s["chord"]) & (np.abs(yp) <= yt)
            near |= (np.abs(np.abs(yp) - yt) < margin) & (xp > -margin) & (xp < s["chord"] + margin)
            near |= (np.abs(xp) < margin) | (np.abs(xp - s["chord"]) < margin)
        ids[inside] = s["body"]
    return ids, near


def test_turned_mask_is_the_brute_force_mask():
    # body 1: a NACA 0012 about its quarter chord with a circle riding 14 cells behind it;
    # body 2: two circles orbiting their body centre; both also translate
    shapes = [_naca(1, 60.3, 50.2, 40.0, 0.15), synth._circle(1, 74.3, 53.2, 4.0),
              synth._circle(2, 150.0, 40.0, 6.0), synth._circle(2, 150.0, 62.0, 3.5)]
    bodies = [synth._body(60.3, 50.2, 40.0, vx=0.05, vy=-0.02, omega=0.013),
              synth._body(150.0, 51.0, 12.0, vx=-0.03, omega=-0.021)]
    sp = _spec(200, 100, shapes, bodies)
    for n in (0, 1, 7, 123, 1000):
        got = oracle.rasterize(sp, n)
        want, near = _brute_mask(sp, n)
        assert near.sum() == 0 or np.array_equal(got[~near], want[~near])
        assert np.array_equal(got, want), f"step {n}: {np.count_nonzero(got != want)} nodes differ"
        assert (got == 1).sum() > 150 and (got == 2).sum() > 100
    # the section has turned: step 123 differs from the translated-only placement
    tr = dict(sp, moving=True)
    assert not np.array_equal(oracle.rasterize(sp, 123), oracle.rasterize(tr, 123))


def test_zero_rotation_is_translation_bit_for_bit():
    # omega = 0 and every shape's reference point at its body centre: cos 0 = 1 and
    # sin 0 = 0 place every shape exactly where pure translation does
    shapes = [_naca(1, 30.4, 25.3, 24.0, -0.2), synth._circle(2, 62.0, 22.0, 5.0)]
    bodies = [synth._body(30.4, 25.3, 24.0, vx=0.07, vy=0.03), synth._body(62.0, 22.0, 10.0, vx=-0.05)]
    rot, tr = _spec(90, 50, shapes, bodies), _spec(90, 50, shapes, bodies, moving=True)
    g0 = synth.random_populations(7, 90, 50)
    a, b = oracle.Domain(rot, g=g0), oracle.Domain(tr, g=g0)
    fa, fb = a.run(60), b.run(60)
    assert np.array_equal(a.g, b.g) and np.array_equal(fa, fb) and np.array_equal(a.mask, b.mask)
    assert not np.array_equal(a.mask, oracle.rasterize(rot))


def test_half_turn_of_a_symmetric_section():
    # a NACA 00xx section at zero incidence turned by pi about its mid-chord point (the
    # body centre; the quarter chord, the shape's reference point, orbits it): the nose
    # now points downstream and the column span is unchanged; the oracle at the step where
    # theta = pi matches the brute force
    chord = 40.0
    N = 400
    omega = math.pi / N
    mid = (40.0, 30.0)
    shapes = [_naca(1, mid[0] - 0.25 * chord, mid[1], chord, 0.0, t=0.24)]
    sp = _spec(80, 60, shapes, [synth._body(mid[0], mid[1], chord, omega=omega)])
    m = oracle.rasterize(sp, N)
    want, near = _brute_mask(sp, N)
    assert np.array_equal(m[~near], want[~near])
    m0 = oracle.rasterize(sp, 0)
    # turned by pi about the mid-chord: the nose now points downstream
    cols0 = np.nonzero(m0.any(axis=0))[0]
    cols = np.nonzero(m.any(axis=0))[0]
    assert abs((cols0.min() + cols0.max()) - (cols.min() + cols.max())) <= 2
    thick0 = m0.sum(axis=0)[cols0.min() + 4]  # near the nose: thick
    thick = m.sum(axis=0)[cols.max() - 4]     # the nose is now at the downstream end
    assert m.sum(axis=0)[cols.min() + 4] < thick0 - 2  # and the thin tail upstream
    assert thick0 > 4 and abs(int(thick0) - int(thick)) <= 2


@pytest.mark.parametrize("lam", [3 / 16, 0.25])
def test_turning_bodies_conserve_mass_and_balance_momentum(lam):
    # P3, P4 with a turning mask: on a periodic box total mass is conserved and the
    # momentum gained each step is minus the force on the bodies
    shapes = [_naca(1, 22.3, 18.1, 20.0, 0.3), synth._circle(2, 50.0, 14.0, 3.0), synth._circle(2, 50.0, 24.0, 3.0)]
    bodies = [synth._body(22.3, 18.1, 20.0, vx=0.02, omega=0.03), synth._body(50.0, 19.0, 10.0, omega=-0.04)]
    sp = _spec(64, 38, shapes, bodies, lam=lam)
    d = oracle.Domain(sp, g=synth.random_populations(13, 64, 38))
    m0 = d.g.sum()
    for _ in range(60):
        jx0, jy0 = (EX[:, None, None] * d.g).sum(), (EY[:, None, None] * d.g).sum()
        fb = d.run(1)[0]
        jx1, jy1 = (EX[:, None, None] * d.g).sum(), (EY[:, None, None] * d.g).sum()
        net = fb.sum(axis=0)
        assert abs((jx1 - jx0) + net[0]) < 1e-14 * 64 * 38
        assert abs((jy1 - jy0) + net[1]) < 1e-14 * 64 * 38
    assert abs(d.g.sum() - m0) < 1e-12 * m0
    assert not np.array_equal(d.mask, oracle.rasterize(dict(sp, moving=True), 60))


def test_oracle_rejects_turning_or_pulsating_coupled_bodies():
    b = synth._body(20.0, 15.0, 10.0, omega=0.01)
    b["dynamics"] = synth.dynamics(1e3)
    with pytest.raises(ValueError):  # coupled bodies translate their shapes only
        oracle.Domain(_spec(40, 30, [synth._circle(1, 20.0, 15.0, 5.0)], [b]))
    p = dict(synth._body(20.0, 15.0, 10.0), deform={"amplitude": 0.1, "rate": 0.02})
    with pytest.raises(ValueError):  # a fixed mask does not pulsate
        oracle.Domain(_spec(40, 30, [synth._circle(1, 20.0, 15.0, 5.0)], [p], moving=False))
    p["dynamics"] = synth.dynamics(1e3)
    with pytest.raises(ValueError):  # coupled bodies do not deform
        oracle.Domain(_spec(40, 30, [synth._circle(1, 20.0, 15.0, 5.0)], [p], moving=True))
