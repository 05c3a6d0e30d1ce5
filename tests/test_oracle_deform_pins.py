"""Pins of the oracle's deforming obstacles (a body pulsates about its centre: at step
index n its shapes are scaled by s(n) = 1 + a sin(nu n), offsets included, and U_O adds
the dilation velocity kappa(n) (x - c), kappa = s'/s), each against something other than
the oracle: the mask against a brute-force numpy rasterisation of the scaled shapes, the
solid-node count against the area of the scaled circle, the corrected velocity inside a
penalized body against the analytic dilation velocity, the zero-amplitude limit bit for
bit equal to pure translation, and the exact mass and momentum balance."""
import math

import numpy as np
import pytest

import oracle
import synth

EX, EY = oracle.EX, oracle.EY


def _spec(nx, ny, shapes, bodies, moving=True, nu=0.05, lam=3 / 16, eta=1e-4):
    sp = synth._spec("deform_pin", nx, ny, nu, list(shapes), list(bodies), 0, 0.02, synth._edges(),
                     magic_lambda=lam, eta=eta)
    sp["moving"] = moving
    return sp


def _deforming(body, amplitude, rate):
    return dict(body, deform={"amplitude": float(amplitude), "rate": float(rate)})


def _naca(body, cx, cy, chord, aoa, t=0.12):
    return {"kind": "naca4", "body": body, "cx": float(cx), "cy": float(cy), "chord": float(chord),
            "thickness": float(t), "aoa_rad": float(aoa)}


def _scale(b, n):
    d = b.get("deform")
    if not d:
        return 1.0, 0.0
    s = 1.0 + d["amplitude"] * math.sin(d["rate"] * n)
    return s, d["amplitude"] * d["rate"] * math.cos(d["rate"] * n) / s


def _brute_mask(spec, n, margin=1e-9):
    nx, ny = spec["nx"], spec["ny"]
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    ids = np.zeros((ny, nx), dtype=np.uint8)
    near = np.zeros((ny, nx), dtype=bool)
    rot = spec["moving"] == 2 and not isinstance(spec["moving"], bool)
    for s in spec["shapes"]:
        b = spec["bodies"][s["body"] - 1]
        th = b["omega"] * n if rot else 0.0
        sc, _ = _scale(b, n)
        dx0, dy0 = s["cx"] - b["cx"], s["cy"] - b["cy"]
        px = b["cx"] + b["vx"] * n + sc * (math.cos(th) * dx0 - math.sin(th) * dy0)
        py = b["cy"] + b["vy"] * n + sc * (math.sin(th) * dx0 + math.cos(th) * dy0)
        if s["kind"] == "circle":
            r = sc * s["radius"]
            g = (X - px) ** 2 + (Y - py) ** 2 - r * r
            inside = g < 0
            near |= np.abs(g) < margin * r
        else:
            a, chord = s["aoa_rad"] - th, sc * s["chord"]
            ca, sa = math.cos(a), math.sin(a)
            lex, ley = px - 0.25 * chord * ca, py + 0.25 * chord * sa
            xp = (X - lex) * ca - (Y - ley) * sa
            yp = (X - lex) * sa + (Y - ley) * ca
            xc = np.clip(xp / chord, 0.0, 1.0)
            yt = 5 * s["thickness"] * chord * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc ** 2
                                                + 0.2843 * xc ** 3 - 0.1015 * xc ** 4)
            inside = (xp >= 0) & (xp <= chord) & (np.abs(yp) <= yt)
            near |= (np.abs(np.abs(yp) - yt) < margin) & (xp > -margin) & (xp < chord + margin)
            near |= (np.abs(xp) < margin) | (np.abs(xp - chord) < margin)
        ids[inside] = s["body"]
    return ids, near


@pytest.mark.parametrize("moving", [True, 2])
def test_pulsating_mask_is_the_brute_force_mask(moving):
    # body 1: a NACA section and an offset circle pulsating together (turning too for a
    # rotating domain); body 2: a rigid circle
    shapes = [_naca(1, 50.3, 40.2, 36.0, 0.1), synth._circle(1, 66.3, 44.2, 4.0), synth._circle(2, 120.0, 40.0, 7.0)]
    bodies = [_deforming(synth._body(52.1, 40.2, 36.0, vx=0.04, vy=-0.01, omega=0.009), 0.35, 0.021),
              synth._body(120.0, 40.0, 14.0, vx=-0.02, omega=0.01)]
    sp = _spec(160, 80, shapes, bodies, moving=moving)
    for n in (0, 5, 37, 160, 400):
        got = oracle.rasterize(sp, n)
        want, near = _brute_mask(sp, n)
        assert np.array_equal(got[~near], want[~near]), f"step {n}"
        assert np.array_equal(got, want)
    # it does pulsate: the section's area follows s(n)^2
    a0 = (oracle.rasterize(sp, 0) == 1).sum()
    n_max = int(round((math.pi / 2) / 0.021))  # s = 1.35
    assert (oracle.rasterize(sp, n_max) == 1).sum() > 1.6 * a0


def test_breathing_circle_area():
    # a circle of radius 15 pulsating by 30 %: its node count is the area of the scaled
    # circle within the Gauss circle bound (perimeter + 4)
    a, nu = 0.3, 2 * math.pi / 300
    sp = _spec(80, 80, [synth._circle(1, 40.25, 39.6, 15.0)], [_deforming(synth._body(40.25, 39.6, 30.0), a, nu)])
    for n in range(0, 300, 23):
        r = 15.0 * (1.0 + a * math.sin(nu * n))
        cnt = (oracle.rasterize(sp, n) == 1).sum()
        assert abs(cnt - math.pi * r * r) <= 2 * math.pi * r + 4


def test_penalized_interior_moves_with_the_dilation():
    # eta = 1e-6: the corrected velocity u = (2 eta u* + U_O) / (2 eta + 1) of every solid
    # node is the body's material velocity, here V + kappa (x - c) with kappa = s'/s
    a, nu = 0.2, 2 * math.pi / 400
    c = (40.3, 30.6)
    b = _deforming(synth._body(c[0], c[1], 24.0, vx=0.01), a, nu)
    sp = _spec(80, 60, [synth._circle(1, c[0], c[1], 12.0)], [b], eta=1e-6)
    d = oracle.Domain(sp, g=synth.random_populations(3, 80, 60, 0.02))
    d.run(57, want_forces=False)
    n = d.steps_done
    _, kap = _scale(b, n)
    cx, cy = c[0] + 0.01 * n, c[1]
    rho, ux, uy = d.moments()
    J, I = np.nonzero(d.mask == 1)
    assert len(J) > 300 and abs(kap) > 1e-3
    want_x = 0.01 + kap * (I - cx)
    want_y = kap * (J - cy)
    assert np.abs(ux[J, I] - want_x).max() < 1e-6 and np.abs(uy[J, I] - want_y).max() < 1e-6
    assert np.abs(want_y).max() > 0.01  # the dilation velocity is not small


def test_zero_amplitude_is_translation_bit_for_bit():
    shapes = [_naca(1, 30.4, 25.3, 24.0, -0.2), synth._circle(2, 62.0, 22.0, 5.0)]
    rigid = [synth._body(30.4, 25.3, 24.0, vx=0.07, vy=0.03), synth._body(62.0, 22.0, 10.0, vx=-0.05)]
    flat = [_deforming(rigid[0], 0.0, 0.05), _deforming(rigid[1], 0.0, 0.03)]
    g0 = synth.random_populations(7, 90, 50)
    a, b = oracle.Domain(_spec(90, 50, shapes, rigid), g=g0), oracle.Domain(_spec(90, 50, shapes, flat), g=g0)
    fa, fb = a.run(60), b.run(60)
    assert np.array_equal(a.g, b.g) and np.array_equal(fa, fb) and np.array_equal(a.mask, b.mask)


@pytest.mark.parametrize("moving", [True, 2])
def test_deforming_bodies_conserve_mass_and_balance_momentum(moving):
    shapes = [_naca(1, 22.3, 18.1, 20.0, 0.3), synth._circle(2, 50.0, 19.0, 6.0)]
    bodies = [_deforming(synth._body(22.3, 18.1, 20.0, vx=0.02, omega=0.02), 0.3, 0.05),
              _deforming(synth._body(50.0, 19.0, 12.0, omega=-0.03), -0.4, 0.08)]
    sp = _spec(64, 38, shapes, bodies, moving=moving, lam=0.25)
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
    assert (d.mask == 2).sum() != (oracle.rasterize(sp, 0) == 2).sum()
