"""Pins of the 3D oracle, for both lattices (D3Q19 and D3Q15), against what the lattice,
the paper's equations and mathematics fix: lattice isotropy, equilibrium and Guo moments, the sphere mask by brute
force, streaming as array rolls and mirror rules, invariant rest and uniform states,
exact mass and momentum balance with bodies, the closed form of a fully penalized box,
and the viscous decay rate of a shear wave (tau_s = nu / c_s^2 + 1/2)."""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import d3 as d3

CS2 = 1.0 / 3.0
LATTICES = [19, 15]


def _lat(q):
    ex, ey, ez, w, opp = d3.lattice(q)
    return np.stack([ex, ey, ez], axis=1).astype(float), w, opp


def _moments(g):
    E, _, _ = _lat(g.shape[0])
    rho = g.sum(axis=0)
    j = [np.tensordot(E[:, d], g, axes=(0, 0)) for d in range(3)]
    return rho, j


def _spec(nx, ny, nz, nu=0.05, lam=3 / 16, edges=None, shapes=(), bodies=(), u0=(0, 0, 0),
          u_in=(0, 0, 0), eta=1e-4, q=19):
    return synth.spec3("pin3", nx, ny, nz, nu, list(shapes), list(bodies), 0, 0.01,
                       edges or synth.edges3(), u_in=u_in, u0=u0, magic_lambda=lam, eta=eta,
                       lattice=q)


@pytest.mark.parametrize("q", LATTICES)
def test_velocity_set_and_isotropy(q):
    # D3Q19: rest, six vectors of length 1, twelve of length sqrt(2), weights 1/3, 1/18,
    # 1/36; D3Q15: rest, six of length 1, eight of length sqrt(3), weights 2/9, 1/9, 1/72.
    # Distinct vectors; opposite pairs; weights summing to 1; odd moments vanish and the
    # second and fourth moments are isotropic: sum w e_i e_j = c_s^2 delta_ij,
    # sum w e_i e_j e_k e_l = c_s^4 (d_ij d_kl + d_ik d_jl + d_il d_jk)
    E, W, OPP = _lat(q)
    assert len({tuple(e) for e in E.astype(int)}) == q
    n2 = (E ** 2).sum(axis=1)
    diag = 2 if q == 19 else 3
    assert sorted(n2.tolist()) == [0] + [1] * 6 + [diag] * (q - 7)
    cls = {19: {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}, 15: {0: 2 / 9, 1: 1 / 9, 3: 1 / 72}}[q]
    for a in range(q):
        assert np.array_equal(E[OPP[a]], -E[a])
        assert W[a] == cls[int(n2[a])]
    assert W.sum() == pytest.approx(1.0, abs=1e-15)
    d = np.eye(3)
    for i in range(3):
        assert abs((W * E[:, i]).sum()) < 1e-16
        for j in range(3):
            assert (W * E[:, i] * E[:, j]).sum() == pytest.approx(CS2 * d[i, j], abs=1e-15)
            for k in range(3):
                assert abs((W * E[:, i] * E[:, j] * E[:, k]).sum()) < 1e-16
                for l in range(3):
                    want = CS2 ** 2 * (d[i, j] * d[k, l] + d[i, k] * d[j, l] + d[i, l] * d[j, k])
                    assert (W * E[:, i] * E[:, j] * E[:, k] * E[:, l]).sum() == pytest.approx(want, abs=1e-15)


@pytest.mark.parametrize("q", LATTICES)
@pytest.mark.parametrize("rho,u", [(1.0, (0.0, 0.0, 0.0)), (0.97, (0.05, -0.03, 0.02))])
def test_equilibrium_moments(rho, u, q):
    E, _, _ = _lat(q)
    f = d3.equilibrium(rho, u, q)
    u = np.array(u)
    assert f.sum() == pytest.approx(rho, rel=1e-14)
    assert np.allclose(E.T @ f, rho * u, atol=1e-15)
    pi = np.einsum("a,ai,aj->ij", f, E, E)
    assert np.allclose(pi, rho * (CS2 * np.eye(3) + np.outer(u, u)), atol=1e-15)


@pytest.mark.parametrize("q", LATTICES)
def test_guo_term_moments(q):
    E, _, _ = _lat(q)
    u, F = np.array([0.04, -0.02, 0.03]), np.array([-3e-4, 7e-4, 2e-4])
    g = d3.guo(u, F, q)
    assert abs(g.sum()) < 1e-18
    assert np.allclose(E.T @ g, F, atol=1e-18)
    assert np.allclose(np.einsum("a,ai,aj->ij", g, E, E), np.outer(u, F) + np.outer(F, u), atol=1e-18)


def test_rasterize_brute_force():
    shapes = [synth.sphere(1, (9.3, 7.7, 6.1), 4.5), synth.cylinder_z(2, 18.0, 10.0, 3.0),
              synth.sphere(3, (17.5, 10.5, 4.0), 2.0)]  # overlaps the cylinder: later wins
    sp = _spec(24, 16, 12, shapes=shapes, bodies=[synth.body3((0, 0, 0), 1)] * 3)
    m = d3.rasterize(sp)
    k, j, i = np.mgrid[0:12, 0:16, 0:24]
    want = np.zeros_like(m)
    want[(i - 9.3) ** 2 + (j - 7.7) ** 2 + (k - 6.1) ** 2 < 4.5 ** 2] = 1
    want[(i - 18.0) ** 2 + (j - 10.0) ** 2 < 9.0] = 2
    want[(i - 17.5) ** 2 + (j - 10.5) ** 2 + (k - 4.0) ** 2 < 4.0] = 3
    assert np.array_equal(m, want)
    # integer ball: points with x^2 + y^2 + z^2 < 25 (strict) by counting
    ball = _spec(21, 21, 21, shapes=[synth.sphere(1, (10, 10, 10), 5.0)], bodies=[synth.body3((0, 0, 0), 1)])
    n = sum(1 for x, y, z in itertools.product(range(-5, 6), repeat=3) if x * x + y * y + z * z < 25)
    assert (d3.rasterize(ball) == 1).sum() == n == 485


@pytest.mark.parametrize("q", LATTICES)
def test_stream_periodic_is_a_roll_and_mirrors(q):
    E, _, _ = _lat(q)
    EX, EY, EZ = (E[:, d].astype(int) for d in range(3))
    g = synth.random_populations3(3, 7, 6, 5, q=q)
    f = d3.stream(_spec(7, 6, 5, q=q), g)
    for a in range(q):
        assert np.array_equal(f[a], np.roll(g[a], (EZ[a], EY[a], EX[a]), axis=(0, 1, 2)))
    # free slip on y and z: a source outside the rows/planes is the mirrored direction at
    # the clamped row/plane
    sp = _spec(7, 6, 5, edges=synth.edges3("periodic", "periodic", "free_slip", "free_slip",
                                           "free_slip", "free_slip"), q=q)
    f = d3.stream(sp, g)
    for a in range(q):
        for k, j, i in itertools.product(range(5), range(6), range(7)):
            sx, sy, sz, src = (i - EX[a]) % 7, j - EY[a], k - EZ[a], a
            if sy < 0 or sy > 5:
                sy = min(max(sy, 0), 5)
                src = [b for b in range(q) if EX[b] == EX[src] and EY[b] == -EY[src] and EZ[b] == EZ[src]][0]
            if sz < 0 or sz > 4:
                sz = min(max(sz, 0), 4)
                src = [b for b in range(q) if EX[b] == EX[src] and EY[b] == EY[src] and EZ[b] == -EZ[src]][0]
            assert f[a, k, j, i] == g[src, sz, sy, sx]


@pytest.mark.parametrize("q", LATTICES)
def test_stream_inlet_outflow_columns(q):
    # x edges: a source west of column 0 is the inlet equilibrium f^eq(rho0, u_in); a source
    # east of the last column is the last column itself (zero gradient)
    E, _, _ = _lat(q)
    EX, EY, EZ = (E[:, d].astype(int) for d in range(3))
    g = synth.random_populations3(4, 6, 5, 4, q=q)
    u_in = (0.05, 0.01, -0.02)
    sp = _spec(6, 5, 4, edges=synth.edges3("inlet", "outflow"), u_in=u_in, q=q)
    f = d3.stream(sp, g)
    feq = d3.equilibrium(1.0, u_in, q)
    for a in range(q):
        for k, j, i in itertools.product(range(4), range(5), range(6)):
            sx, sy, sz = i - EX[a], (j - EY[a]) % 5, (k - EZ[a]) % 4
            want = feq[a] if sx < 0 else g[a, sz, sy, min(sx, 5)]
            assert f[a, k, j, i] == want


@pytest.mark.parametrize("q", LATTICES)
def test_rotating_penalized_box_follows_the_body_velocity(q):
    # chi = 1 everywhere, body translating at V and rotating at omega about c: the corrected
    # velocity u = u* + du of every node is U_O = V + omega x (x - c) within
    # 2 eta |u* - U_O| (Eq. d-V, Eq. velocity-r); fixes the cross product and its sign
    V, w, c = (0.01, -0.02, 0.005), (1e-3, -2e-3, 1.5e-3), (2.25, 2.75, 3.25)
    sp = _spec(6, 5, 7, nu=0.1, eta=1e-7, shapes=[synth.cylinder_z(1, 3.0, 2.0, 100.0)],
               bodies=[synth.body3(c, 1, v=V, w=w)], q=q)
    d = d3.Domain(sp)
    d.run(50, want_forces=False)
    _, ux, uy, uz = d.moments()
    k, j, i = np.mgrid[0:7, 0:5, 0:6]
    r = (i - c[0], j - c[1], k - c[2])
    want = (V[0] + w[1] * r[2] - w[2] * r[1], V[1] + w[2] * r[0] - w[0] * r[2],
            V[2] + w[0] * r[1] - w[1] * r[0])
    for got, exp in zip((ux, uy, uz), want):
        assert np.max(np.abs(got - exp)) < 1e-7


@pytest.mark.parametrize("q", LATTICES)
@pytest.mark.parametrize("edges", [synth.edges3(), synth.channel_edges3()])
def test_uniform_flow_invariant(edges, q):
    u = (0.05, 0.0, 0.0) if edges["west"] == "inlet" else (0.04, -0.02, 0.03)
    sp = _spec(9, 6, 5, edges=edges, u0=u, u_in=u, q=q)
    d = d3.Domain(sp)
    g0 = d.g.copy()
    d.run(20, want_forces=False)
    assert np.max(np.abs(d.g - g0)) < 1e-15


@pytest.mark.parametrize("q", LATTICES)
def test_mass_and_momentum_balance_with_bodies(q):
    shapes = [synth.sphere(1, (6.2, 7.1, 5.3), 3.5), synth.cylinder_z(2, 14.5, 6.0, 2.5)]
    bodies = [synth.body3((6.2, 7.1, 5.3), 7, v=(0.01, 0.0, -0.005), w=(1e-3, -2e-3, 3e-3)),
              synth.body3((14.5, 6.0, 0.0), 5)]
    sp = _spec(19, 13, 11, lam=0.25, shapes=shapes, bodies=bodies, q=q)
    d = d3.Domain(sp, g=synth.random_populations3(5, 19, 13, 11, q=q))
    m0 = d.g.sum()
    for _ in range(25):
        _, j0 = _moments(d.g)
        _, fb = d.step_once()
        _, j1 = _moments(d.g)
        net = fb.sum(axis=0)
        for c in range(3):
            assert abs((j1[c].sum() - j0[c].sum()) + net[c]) < 1e-14 * d.g[0].size
        assert np.abs(net).max() > 1e-6
    assert abs(d.g.sum() - m0) < 1e-12 * m0


@pytest.mark.parametrize("q", LATTICES)
def test_fully_penalized_box_closed_form(q):
    # chi = 1 everywhere (a z-cylinder covering the box), uniform state: one step maps
    # u* - U_O to (u* - U_O)(2 eta - 1)/(2 eta + 1) and the force on the body is
    # -cells 2 rho (U_O - u*)/(2 eta + 1)
    eta = 0.05
    uo = (0.02, -0.01, 0.015)
    sp = _spec(4, 3, 5, nu=0.1, eta=eta, shapes=[synth.cylinder_z(1, 1.5, 1.0, 100.0)],
               bodies=[synth.body3((0, 0, 0), 1, v=uo)], u0=(0.07, 0.03, -0.02), q=q)
    d = d3.Domain(sp)
    assert np.all(d.mask == 1)
    fac = (2 * eta - 1) / (2 * eta + 1)
    for _ in range(8):
        rho, j = _moments(d.g)
        us = np.array([j[c][0, 0, 0] / rho[0, 0, 0] for c in range(3)])
        _, fb = d.step_once()
        rho1, j1 = _moments(d.g)
        us1 = np.array([j1[c][0, 0, 0] / rho1[0, 0, 0] for c in range(3)])
        assert np.allclose(us1 - uo, (us - uo) * fac, rtol=1e-12, atol=1e-17)
        assert np.allclose(fb[0], -60 * 2 * rho[0, 0, 0] * (np.array(uo) - us) / (2 * eta + 1), rtol=1e-11)


@pytest.mark.parametrize("q", LATTICES)
@pytest.mark.parametrize("nu,lam", [(0.1, 3 / 16), (0.02, 0.25)])
def test_shear_wave_decay_rate(nu, lam, q):
    # u_x = A sin(2 pi k / nz) decays as exp(-nu (2 pi / nz)^2 t) (second-order lattice
    # error: about 4x smaller per doubling of nz)
    def rel_err(nz):
        A, steps = 1e-3, int(0.3 * nz * nz / nu / (2 * math.pi) ** 2 * 4)
        sp = _spec(2, 2, nz, nu=nu, lam=lam, q=q)
        kk = np.arange(nz)
        g = np.stack([np.stack([np.stack([d3.equilibrium(1.0, (A * math.sin(2 * math.pi * k / nz), 0, 0), q)
                                          for _ in range(2)], axis=1) for _ in range(2)], axis=1)
                      for k in kk], axis=1)  # [q, nz, 2, 2]
        d = d3.Domain(sp, g=g)
        d.run(steps, want_forces=False)
        _, ux, _, _ = d.moments()
        amp = 2 * (ux[:, 0, 0] * np.sin(2 * math.pi * kk / nz)).mean()
        want = A * math.exp(-nu * (2 * math.pi / nz) ** 2 * steps)
        return abs(amp - want) / want
    e32, e64 = rel_err(32), rel_err(64)
    assert e64 < 0.01
    assert e32 / e64 > 3.0


# ---- moving bodies (prescribed translation) ---------------------------------------------

def _moving(sp):
    return dict(sp, moving=True)


@pytest.mark.parametrize("q", LATTICES)
def test_moving_mask_is_the_translated_mask(q):
    # a body moving by (1/4, 0, -1/8) cells per step covers, after 8 steps, the nodes of
    # the reference mask shifted by (2, 0, -1) (numpy roll, no wrap in this box)
    V = (0.25, 0.0, -0.125)
    sp = _moving(_spec(30, 20, 18, shapes=[synth.sphere(1, (9.3, 10.2, 9.6), 4.4), synth.cylinder_z(2, 20.1, 6.3, 2.6)],
                       bodies=[synth.body3((9.3, 10.2, 9.6), 8.8, v=V), synth.body3((20.1, 6.3, 0.0), 5.2)], q=q))
    m0 = d3.rasterize(sp)
    m8 = d3.rasterize(sp, 8)
    want = m0.copy()
    want[m0 == 1] = 0
    want[np.roll(m0 == 1, (-1, 0, 2), axis=(0, 1, 2))] = 1
    want[m0 == 2] = 2  # the fixed cylinder, drawn later, stays on top
    assert np.array_equal(m8, want)
    d = d3.Domain(sp)
    d.run(8, want_forces=False)
    assert np.array_equal(d.mask, m8)


@pytest.mark.parametrize("q", LATTICES)
def test_moving_body_in_comoving_uniform_flow_is_steady(q):
    # a body moving with the uniform flow of a periodic box: U_O = u everywhere, so the
    # penalization does nothing and the state stays exactly uniform
    u = (0.02, -0.01, 0.015)
    sp = _moving(_spec(24, 16, 14, shapes=[synth.sphere(1, (8.3, 7.9, 6.6), 3.9)],
                       bodies=[synth.body3((8.3, 7.9, 6.6), 7.8, v=u)], u0=u, q=q))
    d = d3.Domain(sp)
    g0 = d.g.copy()
    f = d.run(60)
    assert np.abs(d.g - g0).max() < 1e-13
    assert np.abs(f).max() < 1e-12
    assert not np.array_equal(d.mask, d3.rasterize(sp))  # it did move


@pytest.mark.parametrize("q", LATTICES)
def test_moving_bodies_conserve_mass_and_balance_momentum(q):
    shapes = [synth.sphere(1, (6.2, 7.1, 5.3), 3.5), synth.cylinder_z(2, 14.5, 6.0, 2.5)]
    bodies = [synth.body3((6.2, 7.1, 5.3), 7, v=(0.05, 0.02, -0.03), w=(1e-3, -2e-3, 3e-3)),
              synth.body3((14.5, 6.0, 0.0), 5, v=(-0.04, 0.03, 0.0))]
    sp = _moving(_spec(21, 14, 12, lam=0.25, shapes=shapes, bodies=bodies, q=q))
    d = d3.Domain(sp, g=synth.random_populations3(5, 21, 14, 12, q=q))
    m0 = d.g.sum()
    for _ in range(30):
        _, j0 = _moments(d.g)
        fb = d.run(1)[0]
        _, j1 = _moments(d.g)
        net = fb.sum(axis=0)
        for c in range(3):
            assert abs((j1[c].sum() - j0[c].sum()) + net[c]) < 1e-14 * d.g[0].size
    assert abs(d.g.sum() - m0) < 1e-12 * m0
    assert not np.array_equal(d.mask, d3.rasterize(sp))


def test_moving_run_equals_steps_with_the_geometry_of_each_index():
    # run(n) is n single steps, step m with the mask and body table of index m
    shapes = [synth.sphere(1, (7.2, 6.1, 5.4), 3.1)]
    bodies = [synth.body3((7.2, 6.1, 5.4), 6.2, v=(0.07, -0.03, 0.02), w=(0.0, 0.0, 2e-3))]
    sp = _moving(_spec(18, 13, 11, shapes=shapes, bodies=bodies))
    g0 = synth.random_populations3(9, 18, 13, 11)
    a = d3.Domain(sp, g=g0)
    fa = a.run(12)
    g, fs = g0.copy(), []
    for m in range(12):
        moved = dict(sp, moving=False,
                     shapes=[dict(s, c=tuple(c + v * m for c, v in zip(s["c"], bodies[0]["v"]))) for s in shapes],
                     bodies=[dict(bodies[0], c=tuple(c + v * m for c, v in zip(bodies[0]["c"], bodies[0]["v"])))])
        b = d3.Domain(moved, g=g)
        g, f = b.step_once()
        fs.append(f)
    assert np.array_equal(a.g, g)
    assert np.array_equal(fa, np.stack(fs))
