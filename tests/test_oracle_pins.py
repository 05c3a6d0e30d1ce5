"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself: a published
value, a closed form, an exact invariant, a textbook special case or brute force.
The comment on each names the part of the oracle a plausible mistake would break.
"""
import math

import numpy as np
import pytest

import oracle
import synth

EX, EY, W = oracle.EX, oracle.EY, oracle.W


def _moments(g):
    rho = g.sum(axis=0)
    jx = np.tensordot(EX, g, axes=(0, 0))
    jy = np.tensordot(EY, g, axes=(0, 0))
    return rho, jx, jy


def _spec(nx, ny, nu=0.05, lam=3 / 16, edges=None, shapes=(), bodies=(), u_in=(0, 0),
          u0=(0, 0), eta=1e-4):
    return synth._spec("pin", nx, ny, nu, list(shapes), list(bodies), 0, 0.01,
                       edges or synth._edges(), u_in=u_in, u0=u0, magic_lambda=lam, eta=eta)


# ---- generator -------------------------------------------------------------------------

def test_splitmix64_published_outputs():
    # SplitMix64 seeded with 0: first outputs of the published algorithm.
    r = synth.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                0x06C45D188009454F]
    a = synth.SplitMix64(12345)
    b = synth.SplitMix64(12345)
    v = a.doubles(1000)
    assert np.array_equal(v, np.array([b.next_double() for _ in range(1000)]))
    assert a.state == b.state


# ---- lattice model (Eq. D2Q9, Eq. feq) ------------------------------------------------------

@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (0.97, 0.05, -0.03), (1.2, -0.1, 0.08)])
def test_equilibrium_moments(rho, ux, uy):
    # The D2Q9 equilibrium reproduces rho, rho u and rho (c_s^2 I + u u) exactly
    # (textbook moment constraints); a wrong weight or coefficient breaks one of them.
    f = oracle.equilibrium(rho, ux, uy)
    assert f.sum() == pytest.approx(rho, rel=1e-14)
    assert (EX * f).sum() == pytest.approx(rho * ux, abs=1e-15)
    assert (EY * f).sum() == pytest.approx(rho * uy, abs=1e-15)
    assert (EX * EX * f).sum() == pytest.approx(rho * (1 / 3 + ux * ux), rel=1e-14)
    assert (EY * EY * f).sum() == pytest.approx(rho * (1 / 3 + uy * uy), rel=1e-14)
    assert (EX * EY * f).sum() == pytest.approx(rho * ux * uy, abs=1e-15)
    # the opposite-direction convention of Sec. 2.1: e_{-a} = -e_a
    opp = [0, 3, 4, 1, 2, 7, 8, 5, 6]
    assert np.array_equal(EX[opp], -EX) and np.array_equal(EY[opp], -EY)
    # the D2Q9 velocity set follows the angle formula of Eq. (D2Q9)
    for a in range(1, 5):
        th = (a - 1) * math.pi / 2
        assert (EX[a], EY[a]) == (round(math.cos(th)), round(math.sin(th)))
    for a in range(5, 9):
        th = (2 * a - 9) * math.pi / 4
        assert (EX[a], EY[a]) == (round(math.sqrt(2) * math.cos(th)),
                                  round(math.sqrt(2) * math.sin(th)))


@pytest.mark.parametrize("ux,uy,fx,fy", [(0.0, 0.0, 1e-3, 0.0), (0.04, -0.02, -3e-4, 7e-4)])
def test_guo_term_moments(ux, uy, fx, fy):
    # Guo et al. (2002) forcing: zeroth moment 0, first moment F, second u F + F u.
    F = oracle.guo(ux, uy, fx, fy)
    assert abs(F.sum()) < 1e-18
    assert (EX * F).sum() == pytest.approx(fx, rel=1e-13, abs=1e-19)
    assert (EY * F).sum() == pytest.approx(fy, rel=1e-13, abs=1e-19)
    assert (EX * EX * F).sum() == pytest.approx(2 * ux * fx, abs=1e-18)
    assert (EY * EY * F).sum() == pytest.approx(2 * uy * fy, abs=1e-18)
    assert (EX * EY * F).sum() == pytest.approx(ux * fy + uy * fx, abs=1e-18)


# ---- geometry (Eq. mask function; NACA 4-digit section) ----------------------------------

def _count_int_disc(R2, strict=True):
    n = 0
    r = int(math.isqrt(R2)) + 1
    for x in range(-r, r + 1):
        for y in range(-r, r + 1):
            d = x * x + y * y
            n += (d < R2) if strict else (d <= R2)
    return n


def test_gauss_circle_counts():
    # Lattice points strictly inside integer circles, by integer brute force; the
    # known Gauss circle values N(10) = 317 and N(20) = 1257 (closed disc) minus the
    # r_2(R^2) = 12 points on each circle.
    assert _count_int_disc(100, strict=False) == 317
    assert _count_int_disc(400, strict=False) == 1257
    sp = synth.couette()
    m = oracle.rasterize(sp)
    assert (m == 1).sum() == 1257 - 12 == _count_int_disc(400)
    assert (m == 2).sum() == 128 * 128 - _count_int_disc(2500, strict=False)
    assert m[64, 64] == 1 and m[64, 64 + 20] == 0 and m[64, 64 + 19] == 1
    assert m[0, 0] == 2 and m[64, 64 + 50] == 0 and m[64, 64 + 51] == 2


def test_rasterize_brute_force_small():
    # Brute force on tiny grids, overlapping shapes: later shapes overwrite earlier ones.
    sp = _spec(23, 17, shapes=[synth._circle(1, 7.3, 8.1, 4.4), synth._circle(2, 10.0, 8.0, 3.0),
                               {"kind": "annulus_outside", "body": 3, "cx": 11.0, "cy": 8.5,
                                "radius": 9.2}])
    m = oracle.rasterize(sp)
    want = np.zeros((17, 23), np.uint8)
    for j in range(17):
        for i in range(23):
            if (i - 7.3) ** 2 + (j - 8.1) ** 2 < 4.4 ** 2:
                want[j, i] = 1
            if (i - 10) ** 2 + (j - 8) ** 2 < 9:
                want[j, i] = 2
            if (i - 11) ** 2 + (j - 8.5) ** 2 > 9.2 ** 2:
                want[j, i] = 3
    assert np.array_equal(m, want)


def test_naca0012_ordinates_published(golden_dir=None):
    # NACA 0012 basic thickness form (Abbott & von Doenhoff, Theory of Wing Sections,
    # 1959, Appendix I): half-thickness in percent chord.
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "naca0012_ordinates.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for x, y in rows:
        assert 100 * oracle.naca_half_thickness(float(x), 0.12, 1.0) == pytest.approx(
            float(y), abs=1.5e-3)
    assert oracle.naca_half_thickness(0.0, 0.12, 1.0) == 0.0


def test_naca_mask_area_and_attitude():
    # Area of a NACA 00tt section is 10 t c^2 * integral of the thickness polynomial
    # = 0.685050 t c^2 (closed-form integral); the staircase count matches within 2%.
    c = 200.0
    area = 10 * 0.12 * c * c * (0.2969 * 2 / 3 - 0.1260 / 2 - 0.3516 / 3 + 0.2843 / 4 - 0.1015 / 5)
    for aoa in (0.0, 10.0):
        sp = synth.naca0012(aoa, 500.0, chord=c, nx=400, ny=300)
        sp["shapes"][0]["cx"] = 150.0
        sp["shapes"][0]["cy"] = 150.0
        m = oracle.rasterize(sp)
        assert abs((m == 1).sum() - area) / area < 0.02
        jj, ii = np.nonzero(m)
        # leading edge at x = cx - c/4 cos(aoa); nose-up: the front is higher than the back
        front = ii < np.percentile(ii, 20)
        back = ii > np.percentile(ii, 80)
        if aoa == 0.0:
            assert abs(jj[front].mean() - 150.0) < 0.5 and abs(jj[back].mean() - 150.0) < 0.5
            assert ii.min() == 100 and ii.max() == 300  # x' in [0, c], open trailing edge
        else:
            assert jj[front].mean() > jj[back].mean() + 10
            le_x = 150.0 - 0.25 * c * math.cos(math.radians(aoa))
            assert abs(ii.min() - le_x) <= 1.0
        # the quarter-chord pivot stays at (150, 150): the column through it is
        # centred on the chord line there
        col = jj[ii == 150]
        assert abs(0.5 * (col.min() + col.max()) - 150.0) <= 1.5


# ---- streaming and the domain-edge rules (Eq. streaming) ----------------------------------

def test_stream_periodic_is_a_roll():
    # On a periodic box Eq. (streaming) is a cyclic shift of each population by e_a,
    # which numpy.roll computes independently.
    g = synth.random_populations(21, 13, 9)
    f = oracle.stream(_spec(13, 9), g)
    for a in range(9):
        assert np.array_equal(f[a], np.roll(np.roll(g[a], EY[a], axis=0), EX[a], axis=1))


def test_stream_edge_rules():
    # The edge rules as read for the channel workloads: an equilibrium ghost at the
    # inlet, zero-gradient (copy of the last column) at the outflow, specular
    # reflection at free-slip walls; the x rule first at corners.
    nx, ny, u = 7, 5, (0.04, 0.01)
    sp = _spec(nx, ny, edges=synth._edges("inlet", "outflow", "free_slip", "free_slip"), u_in=u)
    g = synth.random_populations(22, nx, ny)
    f = oracle.stream(sp, g)
    ghost = oracle.equilibrium(1.0, *u)
    refl = [0, 1, 4, 3, 2, 8, 7, 6, 5]
    for a in range(9):
        for j in range(ny):
            for i in range(nx):
                sx, sy, src = i - EX[a], j - EY[a], a
                if sx < 0:
                    assert f[a, j, i] == ghost[a]
                    continue
                sx = min(sx, nx - 1)
                if sy < 0 or sy > ny - 1:
                    sy, src = min(max(sy, 0), ny - 1), refl[a]
                assert f[a, j, i] == g[src, sy, sx]
    # the outflow copies the last column: columns nx-2 and nx-1 differ in g, and the
    # populations entering from the east take the value of column nx-1
    assert f[3, 2, nx - 1] == g[3, 2, nx - 1] != g[3, 2, nx - 2]


# ---- exact invariants of the time step -----------------------------------------------------

EDGE_SETS = [synth._edges(), synth._edges("periodic", "periodic", "free_slip", "free_slip"),
             synth._edges("inlet", "outflow", "free_slip", "free_slip"),
             synth._edges("inlet", "outflow", "periodic", "periodic")]


@pytest.mark.parametrize("edges", EDGE_SETS)
def test_rest_state_exactly_invariant(edges):
    # P1: all populations at w_a rho0, resting bodies, any edges (inlet at U = 0):
    # every term of the update vanishes up to the rounding of the weights (their FP64
    # sum is not exactly 1), so the state stays put to roundoff, without drift, and
    # the momentum, hence every penalization force, is exactly zero.
    sp = _spec(31, 23, edges=edges, shapes=[synth._circle(1, 10, 11, 5), synth._circle(2, 22, 8, 3)],
               bodies=[synth._body(10, 11, 10), synth._body(22, 8, 6)])
    d = oracle.Domain(sp)
    g0 = d.g.copy()
    assert np.array_equal(g0[:, 5, 7], oracle.equilibrium(1.0, 0.0, 0.0))
    f = d.run(50)
    assert np.max(np.abs(d.g - g0) / g0) < 1e-15
    assert np.all(f == 0.0)


@pytest.mark.parametrize("edges,u", [(synth._edges(), (0.05, -0.03)),
                                     (synth._edges("periodic", "periodic", "free_slip", "free_slip"), (0.06, 0.0)),
                                     (synth._edges("inlet", "outflow", "free_slip", "free_slip"), (0.07, 0.0))])
def test_uniform_flow_invariant(edges, u):
    # P2 and the edge rules: a uniform equilibrium flow without obstacles is a fixed
    # point for periodic edges, for free-slip walls parallel to it (specular
    # reflection maps f^eq_a onto f^eq of the mirrored direction), and for an
    # equilibrium inlet at the same velocity with zero-gradient outflow.
    sp = _spec(29, 19, edges=edges, u_in=u, u0=u)
    d = oracle.Domain(sp)
    g0 = d.g.copy()
    d.run(100, want_forces=False)
    assert np.max(np.abs(d.g - g0) / g0) < 1e-14


def test_free_slip_channel_conserves_mass_and_axial_momentum():
    # Specular free-slip walls exert no tangential force: in a periodic-x channel
    # without obstacles the total mass and x-momentum are conserved exactly (roundoff),
    # while y-momentum is not (the walls reverse it).
    sp = _spec(33, 21, nu=0.04, edges=synth._edges("periodic", "periodic", "free_slip", "free_slip"))
    g = synth.random_populations(7, 33, 21)
    d = oracle.Domain(sp, g=g)
    r0, jx0, jy0 = (v.sum() for v in _moments(d.g))
    d.run(300, want_forces=False)
    r1, jx1, jy1 = (v.sum() for v in _moments(d.g))
    assert abs(r1 - r0) / r0 < 1e-13
    assert abs(jx1 - jx0) < 1e-13 * r0
    assert abs(jy1 - jy0) > 1e-6  # the walls do act on the normal component


def test_mass_conserved_periodic_with_moving_bodies():
    # P3: sum_a Omega_a = 0 and sum_a F_a = 0, so total mass is conserved on a periodic
    # box, with penalized moving bodies and a random non-equilibrium start.
    sp = _spec(40, 30, nu=0.03, shapes=[synth._circle(1, 12, 14, 6), synth._circle(2, 28, 16, 4)],
               bodies=[synth._body(12, 14, 12, omega=3e-3), synth._body(28, 16, 8, vx=0.02, vy=-0.01)])
    d = oracle.Domain(sp, g=synth.random_populations(11, 40, 30))
    m0 = d.g.sum()
    f = d.run(2000)
    assert abs(d.g.sum() - m0) / m0 < 1e-12
    assert np.abs(f).max() > 1e-4  # bodies do push on the fluid


def test_momentum_balance_equals_body_forces():
    # P4: each cell gains exactly its F_VP in the collision (sum e Omega = F/(2 tau_a),
    # sum e F^a = F with the (1 - 1/(2 tau_a)) factor), streaming on a periodic box
    # conserves momentum, so P(n+1) - P(n) = -(sum of the forces on the bodies).
    sp = _spec(37, 26, nu=0.05, lam=0.25,
               shapes=[synth._circle(1, 10, 12, 5), synth._circle(2, 26, 13, 4.5)],
               bodies=[synth._body(10, 12, 10, vx=0.01, omega=-2e-3), synth._body(26, 13, 9)])
    d = oracle.Domain(sp, g=synth.random_populations(3, 37, 26))
    for _ in range(40):
        _, jx0, jy0 = (v.sum() for v in _moments(d.g))
        _, fb = d.step_once()
        _, jx1, jy1 = (v.sum() for v in _moments(d.g))
        net = fb.sum(axis=0)
        assert abs((jx1 - jx0) + net[0]) < 1e-14 * 37 * 26
        assert abs((jy1 - jy0) + net[1]) < 1e-14 * 37 * 26
        assert np.abs(net).max() > 1e-6


def test_fully_penalized_box_closed_form():
    # P5: chi = 1 everywhere, uniform state, periodic: streaming is the identity and
    # one step maps u* - U_O to (u* - U_O)(2 eta - 1)/(2 eta + 1) (Eq. d-V, Eq.
    # force-density and the collision's momentum balance); rho stays constant and
    # the force on the body is -cells * 2 rho (U_O - u*)/(2 eta + 1).
    eta = 0.05
    uo = (0.02, -0.01)
    sp = _spec(6, 5, nu=0.1, eta=eta, shapes=[{"kind": "annulus_outside", "body": 1, "cx": -0.5,
                                               "cy": -0.5, "radius": 0.0}],
               bodies=[synth._body(0, 0, 1, vx=uo[0], vy=uo[1])], u0=(0.07, 0.03))
    d = oracle.Domain(sp)
    assert np.all(d.mask == 1)
    fac = (2 * eta - 1) / (2 * eta + 1)
    for _ in range(12):
        rho, jx, jy = _moments(d.g)
        us = np.array([jx[0, 0] / rho[0, 0], jy[0, 0] / rho[0, 0]])
        _, fb = d.step_once()
        rho1, jx1, jy1 = _moments(d.g)
        us1 = np.array([jx1[0, 0] / rho1[0, 0], jy1[0, 0] / rho1[0, 0]])
        assert np.allclose(us1 - uo, (us - uo) * fac, rtol=1e-12, atol=1e-17)
        assert rho1[0, 0] == pytest.approx(rho[0, 0], rel=1e-14)
        want = -30 * 2 * rho[0, 0] * (np.array(uo) - us) / (2 * eta + 1)
        assert np.allclose(fb[0], want, rtol=1e-11)


def _moving(sp):
    return dict(sp, moving=True)


def test_moving_mask_is_the_translated_mask():
    # Moving obstacles (Sec. 2.2: chi and U_O may depend on time). With velocities that
    # are exact binary fractions the translated shapes land on whole cells after 8 steps
    # (4 and -2 cells): the mask is the reference mask rolled by those cells (numpy).
    sp = _moving(_spec(96, 64, shapes=[synth._circle(1, 30.0, 32.0, 7.5),
                                       {"kind": "naca4", "body": 2, "cx": 60.0, "cy": 20.0,
                                        "chord": 24.0, "thickness": 0.12, "aoa_rad": 0.1}],
                       bodies=[synth._body(30.0, 32.0, 15.0, vx=0.5, vy=-0.25),
                               synth._body(60.0, 20.0, 24.0, vx=-0.125, vy=0.375)]))
    m0 = oracle.rasterize(sp, 0)
    assert np.array_equal(m0, oracle.rasterize(sp))
    m8 = oracle.rasterize(sp, 8)
    want = np.zeros_like(m0)
    c1 = np.roll(np.roll(np.where(m0 == 1, 1, 0), 4, axis=1), -2, axis=0)
    c2 = np.roll(np.roll(np.where(m0 == 2, 2, 0), -1, axis=1), 3, axis=0)
    want = np.maximum(c1, c2).astype(np.uint8)
    assert (m0 == 1).sum() > 150 and (m0 == 2).sum() > 40
    assert np.array_equal(m8, want)
    # and the run re-rasterises: after 8 steps the domain holds the mask of step 8
    d = oracle.Domain(sp)
    d.run(8, want_forces=False)
    assert np.array_equal(d.mask, m8)


def test_moving_run_equals_single_steps():
    # The step from index n to n + 1 uses the geometry of index n (mask and centres): the
    # C loop over steps gives bit for bit the state of single steps taken with the mask
    # and body table of each index.
    sp = _moving(_spec(37, 26, nu=0.05, lam=0.25, shapes=[synth._circle(1, 10, 12, 5)],
                       bodies=[synth._body(10, 12, 10, vx=0.3, vy=-0.2, omega=2e-3)]))
    g0 = synth.random_populations(11, 37, 26)
    a = oracle.Domain(sp, g=g0)
    fa = a.run(7)
    b = oracle.Domain(sp, g=g0)
    fb = np.array([b.step_once()[1] for _ in range(7)])
    assert np.array_equal(a.g, b.g) and np.array_equal(fa, fb)
    assert not np.array_equal(a.mask, oracle.rasterize(sp))


def test_moving_body_in_comoving_uniform_flow_is_steady():
    # A body moving with the velocity of a uniform flow: U_O = u everywhere, so the
    # penalization does nothing (du = 0, F_VP = 0) and the uniform equilibrium stays
    # as it is, although the mask moves by a non-integer distance every step.
    u = (0.03, -0.011)
    sp = _moving(_spec(40, 30, shapes=[synth._circle(1, 15.0, 14.0, 6.0)],
                       bodies=[synth._body(15.0, 14.0, 12.0, vx=u[0], vy=u[1])], u0=u))
    d = oracle.Domain(sp)
    g0 = d.g.copy()
    f = d.run(150)
    # roundoff only: u* - U_O ~ 1e-17 per node (a wrong mask or centre gives ~1e-2)
    assert np.max(np.abs(d.g - g0)) < 1e-13
    assert np.max(np.abs(f)) < 1e-13
    assert not np.array_equal(d.mask, oracle.rasterize(sp))  # it has moved


def test_moving_bodies_conserve_mass_and_balance_momentum():
    # A moving, rotating body in a periodic box: mass is conserved exactly and the
    # momentum gained each step is minus the force on the bodies (P3, P4 with chi(t)).
    sp = _moving(_spec(37, 26, nu=0.05, lam=0.25,
                       shapes=[synth._circle(1, 10, 12, 5), synth._circle(2, 26, 13, 4.5)],
                       bodies=[synth._body(10, 12, 10, vx=0.05, vy=0.02, omega=-2e-3),
                               synth._body(26, 13, 9, vx=-0.03)]))
    d = oracle.Domain(sp, g=synth.random_populations(3, 37, 26))
    m0 = d.g.sum()
    for _ in range(60):
        _, jx0, jy0 = (v.sum() for v in _moments(d.g))
        _, fb = d.step_once()
        _, jx1, jy1 = (v.sum() for v in _moments(d.g))
        net = fb.sum(axis=0)
        assert abs((jx1 - jx0) + net[0]) < 1e-14 * 37 * 26
        assert abs((jy1 - jy0) + net[1]) < 1e-14 * 37 * 26
    assert abs(d.g.sum() - m0) < 1e-12 * m0
    assert not np.array_equal(d.mask, oracle.rasterize(sp))


def test_moving_body_velocity_about_the_moving_centre():
    # chi = 1 everywhere (an "outside" annulus of radius 0), a body translating at V and
    # rotating at Omega: the corrected velocity u = u* + du of every node is U_O(x, t) =
    # V + Omega z x (x - c(t)) within 2 eta |u* - U_O| (Eq. d-V, Eq. velocity-r), with the
    # centre c(t) = c0 + V t moving; a centre left at c0 would be off by Omega V t.
    # (|u* - U_O| reaches a few 1e-2 where the periodic wrap meets the rotation's jump.)
    eta = 1e-6
    # (the centre never lands on a node, where the radius-0 annulus would leave a fluid node)
    V, om, c0 = (0.02, 0.01), 1e-3, (10.25, 8.25)
    sp = _moving(_spec(20, 16, nu=0.1, eta=eta,
                       shapes=[{"kind": "annulus_outside", "body": 1, "cx": c0[0], "cy": c0[1],
                                "radius": 0.0}],
                       bodies=[synth._body(c0[0], c0[1], 1.0, vx=V[0], vy=V[1], omega=om)]))
    d = oracle.Domain(sp)
    d.run(200, want_forces=False)
    assert np.all(d.mask == 1)
    _, ux, uy = d.moments()
    j, i = np.mgrid[0:16, 0:20]
    cx, cy = c0[0] + V[0] * 200, c0[1] + V[1] * 200
    assert np.max(np.abs(ux - (V[0] - om * (j - cy)))) < 1e-5
    assert np.max(np.abs(uy - (V[1] + om * (i - cx)))) < 1e-5
    assert om * V[0] * 200 > 1e-3  # the error a fixed centre would make


@pytest.mark.parametrize("nu,lam", [(0.1, 3 / 16), (0.02, 0.25)])
def test_shear_wave_decay_rate(nu, lam):
    # P6: a shear wave u_x = u0 sin(2 pi j / NY) decays as exp(-nu k^2 t) with
    # nu = c_s^2 (tau_s - 1/2); pins the tau_s <-> nu reading. The lattice error is
    # second order: about 4x smaller per doubling of NY.
    def rel_err(ny):
        nx = 4
        sp = _spec(nx, ny, nu=nu, lam=lam)
        j = np.arange(ny)
        g = np.zeros((9, ny, nx))
        for jj in range(ny):
            g[:, jj, :] = oracle.equilibrium(1.0, 1e-3 * math.sin(2 * math.pi * jj / ny), 0.0)[:, None]
        d = oracle.Domain(sp, g=g)
        s = np.sin(2 * math.pi * j / ny)
        a0 = 2 * np.mean(d.moments()[1][:, 0] * s)
        steps = int(0.3 * ny * ny / (nu * 4 * math.pi ** 2))
        d.run(steps, want_forces=False)
        a1 = 2 * np.mean(d.moments()[1][:, 0] * s)
        k = 2 * math.pi / ny
        return (-math.log(a1 / a0) / steps) / (nu * k * k) - 1.0
    e32, e64 = rel_err(32), rel_err(64)
    assert abs(e64) < 0.01
    assert 3.5 < e32 / e64 < 4.5


def test_srt_reduction():
    # P7: with Lambda = (tau_s - 1/2)^2, tau_a = tau_s and the TRT update with split
    # forcing equals the independently written SRT update with the unsplit Guo term.
    nu = 0.07
    tau = 3 * nu + 0.5
    sp = _spec(27, 21, nu=nu, lam=(tau - 0.5) ** 2,
               edges=synth._edges("inlet", "outflow", "free_slip", "free_slip"), u_in=(0.03, 0.0),
               shapes=[synth._circle(1, 9, 10, 4.5)], bodies=[synth._body(9, 10, 9, omega=4e-3)])
    assert oracle.tau_a(sp) == pytest.approx(oracle.tau_s(sp), rel=1e-15)
    g = synth.random_populations(5, 27, 21)
    a = oracle.Domain(sp, g=g)
    b = oracle.Domain(sp, g=g)
    fa = a.run(20)
    fb = b.run(20, srt=True)
    assert np.max(np.abs(a.g - b.g) / np.abs(b.g)) < 1e-14
    assert np.allclose(fa, fb, rtol=1e-12, atol=1e-16)


# ---- Couette flow (Sec. 3.1) ------------------------------------------------------------------

def _couette_error(sp, srt=False):
    n = sp["nx"]
    ri = sp["shapes"][0]["radius"]
    ro = sp["shapes"][1]["radius"]
    u0 = sp["bodies"][0]["omega"] * ri
    d = oracle.Domain(sp)
    f = d.run(sp["steps"], srt=srt)
    rho, ux, uy = d.moments()
    c = n / 2.0
    j, i = np.mgrid[0:n, 0:n]
    x, y = i - c, j - c
    r = np.hypot(x, y)
    sel = (r >= ri + 1) & (r <= ro - 1)
    rr = np.where(r > 0, r, 1)
    ut = (-y * ux + x * uy) / rr
    ur = (x * ux + y * uy) / rr
    A = -u0 * ri / (ro ** 2 - ri ** 2)
    B = u0 * ri * ro ** 2 / (ro ** 2 - ri ** 2)
    ex = A * rr + B / rr
    err = math.sqrt(((ut - ex)[sel] ** 2).sum() / (ex[sel] ** 2).sum())
    return err, np.abs(ur[sel]).max() / u0, d, f


def test_couette_closed_form_and_trt_properties():
    # P8: steady cylindrical Couette flow between a rotating core (r < 20) and a
    # resting outer solid (r > 50) follows u_theta = A r + B/r (textbook form of the
    # profile of Sec. 3.1) to within the staircase-mask error, with negligible radial
    # flow. TRT's steady error at fixed Lambda does not depend on the viscosity,
    # unlike SRT's; at tau_s = 1.4 TRT is the more accurate of the two (Sec. 3.1).
    sp = synth.couette()
    err, ur, d, f = _couette_error(sp)
    assert err < 0.03 and ur < 0.03
    # P9: the mask and the state are symmetric under a 90-degree rotation about
    # (64, 64) (with periodic wrap), so the net force on the core vanishes.
    n = 128
    rot = [0, 2, 3, 4, 1, 6, 7, 8, 5]  # direction a -> a rotated by +90 degrees
    j, i = np.mgrid[0:n, 0:n]
    src_i, src_j = j % n, (n - i) % n  # node (i, j) came from (j, n - i) under +90 rotation
    grot = np.empty_like(d.g)
    for a in range(9):
        grot[rot[a]] = d.g[a][src_j, src_i]
    assert np.max(np.abs(grot - d.g)) < 1e-13
    assert np.abs(f[-1, 0]).max() < 1e-10
    sp_hi = synth.couette(nu=0.3, steps=8000)
    e_trt, _, _, _ = _couette_error(sp_hi)
    e_srt, _, _, _ = _couette_error(sp_hi, srt=True)
    assert abs(e_trt - err) / err < 0.05
    assert e_trt < e_srt


# ---- diagnostics (Sec. 3) -------------------------------------------------------------------

def test_diagnostics_closed_forms():
    n = np.arange(40000)
    D, U = 40.0, 0.05
    f_true = 0.169 * U / D
    cl = 0.3 * np.sin(2 * math.pi * f_true * n + 0.3) + 0.01
    assert oracle.strouhal(cl, D, U) == pytest.approx(0.169, rel=2e-4)
    assert oracle.rms(cl) == pytest.approx(0.3 / math.sqrt(2), rel=2e-3)
    # a weaker second tone (an acoustic standing wave at 3.5x the frequency) adds zero
    # crossings but leaves the spectral peak at the shedding frequency
    mixed = cl + 0.15 * np.sin(2 * math.pi * 3.5 * f_true * n)
    assert oracle.strouhal_fft(mixed, D, U) == pytest.approx(0.169, rel=3e-3)
    assert oracle.strouhal(mixed, D, U) > 0.2
    cd, cl2 = oracle.coefficients(np.array([[0.5 * U * U * D * 1.3, -0.5 * U * U * D * 0.2]]), U, D)
    assert cd[0] == pytest.approx(1.3) and cl2[0] == pytest.approx(-0.2)
