"""Pins of the oracle's fluid-structure coupling (bodies that move in response to their
force: semi-implicit Euler of M dv/dt = F - k (x - x0) - c v after every step, F the mean
of the last two steps' forces), each against something other than the oracle: an exact
momentum invariant of fluid plus body in a closed box, the closed-form solution of the
discrete damped oscillator when the fluid force vanishes, bit-identity with fixed and
prescribed motion for an infinitely heavy body, fluid damping, the fluid moving with
the body at its current position, the drag direction, and stability for light bodies."""
import math

import numpy as np
import pytest

import oracle
import synth

EX, EY = oracle.EX, oracle.EY


def _momentum(g):
    return float((EX[:, None, None] * g).sum()), float((EY[:, None, None] * g).sum())


def _box(nx, ny, body, shapes, eta=1e-4, nu=0.05):
    sp = synth._spec("fsi_pin", nx, ny, nu, shapes, [body], 0, 0.02, synth._edges(), eta=eta)
    sp["moving"] = True
    return sp


def test_fluid_plus_body_momentum_is_conserved():
    # closed periodic box: the fluid gains -F_n in step n (the force on the body is
    # -sum F_VP) and a free body without springs gains M dv = (F_n + F_{n-1}) / 2, so
    # Q_n = P_fluid + M v + F_{n-1} / 2 is invariant (telescoping). A sign error, a lost
    # force memory or an unfiltered force breaks it.
    M = 3.0 * math.pi * 5.2 ** 2  # three times the mass of the fluid the body displaces
    b = synth._body(20.3, 17.6, 10.0, vx=0.004, vy=-0.003)
    b["dynamics"] = synth.dynamics(M)
    sp = _box(44, 36, b, [synth._circle(1, 20.3, 17.6, 5.2)])
    d = oracle.Domain(sp, g=synth.random_populations(17, 44, 36, 0.1))

    def q():
        px, py = _momentum(d.g)
        return (px + M * d.state[0, 2] + 0.5 * d.state[0, 4], py + M * d.state[0, 3] + 0.5 * d.state[0, 5])

    q0 = q()
    for _ in range(120):
        f = d.run(1)
        qn = q()
        assert abs(qn[0] - q0[0]) < 1e-11 and abs(qn[1] - q0[1]) < 1e-11
        assert np.abs(f).max() > 1e-5
        assert np.array_equal(d.state[0, 4:6], f[0, 0])  # the force memory is this step's force
    moved = math.hypot(d.state[0, 0] - 20.3, d.state[0, 1] - 17.6)
    assert moved > 0.05  # the body did move through the lattice


def test_light_body_stays_bounded():
    # the two-step mean removes the alternating component of the penalized interior's
    # force: a body only 1.5 times heavier than the fluid it displaces stays bounded in
    # a closed box (the force of step n alone makes it diverge within a few dozen steps)
    M = 1.5 * math.pi * 5.2 ** 2
    b = synth._body(20.3, 17.6, 10.0, vx=0.004, vy=-0.003)
    b["dynamics"] = synth.dynamics(M)
    sp = _box(44, 36, b, [synth._circle(1, 20.3, 17.6, 5.2)])
    d = oracle.Domain(sp, g=synth.random_populations(17, 44, 36, 0.1))
    f = d.run(1500)
    assert np.isfinite(f).all() and np.abs(f[-100:]).max() < 0.01 * np.abs(f[:20]).max()
    assert np.abs(d.state[0, 2:4]).max() < 0.01


@pytest.mark.parametrize("zeta_c", [0.0, 0.4])
def test_negligible_fluid_force_gives_the_discrete_oscillator(zeta_c):
    # eta = 1e12: F_VP ~ 1e-14, the body is a discrete oscillator. Semi-implicit Euler
    # with u = y - y0: u_{m+1} = (2 - c/M - k/M) u_m - (1 - c/M) u_{m-1}, u_0 = 0,
    # u_1 = v0 (1 - c/M): u_m = A r^m sin(m theta), r^2 = 1 - c/M,
    # 2 r cos(theta) = 2 - c/M - k/M. The x axis is not free: it keeps vx = 0.
    M, k = 80.0, 2.0
    c = zeta_c
    v0 = 0.02
    b = synth._body(24.0, 20.0, 8.0, vx=0.0, vy=v0)
    b["dynamics"] = synth.dynamics(M, (0.0, k), (0.0, c), free=(0, 1))
    sp = _box(48, 40, b, [synth._circle(1, 24.0, 20.0, 4.0)], eta=1e12)
    d = oracle.Domain(sp)
    n = 300
    track = np.zeros((n, 1, 4))
    d.run(n, track=track)
    r = math.sqrt(1.0 - c / M)
    theta = math.acos((2.0 - c / M - k / M) / (2.0 * r))
    A = v0 * (1.0 - c / M) / (r * math.sin(theta))
    m = np.arange(n)
    want = A * r ** m * np.sin(m * theta)
    u = track[:, 0, 1] - 20.0
    assert np.abs(u - want).max() < 1e-8
    assert np.abs(u).max() > 0.05  # it oscillates with an amplitude of several hundredths
    assert (track[:, 0, 0] == 24.0).all() and (track[:, 0, 2] == 0.0).all()


def test_infinitely_heavy_body_at_rest_is_the_fixed_body():
    # M = 1e300, v0 = 0: velocity increments of ~1e-301 vanish against the centre and
    # against u*, so every step equals the fixed body's, bit for bit.
    b = synth._body(18.4, 15.2, 9.0)
    fixed = _box(40, 31, dict(b), [synth._circle(1, 18.4, 15.2, 4.5)])
    heavy_b = dict(b)
    heavy_b["dynamics"] = synth.dynamics(1e300)
    heavy = _box(40, 31, heavy_b, [synth._circle(1, 18.4, 15.2, 4.5)])
    g0 = synth.random_populations(5, 40, 31)
    a, h = oracle.Domain(fixed, g=g0), oracle.Domain(heavy, g=g0)
    fa, fh = a.run(200), h.run(200)
    assert np.array_equal(a.g, h.g)
    assert np.array_equal(fa, fh)
    assert h.state[0, 0] == 18.4 and h.state[0, 1] == 15.2


def test_fluid_moves_with_the_body_at_its_current_position():
    # a heavy body launched across a fluid at rest: the penalization drags the fluid
    # inside the body at its current position, many cells from where it started.
    M = 1e6
    b = synth._body(32.0, 20.0, 10.0, vx=0.0, vy=0.03)
    b["dynamics"] = synth.dynamics(M, free=(0, 1))
    sp = _box(64, 64, b, [synth._circle(1, 32.0, 20.0, 5.0)], nu=0.1)
    d = oracle.Domain(sp)
    d.run(600, want_forces=False)
    y = d.state[0, 1]
    assert y > 20.0 + 17.0
    st = oracle.stream(sp, d.g)
    rho = st.sum(axis=0)
    uy_star = (EY[:, None, None] * st).sum(axis=0) / rho
    j = int(round(y))
    assert abs(uy_star[j, 32] - d.state[0, 3]) < 0.1 * d.state[0, 3]


def test_infinitely_heavy_moving_body_is_the_prescribed_motion():
    # M = 1e300 launched with velocity V: the velocity never changes and the centre
    # advances by V every step, so each step sees the mask and U_O of the prescribed
    # motion c + V n (positions agree to rounding; no node lies that close to the
    # circle here): identical populations and forces. Using the state after the update
    # for a step, or not moving the shapes, would differ from the first step on.
    V = (0.013, -0.0071)
    b = synth._body(22.4, 19.7, 10.0, vx=V[0], vy=V[1])
    pres = _box(48, 40, dict(b), [synth._circle(1, 22.4, 19.7, 5.1)])
    hb = dict(b)
    hb["dynamics"] = synth.dynamics(1e300)
    heavy = _box(48, 40, hb, [synth._circle(1, 22.4, 19.7, 5.1)])
    g0 = synth.random_populations(23, 48, 40)
    a, h = oracle.Domain(pres, g=g0), oracle.Domain(heavy, g=g0)
    fa, fh = a.run(400), h.run(400)
    assert np.array_equal(a.g, h.g)
    assert np.array_equal(fa, fh)
    assert abs(h.state[0, 0] - (22.4 + 400 * V[0])) < 1e-12
    assert abs(h.state[0, 1] - (19.7 + 400 * V[1])) < 1e-12
    assert np.array_equal(a.mask, h.mask)


def test_free_body_in_a_stream_is_dragged_downstream():
    U = 0.04
    b = synth._body(30.0, 20.0, 10.0)
    b["dynamics"] = synth.dynamics(25.0 * math.pi * 25.0, free=(1, 0))
    sp = synth._spec("drag", 120, 40, 0.05, [synth._circle(1, 30.0, 20.0, 5.0)], [b], 0, U,
                     synth._channel_edges(), u_in=(U, 0.0), u0=(U, 0.0))
    sp["moving"] = True
    d = oracle.Domain(sp)
    track = np.zeros((400, 1, 4))
    d.run(400, track=track)
    vx = track[:, 0, 2]
    # after the first steps of the impulsive start the body accelerates monotonically
    # and stays slower than the stream
    assert (np.diff(vx[3:]) > 0).all() and 0.0 < vx[-1] < U
    assert (track[:, 0, 3] == 0.0).all()


def test_fluid_damps_a_spring_mounted_body():
    # a body on a spring launched across fluid at rest: the penalization drags the fluid
    # with the body's current velocity, so the fluid takes energy out of the oscillation
    # (U_O must follow the body's velocity, not its initial one)
    r = 5.0
    M = 20.0 * math.pi * r * r
    k = M * (2.0 * math.pi / 60.0) ** 2
    b = synth._body(32.0, 32.0, 2 * r, vx=0.0, vy=0.02)
    b["dynamics"] = synth.dynamics(M, (0.0, k), free=(0, 1))
    sp = _box(64, 64, b, [synth._circle(1, 32.0, 32.0, r)], nu=0.05)
    d = oracle.Domain(sp)
    track = np.zeros((600, 1, 4))
    d.run(600, track=track)
    u = track[:, 0, 1] - 32.0
    first, last = np.abs(u[:60]).max(), np.abs(u[-60:]).max()
    assert first > 0.1 and last < 0.7 * first
