"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only draws random numbers and lays out problem descriptions. It holds
none of the method's arithmetic: no lattice weights, equilibria, relaxation rates,
masks or forces. Both the FP64 oracle (``oracle/``) and the CUDA library read the
plain dictionaries produced here and derive everything else on their own side.

Random numbers come from SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds and a final xor-shift. Doubles in [0, 1) are
(x >> 11) * 2^-53.

A problem description (``spec``) is a dict with keys:

  name, nx, ny                 grid size; node (i, j) sits at (i, j), i along the flow
  nu                           kinematic viscosity in lattice units
  magic_lambda, eta, rho0      TRT magic parameter, penalization parameter, reference density
  u_in, u0                     inlet velocity (ux, uy); uniform initial velocity (ux, uy)
  edges                        {"west": "periodic"|"inlet", "east": "periodic"|"outflow",
                                "south"/"north": "periodic"|"free_slip"}
  shapes                       list of {"kind": "circle"|"annulus_outside"|"naca4", "body": k,
                                "cx", "cy", "radius", "chord", "thickness", "aoa_rad"};
                                later shapes overwrite earlier ones
  bodies                       list of {"cx", "cy", "vx", "vy", "omega", "ref_length"};
                                body k (1-based) is bodies[k-1]; rigid motion V + omega x (x - c)
  steps                        number of time steps of the workload
  U                            free-stream speed used for force coefficients
"""
from __future__ import annotations

import math

import numpy as np

_MASK64 = (1 << 64) - 1

# Seeds of the workloads (the paper's arXiv number and its successor).
SEED_BATCH = 190108766
SEED_SERVED = 190108767


class SplitMix64:
    """SplitMix64 counter-based generator (Steele, Lea & Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def next_double(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.next_double()

    def doubles(self, n: int) -> np.ndarray:
        """n doubles in [0, 1), vectorised; identical to n calls of next_double()."""
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + idx * np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * 0x9E3779B97F4A7C15) & _MASK64
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# Typical magnitudes of the nine populations of a near-rest state, grouped as
# rest / axis / diagonal. These are round numbers owned by this generator, not
# the lattice weights of any model.
_POP_SCALE = np.array([0.44, 0.11, 0.11, 0.11, 0.11, 0.028, 0.028, 0.028, 0.028])


def random_populations(seed: int, nx: int, ny: int, amp: float = 0.1) -> np.ndarray:
    """Positive random populations, float64 array of shape [9, ny, nx].

    Value = scale[q] * (1 + amp * (xi - 0.5)), xi drawn in (q, j, i) order.
    Any positive set of nine values is a valid lattice state; this one carries
    density ~0.98 and velocities of order 1e-2 with cell-to-cell noise.
    """
    xi = SplitMix64(seed).doubles(9 * ny * nx).reshape(9, ny, nx)
    return _POP_SCALE[:, None, None] * (1.0 + amp * (xi - 0.5))


# --------------------------------------------------------------------------------------
# Problem descriptions.

def _edges(west="periodic", east="periodic", south="periodic", north="periodic"):
    return {"west": west, "east": east, "south": south, "north": north}


def _channel_edges():
    return _edges("inlet", "outflow", "free_slip", "free_slip")


def _circle(body, cx, cy, radius):
    return {"kind": "circle", "body": body, "cx": float(cx), "cy": float(cy),
            "radius": float(radius)}


def _body(cx, cy, ref_length, vx=0.0, vy=0.0, omega=0.0):
    return {"cx": float(cx), "cy": float(cy), "vx": float(vx), "vy": float(vy),
            "omega": float(omega), "ref_length": float(ref_length)}


def dynamics(mass, stiffness=(0.0, 0.0), damping=(0.0, 0.0), free=(1, 1)):
    """Rigid-body dynamics of a coupled body: mass, springs (k_x, k_y) anchored at the
    initial centre, dampers (c_x, c_y), and which axes respond to the force."""
    return {"mass": float(mass), "stiffness": (float(stiffness[0]), float(stiffness[1])),
            "damping": (float(damping[0]), float(damping[1])), "free": (int(free[0]), int(free[1]))}


def spring_cylinder(nx=480, ny=240, D=24.0, U=0.05, re=100.0, mass_ratio=10.0,
                    reduced_velocity=5.0, zeta=0.0, steps=40000):
    """An elastically mounted cylinder free to move across the stream (y): mass ratio
    m* = M / (rho0 pi D^2 / 4), natural frequency f_n = U / (U* D), spring k = M (2 pi f_n)^2,
    damping c = 2 zeta M 2 pi f_n; uniform inflow, zero-gradient outflow, free-slip walls."""
    nu = U * D / re
    cx, cy = nx / 4.0, ny / 2.0
    M = mass_ratio * math.pi * D * D / 4.0
    wn = 2.0 * math.pi * U / (reduced_velocity * D)
    body = _body(cx, cy, D)
    body["dynamics"] = dynamics(M, (0.0, M * wn * wn), (0.0, 2.0 * zeta * M * wn), free=(0, 1))
    sp = _spec(f"spring_cylinder_{nx}x{ny}_re{re:g}_ur{reduced_velocity:g}", nx, ny, nu,
               [_circle(1, cx, cy, D / 2.0)], [body], steps, U, _channel_edges(),
               u_in=(U, 0.0), u0=(U, 0.0))
    sp["moving"] = True
    return sp


def _spec(name, nx, ny, nu, shapes, bodies, steps, U, edges, u_in=(0.0, 0.0),
          u0=(0.0, 0.0), magic_lambda=3.0 / 16.0, eta=1e-4, rho0=1.0):
    return {"name": name, "nx": int(nx), "ny": int(ny), "nu": float(nu),
            "magic_lambda": float(magic_lambda), "eta": float(eta), "rho0": float(rho0),
            "u_in": (float(u_in[0]), float(u_in[1])), "u0": (float(u0[0]), float(u0[1])),
            "edges": edges, "shapes": shapes, "bodies": bodies, "steps": int(steps),
            "U": float(U)}


def couette(n=128, r_inner=20.0, r_outer=50.0, u_wall=0.01, nu=0.1, steps=20000,
            magic_lambda=3.0 / 16.0, eta=1e-4):
    """Cylindrical Couette flow (paper Sec. 3.1): rotating solid core r < R_i, resting
    solid outside r > R_o, periodic box. Defaults: the 128x128 FP64 workload."""
    c = n / 2.0
    shapes = [_circle(1, c, c, r_inner),
              {"kind": "annulus_outside", "body": 2, "cx": c, "cy": c,
               "radius": float(r_outer)}]
    bodies = [_body(c, c, 2 * r_inner, omega=u_wall / r_inner), _body(c, c, 2 * r_outer)]
    return _spec(f"couette_{n}", n, n, nu, shapes, bodies, steps, u_wall, _edges(),
                 magic_lambda=magic_lambda, eta=eta)


def single_cylinder(nx=1600, ny=800, D=40.0, cx=400.0, cy=400.0, U=0.05, re=100.0,
                    steps=200000):
    """Flow past one fixed cylinder (paper Sec. 3.2) in a channel with uniform inflow,
    zero-gradient outflow and free-slip lateral edges."""
    nu = U * D / re
    return _spec(f"cylinder_{nx}x{ny}_re{re:g}", nx, ny, nu, [_circle(1, cx, cy, D / 2)],
                 [_body(cx, cy, D)], steps, U, _channel_edges(), u_in=(U, 0.0),
                 u0=(U, 0.0))


def precision_cylinder(large=True):
    """Re=200 cylinder of the precision sweep: 2400x1200 with D=60 at (600, 600), U=0.05
    (300k steps); or the oracle-sized 600x300 case. At that size D=15 (grid Reynolds
    number U/nu = 13) diverges in the FP64 oracle within 1500 steps at U=0.05 and at
    U=0.1, so the small case uses D=30 (U/nu = 6.7), offset half a cell in y so that
    shedding does not wait for roundoff to break the symmetry, 80k steps (shedding
    saturates after about 40k)."""
    if large:
        return single_cylinder(2400, 1200, 60.0, 600.0, 600.0, 0.05, 200.0, 300000)
    return single_cylinder(600, 300, 30.0, 150.0, 150.5, 0.05, 200.0, 80000)


def _fits_tandem(W, H, D, L):
    xu = max(W / 4.0 - L / 2.0, 2 * D)
    return xu + L <= W - 4 * D and H / 2.0 - D / 2.0 >= D


def _fits_side(W, H, D, gap):
    half = (D + gap) / 2.0
    return H / 2.0 - half - D / 2.0 >= D and max(W / 4.0, 2 * D) <= W - 4 * D


def batched_domains(n=64, seed=SEED_BATCH, steps=50000, D=40.0, U=0.05, log=None):
    """The batched uneven-domain workload: n domains, first half tandem pairs
    (centre spacing L/D in [1.5, 6]) and second half side-by-side pairs (surface gap
    g/D in [0.5, 3]). Per domain, draws in order: W in [400, 2000] (rounded to even),
    Re in [40, 200], then the spacing, redrawn up to 20 times until the pair fits
    (upstream centre >= 2D from the inlet, downstream centre <= W - 4D, >= 1D lateral
    clearance), else clamped to the largest fitting spacing."""
    rng = SplitMix64(seed)
    specs = []
    for d in range(n):
        W = 2 * int(round(rng.uniform(400.0, 2000.0) / 2.0))
        H = W // 2
        re = rng.uniform(40.0, 200.0)
        nu = U * D / re
        tandem = d < n // 2
        lo, hi = (1.5, 6.0) if tandem else (0.5, 3.0)
        fits = _fits_tandem if tandem else _fits_side
        val = None
        for _ in range(20):
            cand = rng.uniform(lo, hi)
            if fits(W, H, D, cand * D):
                val = cand
                break
        if val is None:
            # largest spacing on a 1/1000 grid that fits (at least the lower end)
            val = lo
            k = int(math.floor((hi - lo) * 1000))
            for s in range(k, -1, -1):
                cand = lo + s / 1000.0
                if fits(W, H, D, cand * D):
                    val = cand
                    break
            if log is not None:
                log.append((d, "clamped", val))
        if tandem:
            L = val * D
            xu = max(W / 4.0 - L / 2.0, 2 * D)
            c = [(xu, H / 2.0), (xu + L, H / 2.0)]
        else:
            half = (D + val * D) / 2.0
            x = max(W / 4.0, 2 * D)
            c = [(x, H / 2.0 + half), (x, H / 2.0 - half)]
        shapes = [_circle(k + 1, cx, cy, D / 2) for k, (cx, cy) in enumerate(c)]
        bodies = [_body(cx, cy, D) for (cx, cy) in c]
        sp = _spec(f"batch{d:02d}_{'tandem' if tandem else 'side'}_{W}x{H}", W, H, nu,
                   shapes, bodies, steps, U, _channel_edges(), u_in=(U, 0.0), u0=(U, 0.0))
        sp["arrangement"] = ("tandem", val) if tandem else ("side_by_side", val)
        sp["re"] = re
        specs.append(sp)
    return specs


def counter_rotating_pair(alpha, re=100.0, D=40.0, U=0.05, nx=1200, ny=600, gap=3.0,
                          steps=50000):
    """Two counter-rotating cylinders stacked across the flow (paper Sec. 3.4), surface
    gap `gap`*D, pair midpoint at (H/2, H/2); rotation rate alpha = Omega D / (2U);
    upper cylinder clockwise (Omega < 0), lower counter-clockwise."""
    nu = U * D / re
    om = 2.0 * alpha * U / D
    half = (D + gap * D) / 2.0
    x, y = ny / 2.0, ny / 2.0
    c = [(x, y + half, -om), (x, y - half, om)]
    shapes = [_circle(k + 1, cx, cy, D / 2) for k, (cx, cy, _) in enumerate(c)]
    bodies = [_body(cx, cy, D, omega=o) for (cx, cy, o) in c]
    sp = _spec(f"rotating_a{alpha:.3f}", nx, ny, nu, shapes, bodies, steps, U,
               _channel_edges(), u_in=(U, 0.0), u0=(U, 0.0))
    sp["alpha"] = alpha
    return sp


def naca0012(aoa_deg, re, chord=200.0, U=0.05, nx=2000, ny=1000, steps=50000):
    """NACA-0012 airfoil (paper Sec. 3.5), quarter chord at (H/2, H/2), nose-up AOA
    positive; Re on the chord."""
    nu = U * chord / re
    x, y = ny / 2.0, ny / 2.0
    shapes = [{"kind": "naca4", "body": 1, "cx": x, "cy": y, "chord": float(chord),
               "thickness": 0.12, "aoa_rad": math.radians(aoa_deg)}]
    bodies = [_body(x, y, chord)]
    sp = _spec(f"naca0012_aoa{aoa_deg:.2f}_re{re:.0f}", nx, ny, nu, shapes, bodies,
               steps, U, _channel_edges(), u_in=(U, 0.0), u0=(U, 0.0))
    sp["aoa_deg"] = aoa_deg
    sp["re"] = re
    return sp


def paper_pair(arrangement, spacing, re=200.0, D=40.0, U=0.05, nx=2048, ny=1024, steps=240000):
    """A pair of fixed cylinders as in the paper's pair experiments (Sec. 3.3): domain
    2048 x 1024, D = 40, Re 200, centre-to-centre distance `spacing` * D, pair midpoint at
    (H/2, H/2 + 1/2) (half a cell off the axis so that shedding does not wait for
    roundoff); "tandem" along the flow, "side" across it. Body 1 is the upstream (tandem)
    or upper (side-by-side) cylinder."""
    nu = U * D / re
    mx, my = ny / 2.0, ny / 2.0 + 0.5
    half = spacing * D / 2.0
    c = [(mx - half, my), (mx + half, my)] if arrangement == "tandem" else [(mx, my + half), (mx, my - half)]
    shapes = [_circle(k + 1, x, y, D / 2) for k, (x, y) in enumerate(c)]
    bodies = [_body(x, y, D) for (x, y) in c]
    sp = _spec(f"{arrangement}_{spacing:g}D_re{re:g}", nx, ny, nu, shapes, bodies, steps, U,
               _channel_edges(), u_in=(U, 0.0), u0=(U, 0.0))
    sp["arrangement"], sp["spacing"] = arrangement, spacing
    return sp


def paper_rotating_pair(omega_n, re=150.0, D=40.0, U=0.02, nx=2048, ny=1024, steps=300000):
    """The paper's two counter-rotating cylinders (Sec. 3.4): side by side, centre-to-centre
    distance 2D, midpoint at (H/2, H/2), Re 150, normalized rotation rate
    omega_n = Omega D / (2 U); the upper cylinder turns clockwise, the lower one
    counter-clockwise (their surfaces move upstream in the gap). U = 0.02 keeps the surface
    speed omega_n U at 0.08 or less (the paper's U = 0.01 gives tau_s = 0.508; at
    omega_n = 1.5 both give the lower cylinder's C_d and C_l within 1 %)."""
    sp = counter_rotating_pair(omega_n, re=re, D=D, U=U, nx=nx, ny=ny, gap=1.0, steps=steps)
    sp["name"] = f"rotating_w{omega_n:g}_re{re:g}"
    return sp


def served_requests(seed=SEED_SERVED, rate=20.0, duration=600.0, step_lo=20000,
                    step_hi=100000):
    """Poisson request stream of the served workload: arrival time, then a 50/50
    draw between a counter-rotating pair (alpha in [0, 2], Re 100, 1200x600) and a
    NACA-0012 (AOA in [0, 10] deg, Re in [500, 1000], 2000x1000), then the step
    count in [step_lo, step_hi]. Returns a list of (arrival_s, spec)."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    while True:
        t += -math.log(1.0 - rng.next_double()) / rate
        if t >= duration:
            break
        if rng.next_double() < 0.5:
            sp = counter_rotating_pair(rng.uniform(0.0, 2.0))
        else:
            aoa = rng.uniform(0.0, 10.0)
            sp = naca0012(aoa, rng.uniform(500.0, 1000.0))
        sp["steps"] = int(step_lo + (step_hi - step_lo) * rng.next_double())
        out.append((t, sp))
    return out


def parity_case(name: str):
    """Small cases for GPU-vs-oracle parity: odd/unaligned and aligned grids, two
    circles (one rotating), periodic or channel edges, both magic parameters."""
    if name == "periodic_97x61":
        shapes = [_circle(1, 30.0, 30.0, 9.0), _circle(2, 70.0, 33.0, 6.0)]
        bodies = [_body(30.0, 30.0, 18.0, omega=2e-3), _body(70.0, 33.0, 12.0, vx=0.01)]
        return _spec(name, 97, 61, 0.06, shapes, bodies, 1000, 0.02, _edges(),
                     magic_lambda=3.0 / 16.0)
    if name == "channel_97x61":
        shapes = [_circle(1, 25.0, 31.0, 7.0), _circle(2, 55.0, 20.0, 5.0)]
        bodies = [_body(25.0, 31.0, 14.0, omega=-1.5e-3), _body(55.0, 20.0, 10.0)]
        return _spec(name, 97, 61, 0.04, shapes, bodies, 1000, 0.03, _channel_edges(),
                     u_in=(0.03, 0.0), u0=(0.03, 0.0), magic_lambda=0.25)
    if name == "channel_256x128":
        shapes = [_circle(1, 60.0, 64.0, 12.0), _circle(2, 140.0, 50.0, 10.0)]
        bodies = [_body(60.0, 64.0, 24.0, omega=1e-3), _body(140.0, 50.0, 20.0)]
        return _spec(name, 256, 128, 0.05, shapes, bodies, 1000, 0.04, _channel_edges(),
                     u_in=(0.04, 0.0), u0=(0.04, 0.0), magic_lambda=3.0 / 16.0)
    if name == "mixed_edges_61x47":
        # periodic in x, free-slip in y, one NACA section and one circle
        shapes = [{"kind": "naca4", "body": 1, "cx": 25.0, "cy": 23.0, "chord": 30.0,
                   "thickness": 0.12, "aoa_rad": math.radians(8.0)},
                  _circle(2, 50.0, 10.0, 4.0)]
        bodies = [_body(25.0, 23.0, 30.0), _body(50.0, 10.0, 8.0, vy=0.005)]
        return _spec(name, 61, 47, 0.03, shapes, bodies, 1000, 0.02,
                     _edges("periodic", "periodic", "free_slip", "free_slip"),
                     u0=(0.02, 0.0), magic_lambda=0.25)
    raise KeyError(name)


PARITY_CASES = ("periodic_97x61", "channel_97x61", "channel_256x128", "mixed_edges_61x47")


# --------------------------------------------------------------------------------------
# 3D (D3Q19) inputs: same conventions, nineteen directions (rest, six axis, twelve face
# diagonals), arrays [19, nz, ny, nx].

_POP_SCALE3 = {19: np.array([0.33] + [0.055] * 6 + [0.028] * 12),
               15: np.array([0.22] + [0.11] * 6 + [0.014] * 8)}


def random_populations3(seed: int, nx: int, ny: int, nz: int, amp: float = 0.1, q: int = 19) -> np.ndarray:
    """Positive random populations [q, nz, ny, nx] of D3Q19 (q = 19) or D3Q15 (q = 15):
    scale[a] * (1 + amp * (xi - 0.5)), xi drawn in (a, k, j, i) order (density ~0.99,
    velocities of order 1e-2)."""
    xi = SplitMix64(seed).doubles(q * nz * ny * nx).reshape(q, nz, ny, nx)
    return _POP_SCALE3[q][:, None, None, None] * (1.0 + amp * (xi - 0.5))


def edges3(west="periodic", east="periodic", south="periodic", north="periodic",
           bottom="periodic", top="periodic"):
    return {"west": west, "east": east, "south": south, "north": north, "bottom": bottom,
            "top": top}


def channel_edges3():
    return edges3("inlet", "outflow", "free_slip", "free_slip", "free_slip", "free_slip")


def sphere(body, c, radius):
    return {"kind": "sphere", "body": int(body), "c": tuple(float(v) for v in c), "radius": float(radius)}


def cylinder_z(body, cx, cy, radius):
    return {"kind": "cylinder_z", "body": int(body), "c": (float(cx), float(cy), 0.0),
            "radius": float(radius)}


def body3(c, ref_length, v=(0.0, 0.0, 0.0), w=(0.0, 0.0, 0.0)):
    return {"c": tuple(float(x) for x in c), "v": tuple(float(x) for x in v),
            "w": tuple(float(x) for x in w), "ref_length": float(ref_length)}


def spec3(name, nx, ny, nz, nu, shapes, bodies, steps, U, edges, u_in=(0.0, 0.0, 0.0),
          u0=(0.0, 0.0, 0.0), magic_lambda=3.0 / 16.0, eta=1e-4, rho0=1.0, lattice=19):
    return {"name": name, "lattice": int(lattice), "nx": int(nx), "ny": int(ny), "nz": int(nz), "nu": float(nu),
            "magic_lambda": float(magic_lambda), "eta": float(eta), "rho0": float(rho0),
            "u_in": tuple(float(v) for v in u_in), "u0": tuple(float(v) for v in u0),
            "edges": edges, "shapes": shapes, "bodies": bodies, "steps": int(steps), "U": float(U)}


def sphere_channel(nx=384, ny=128, nz=128, D=32.0, U=0.05, re=100.0, steps=20000):
    """Flow past a sphere in a channel (uniform inflow, zero-gradient outflow, free-slip
    walls): the 3D counterpart of the single-cylinder case, sphere centre off the axes
    by half a cell."""
    nu = U * D / re
    c = (nx / 4.0, ny / 2.0 + 0.5, nz / 2.0 + 0.5)
    return spec3(f"sphere_{nx}x{ny}x{nz}_re{re:g}", nx, ny, nz, nu, [sphere(1, c, D / 2)],
                 [body3(c, D)], steps, U, channel_edges3(), u_in=(U, 0.0, 0.0), u0=(U, 0.0, 0.0))
