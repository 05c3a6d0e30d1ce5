"""FP64 CPU oracle of the TRT-LBM-VP method in 3D (D3Q19 or D3Q15) — TEST INFRASTRUCTURE.

The arithmetic lives in ``lbm_oracle3d.c`` (plain C, FP64, one node at a time); this
module builds it with gcc and marshals numpy arrays. Only the tests and the benchmark's
CPU baseline use it; the CUDA library never does. Pinned by tests/test_oracle3d_pins.py.

Spec of a 3D case: nx, ny, nz, nu, magic_lambda, eta, rho0, u_in (3), u0 (3), edges
{west, east, south, north, bottom, top}, shapes [{kind: sphere | cylinder_z, body,
c (3), radius}], bodies [{c, v, w (3 each), ref_length}], and optionally lattice 19
(default, D3Q19) or 15 (D3Q15).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "lbm_oracle3d.c")
_DEFAULT_LIB = os.path.join(_HERE, "_build", "liboracle3d.so")
_LIB = _DEFAULT_LIB
_lock = threading.Lock()
_lib = None

EDGE = {"periodic": 0, "inlet": 1, "outflow": 2, "free_slip": 3}
SHAPE = {"sphere": 0, "cylinder_z": 1}


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nu", C.c_double),
                ("magic_lambda", C.c_double), ("eta", C.c_double), ("rho0", C.c_double),
                ("u_in", C.c_double * 3), ("west", C.c_int32), ("east", C.c_int32),
                ("south", C.c_int32), ("north", C.c_int32), ("bottom", C.c_int32),
                ("top", C.c_int32), ("q", C.c_int32)]


class _Body(C.Structure):
    _fields_ = [("c", C.c_double * 3), ("v", C.c_double * 3), ("w", C.c_double * 3),
                ("amp", C.c_double), ("rate", C.c_double), ("kappa", C.c_double),
                ("deform", C.c_int32), ("pad", C.c_int32)]


class _Dynamics(C.Structure):
    _fields_ = [("mass", C.c_double), ("k", C.c_double * 3), ("c", C.c_double * 3),
                ("free_axis", C.c_int32 * 3), ("active", C.c_int32)]


def _dynamics_of(spec):
    """Body dynamics of a 3D spec (bodies with a "dynamics" entry respond to their force:
    mass, stiffness (3), damping (3), free (3))."""
    bs = spec["bodies"]
    arr = (_Dynamics * max(1, len(bs)))()
    active = False
    for k, b in enumerate(bs):
        d = b.get("dynamics")
        if d:
            active = True
            arr[k] = _Dynamics(d["mass"], (C.c_double * 3)(*d["stiffness"]), (C.c_double * 3)(*d["damping"]),
                               (C.c_int32 * 3)(*[int(v) for v in d["free"]]), 1)
    return arr, active


class _Shape(C.Structure):
    _fields_ = [("kind", C.c_int32), ("body", C.c_int32), ("c", C.c_double * 3),
                ("radius", C.c_double)]


def build(force: bool = False) -> str:
    with _lock:
        if not force and os.path.exists(_LIB) and (
                _LIB != _DEFAULT_LIB or os.path.getmtime(_LIB) >= os.path.getmtime(SRC)):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-std=c11", "-fopenmp", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        u8p = C.POINTER(C.c_uint8)
        i32p = C.POINTER(C.c_int32)
        P, B, S = C.POINTER(_Params), C.POINTER(_Body), C.POINTER(_Shape)
        L.ora3_tau_s.restype = C.c_double
        L.ora3_tau_s.argtypes = [P]
        L.ora3_tau_a.restype = C.c_double
        L.ora3_tau_a.argtypes = [P]
        L.ora3_equilibrium.argtypes = [C.c_int32, C.c_double, dp, dp]
        L.ora3_guo.argtypes = [C.c_int32, dp, dp, dp]
        L.ora3_rasterize.argtypes = [C.c_int32, C.c_int32, C.c_int32, S, C.c_int32, u8p]
        L.ora3_stream.argtypes = [P, dp, dp]
        L.ora3_step_trt.argtypes = [P, u8p, B, C.c_int32, dp, dp, dp]
        L.ora3_run.restype = C.c_int
        L.ora3_run.argtypes = [P, u8p, B, C.c_int32, dp, C.c_int64, dp]
        L.ora3_init.argtypes = [P, dp, dp]
        L.ora3_moments.argtypes = [P, u8p, B, dp, dp, dp, dp, dp]
        L.ora3_rasterize_at.argtypes = [C.c_int32, C.c_int32, C.c_int32, S, C.c_int32, B, C.c_int32,
                                        C.c_int64, u8p]
        L.ora3_run_fsi.restype = C.c_int
        L.ora3_run_fsi.argtypes = [P, S, C.c_int32, B, C.POINTER(_Dynamics), C.c_int32, dp, C.c_int64,
                                   C.c_int64, dp, dp, dp]
        L.ora3_sincos.restype = None
        L.ora3_sincos.argtypes = [C.c_double, dp, dp]
        L.ora3_bodies_at.restype = None
        L.ora3_bodies_at.argtypes = [B, C.c_int32, C.c_int64, B]
        L.ora3_run_moving.restype = C.c_int
        L.ora3_run_moving.argtypes = [P, S, C.c_int32, B, C.c_int32, dp, C.c_int64, C.c_int64, dp]
        L.ora3_lattice.restype = C.c_int32
        L.ora3_lattice.argtypes = [C.c_int32, i32p, i32p, i32p, dp, i32p]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u8(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _vec(x):
    return (C.c_double * 3)(*[float(v) for v in x])


def nq(spec_or_q=19) -> int:
    """Number of directions of a spec's lattice (or of a lattice given as 15 or 19)."""
    q = spec_or_q.get("lattice", 19) if isinstance(spec_or_q, dict) else int(spec_or_q)
    return 15 if q == 15 else 19


def lattice(q=19):
    """(EX, EY, EZ, W, OPP) of the oracle's D3Q19 (q = 19) or D3Q15 (q = 15) velocity set."""
    n = nq(q)
    ex, ey, ez, opp = (np.zeros(n, dtype=np.int32) for _ in range(4))
    w = np.zeros(n)
    i32 = C.POINTER(C.c_int32)
    got = lib().ora3_lattice(n, ex.ctypes.data_as(i32), ey.ctypes.data_as(i32), ez.ctypes.data_as(i32),
                             _dp(w), opp.ctypes.data_as(i32))
    assert got == n
    return ex, ey, ez, w, opp


def params_of(spec) -> _Params:
    e = spec["edges"]
    return _Params(spec["nx"], spec["ny"], spec["nz"], spec["nu"], spec["magic_lambda"],
                   spec["eta"], spec["rho0"], _vec(spec["u_in"]), EDGE[e["west"]],
                   EDGE[e["east"]], EDGE[e["south"]], EDGE[e["north"]], EDGE[e["bottom"]],
                   EDGE[e["top"]], nq(spec))


def _shapes_of(spec):
    shp = spec["shapes"]
    arr = (_Shape * max(1, len(shp)))()
    for k, s in enumerate(shp):
        arr[k] = _Shape(SHAPE[s["kind"]], s["body"], _vec(s["c"]), s["radius"])
    return arr, len(shp)


def _bodies_of(spec):
    bs = spec["bodies"]
    arr = (_Body * max(1, len(bs)))()
    for k, b in enumerate(bs):
        d = b.get("deform")
        arr[k] = _Body(_vec(b["c"]), _vec(b["v"]), _vec(b["w"]), float(d["amplitude"]) if d else 0.0,
                       float(d["rate"]) if d else 0.0, 0.0, 1 if d else 0, 0)
    return arr, len(bs)


def tau_s(spec):
    return lib().ora3_tau_s(C.byref(params_of(spec)))


def equilibrium(rho, u, q=19):
    out = np.zeros(nq(q))
    lib().ora3_equilibrium(nq(q), rho, _dp(np.ascontiguousarray(u, dtype=np.float64)), _dp(out))
    return out


def guo(u, F, q=19):
    out = np.zeros(nq(q))
    lib().ora3_guo(nq(q), _dp(np.ascontiguousarray(u, dtype=np.float64)),
                   _dp(np.ascontiguousarray(F, dtype=np.float64)), _dp(out))
    return out


def sincos(t: float):
    """(sin t, cos t) of the 3D oracle's own FP64 evaluation (reduction by pi/2, Taylor)."""
    s, c = C.c_double(), C.c_double()
    lib().ora3_sincos(float(t), C.byref(s), C.byref(c))
    return s.value, c.value


def rasterize(spec, step=None):
    """Body-id mask uint8 [nz, ny, nx]; with `step`, the mask of a moving domain at that
    step index (shapes translated with their bodies)."""
    m = np.zeros((spec["nz"], spec["ny"], spec["nx"]), dtype=np.uint8)
    arr, n = _shapes_of(spec)
    if step is None:
        lib().ora3_rasterize(spec["nx"], spec["ny"], spec["nz"], arr, n, _u8(m))
    else:
        bodies, nb = _bodies_of(spec)
        lib().ora3_rasterize_at(spec["nx"], spec["ny"], spec["nz"], arr, n, bodies, nb, int(step), _u8(m))
    return m


def stream(spec, g):
    g = np.ascontiguousarray(g, dtype=np.float64)
    f = np.zeros_like(g)
    lib().ora3_stream(C.byref(params_of(spec)), _dp(g), _dp(f))
    return f


class Domain:
    """One 3D simulation: post-collision populations g [Q, nz, ny, nx] in FP64. A spec with
    "moving": True has bodies that translate with their velocities (mask and centres
    follow them before every step)."""

    def __init__(self, spec, mask=None, g=None):
        self.spec = spec
        self.p = params_of(spec)
        self.moving = bool(spec.get("moving", False))
        if self.moving and mask is not None:
            raise ValueError("a moving domain's mask follows its shapes")
        self.mask = np.ascontiguousarray(rasterize(spec) if mask is None else mask, dtype=np.uint8)
        self.bodies, self.nb = _bodies_of(spec)
        self.shapes, self.ns = _shapes_of(spec)
        self.dyn, self.fsi = _dynamics_of(spec)
        if self.fsi and not self.moving:
            raise ValueError("bodies with dynamics need a moving domain")
        deforming = any(b.get("deform") for b in spec["bodies"])
        if deforming and not self.moving:
            raise ValueError("deforming bodies need a moving domain")
        for s in spec["shapes"]:
            if s["kind"] != "sphere" and spec["bodies"][s["body"] - 1].get("deform"):
                raise ValueError("a pulsating 3D body is made of spheres (its dilation is isotropic)")
        if deforming and self.fsi:
            raise ValueError("coupled bodies do not deform")
        # x[3], v[3] and the previous step's force[3] of every body (used by coupled bodies)
        self.state = np.array([list(b["c"]) + list(b["v"]) + [0.0, 0.0, 0.0] for b in spec["bodies"]],
                              dtype=np.float64).reshape(-1, 9)
        shape = (nq(spec), spec["nz"], spec["ny"], spec["nx"])
        if g is None:
            self.g = np.zeros(shape)
            lib().ora3_init(C.byref(self.p), _dp(np.asarray(spec["u0"], dtype=np.float64)), _dp(self.g))
        else:
            self.g = np.ascontiguousarray(g, dtype=np.float64).copy()
        self.steps_done = 0

    def run(self, n: int, want_forces: bool = True, track=None):
        """Advance n steps; the force on each body per step, [n, nbodies, 3]. `track`, an
        array [n, nbodies, 6], receives each coupled run's (x, v) of every step."""
        forces = np.zeros((n, max(self.nb, 1), 3)) if want_forces else None
        if self.fsi:
            st = np.ascontiguousarray(self.state).copy()
            tr = np.zeros((n, max(self.nb, 1), 6)) if track is not None else None
            rc = lib().ora3_run_fsi(C.byref(self.p), self.shapes, self.ns, self.bodies, self.dyn, self.nb,
                                    _dp(self.g), self.steps_done, n, _dp(st),
                                    _dp(forces) if want_forces else None, _dp(tr) if tr is not None else None)
            if rc != 0:
                raise MemoryError("oracle run failed to allocate")
            self.state = st
            if tr is not None:
                track[...] = tr[:, : self.nb]
            self.steps_done += n
            self.mask = self._mask_now()
            return forces[:, : self.nb] if want_forces else None
        if self.moving:
            rc = lib().ora3_run_moving(C.byref(self.p), self.shapes, self.ns, self.bodies, self.nb,
                                       _dp(self.g), self.steps_done, n, _dp(forces) if want_forces else None)
        else:
            rc = lib().ora3_run(C.byref(self.p), _u8(self.mask), self.bodies, self.nb, _dp(self.g), n,
                                _dp(forces) if want_forces else None)
        if rc != 0:
            raise MemoryError("oracle run failed to allocate")
        self.steps_done += n
        if self.moving:
            self.mask = rasterize(self.spec, self.steps_done)
        return forces[:, : self.nb] if want_forces else None

    def bodies_now(self):
        """Body table at the current step index (centres moved for a moving domain, coupled
        bodies at their state): [nbodies, 9] (c, v, w)."""
        out = np.array([list(b["c"]) + list(b["v"]) + list(b["w"]) for b in self.spec["bodies"]],
                       dtype=np.float64).reshape(-1, 9)
        if self.moving:
            out[:, 0:3] = out[:, 0:3] + out[:, 3:6] * float(self.steps_done)
        for k in range(self.nb):
            if self.fsi and self.dyn[k].active:
                out[k, 0:6] = self.state[k, 0:6]
        return out

    def _mask_now(self):
        """The mask at the current step index (coupled bodies at their current state)."""
        if not self.fsi:
            return rasterize(self.spec, self.steps_done)
        shapes = []
        for s in self.spec["shapes"]:
            k = s["body"] - 1
            if 0 <= k < self.nb and self.dyn[k].active:
                c0 = self.spec["bodies"][k]["c"]
                s = dict(s, c=tuple(s["c"][d] + (float(self.state[k, d]) - c0[d]) for d in range(3)))
            shapes.append(s)
        bodies = [dict(b, v=(0.0, 0.0, 0.0)) if self.dyn[k].active else b
                  for k, b in enumerate(self.spec["bodies"])]
        return rasterize(dict(self.spec, shapes=shapes, bodies=bodies), self.steps_done)

    def step_once(self):
        if self.moving:
            raise ValueError("use run() for a moving domain")
        out = np.zeros_like(self.g)
        fb = np.zeros((max(self.nb, 1), 3))
        lib().ora3_step_trt(C.byref(self.p), _u8(self.mask), self.bodies, self.nb, _dp(self.g),
                            _dp(out), _dp(fb))
        self.g = out
        self.steps_done += 1
        return out, fb[: self.nb]

    def moments(self):
        shp = (self.spec["nz"], self.spec["ny"], self.spec["nx"])
        rho, ux, uy, uz = (np.zeros(shp) for _ in range(4))
        bodies = self.bodies
        if self.moving:
            bodies = (_Body * max(1, self.nb))()
            lib().ora3_bodies_at(self.bodies, self.nb, self.steps_done, bodies)  # incl. kappa
            for k, row in enumerate(self.bodies_now()):
                for d in range(3):
                    bodies[k].c[d], bodies[k].v[d] = float(row[d]), float(row[3 + d])
        lib().ora3_moments(C.byref(self.p), _u8(self.mask), bodies, _dp(self.g), _dp(rho),
                           _dp(ux), _dp(uy), _dp(uz))
        return rho, ux, uy, uz
