"""FP64 CPU oracle of the TRT-LBM-VP method (arXiv:1901.08766) — TEST INFRASTRUCTURE.

Only the tests, the package smoke check and the benchmark's CPU-baseline / reference
arm may import this module. The CUDA library never calls it and shares no code
with it. The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, one node at a
time, in the paper's notation); this file builds it with gcc, marshals numpy
arrays through ctypes and adds the host-side diagnostics (force coefficients and
the Strouhal number, Sec. 3).

Every function here is pinned by the ``-m "not gpu"`` tests against closed forms,
invariants, reductions and brute force (see tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_DEFAULT_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_LIB = _DEFAULT_LIB
_lock = threading.Lock()
_lib = None

EDGE = {"periodic": 0, "inlet": 1, "outflow": 2, "free_slip": 3}
SHAPE = {"circle": 0, "annulus_outside": 1, "naca4": 2}

# D2Q9 constants of the oracle, Eq. (D2Q9) and the weights under Eq. (feq).
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nu", C.c_double),
                ("magic_lambda", C.c_double), ("eta", C.c_double), ("rho0", C.c_double),
                ("u_in_x", C.c_double), ("u_in_y", C.c_double), ("west", C.c_int32),
                ("east", C.c_int32), ("south", C.c_int32), ("north", C.c_int32)]


class _Body(C.Structure):
    _fields_ = [("cx", C.c_double), ("cy", C.c_double), ("vx", C.c_double),
                ("vy", C.c_double), ("omega", C.c_double), ("amp", C.c_double),
                ("rate", C.c_double), ("kappa", C.c_double), ("deform", C.c_int32),
                ("pad", C.c_int32)]


class _Dynamics(C.Structure):
    _fields_ = [("mass", C.c_double), ("kx", C.c_double), ("ky", C.c_double), ("cx", C.c_double),
                ("cy", C.c_double), ("free_x", C.c_int32), ("free_y", C.c_int32),
                ("active", C.c_int32)]


class _Shape(C.Structure):
    _fields_ = [("kind", C.c_int32), ("body", C.c_int32), ("cx", C.c_double),
                ("cy", C.c_double), ("radius", C.c_double), ("chord", C.c_double),
                ("thickness", C.c_double), ("aoa_rad", C.c_double)]


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into _build/liboracle.so (gcc, -O2, no FP contraction)."""
    with _lock:
        if not force and os.path.exists(_LIB) and (
                _LIB != _DEFAULT_LIB or os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-std=c11", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        return _LIB


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops over rows (results do not depend on them:
    nodes are independent and body forces are summed serially afterwards); returns the
    number now in effect."""
    lib()
    gomp = C.CDLL("libgomp.so.1")
    gomp.omp_set_num_threads(int(n))
    gomp.omp_get_max_threads.restype = C.c_int
    return int(gomp.omp_get_max_threads())


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        u8p = C.POINTER(C.c_uint8)
        L.ora_tau_s.restype = C.c_double
        L.ora_tau_s.argtypes = [C.POINTER(_Params)]
        L.ora_tau_a.restype = C.c_double
        L.ora_tau_a.argtypes = [C.POINTER(_Params)]
        L.ora_equilibrium.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.ora_guo.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, dp]
        L.ora_naca_half_thickness.restype = C.c_double
        L.ora_naca_half_thickness.argtypes = [C.c_double, C.c_double, C.c_double]
        L.ora_rasterize.argtypes = [C.c_int32, C.c_int32, C.POINTER(_Shape), C.c_int32, u8p]
        for fn in (L.ora_step_trt, L.ora_step_srt):
            fn.argtypes = [C.POINTER(_Params), u8p, C.POINTER(_Body), C.c_int32, dp, dp, dp]
        L.ora_run.restype = C.c_int
        L.ora_run.argtypes = [C.POINTER(_Params), u8p, C.POINTER(_Body), C.c_int32, dp,
                              C.c_int64, dp, C.c_int32]
        L.ora_init.argtypes = [C.POINTER(_Params), C.c_double, C.c_double, dp]
        L.ora_stream.argtypes = [C.POINTER(_Params), dp, dp]
        L.ora_moments.argtypes = [C.POINTER(_Params), u8p, C.POINTER(_Body), dp, dp, dp, dp]
        L.ora_rasterize_at.argtypes = [C.c_int32, C.c_int32, C.POINTER(_Shape), C.c_int32,
                                       C.POINTER(_Body), C.c_int32, C.c_int64, u8p]
        L.ora_rasterize_rot.restype = None
        L.ora_rasterize_rot.argtypes = L.ora_rasterize_at.argtypes
        L.ora_sincos.restype = None
        L.ora_sincos.argtypes = [C.c_double, dp, dp]
        L.ora_run_moving_mode.restype = C.c_int
        L.ora_run_moving_mode.argtypes = [C.POINTER(_Params), C.POINTER(_Shape), C.c_int32,
                                          C.POINTER(_Body), C.c_int32, dp, C.c_int64, C.c_int64,
                                          dp, C.c_int32, C.c_int32]
        L.ora_run_moving.restype = C.c_int
        L.ora_run_moving.argtypes = [C.POINTER(_Params), C.POINTER(_Shape), C.c_int32,
                                     C.POINTER(_Body), C.c_int32, dp, C.c_int64, C.c_int64, dp,
                                     C.c_int32]
        L.ora_run_fsi.restype = C.c_int
        L.ora_run_fsi.argtypes = [C.POINTER(_Params), C.POINTER(_Shape), C.c_int32,
                                  C.POINTER(_Body), C.POINTER(_Dynamics), C.c_int32, dp,
                                  C.c_int64, C.c_int64, dp, dp, dp]
        L.ora_bodies_at.argtypes = [C.POINTER(_Body), C.c_int32, C.c_int64, C.POINTER(_Body)]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def params_of(spec) -> _Params:
    e = spec["edges"]
    return _Params(spec["nx"], spec["ny"], spec["nu"], spec["magic_lambda"], spec["eta"],
                   spec["rho0"], spec["u_in"][0], spec["u_in"][1], EDGE[e["west"]],
                   EDGE[e["east"]], EDGE[e["south"]], EDGE[e["north"]])


def _shapes_of(spec):
    shp = spec["shapes"]
    arr = (_Shape * max(1, len(shp)))()
    for k, s in enumerate(shp):
        arr[k] = _Shape(SHAPE[s["kind"]], s["body"], s["cx"], s["cy"], s.get("radius", 0.0),
                        s.get("chord", 0.0), s.get("thickness", 0.0), s.get("aoa_rad", 0.0))
    return arr, len(shp)


def _bodies_of(spec):
    bs = spec["bodies"]
    arr = (_Body * max(1, len(bs)))()
    for k, b in enumerate(bs):
        d = b.get("deform")
        arr[k] = _Body(b["cx"], b["cy"], b["vx"], b["vy"], b["omega"],
                       float(d["amplitude"]) if d else 0.0, float(d["rate"]) if d else 0.0, 0.0,
                       1 if d else 0, 0)
    return arr, len(bs)


def tau_s(spec) -> float:
    return lib().ora_tau_s(C.byref(params_of(spec)))


def tau_a(spec) -> float:
    return lib().ora_tau_a(C.byref(params_of(spec)))


def equilibrium(rho, ux, uy) -> np.ndarray:
    out = np.zeros(9)
    lib().ora_equilibrium(rho, ux, uy, _dp(out))
    return out


def guo(ux, uy, fx, fy) -> np.ndarray:
    out = np.zeros(9)
    lib().ora_guo(ux, uy, fx, fy, _dp(out))
    return out


def naca_half_thickness(xc, t=0.12, chord=1.0) -> float:
    return lib().ora_naca_half_thickness(xc, t, chord)


def stream(spec, g) -> np.ndarray:
    """Step (3) alone: the streamed populations f [9, ny, nx] of a state g."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    f = np.zeros_like(g)
    lib().ora_stream(C.byref(params_of(spec)), _dp(g), _dp(f))
    return f


def sincos(t: float):
    """(sin t, cos t) of the oracle's own FP64 evaluation (reduction by pi/2, Taylor)."""
    s, c = C.c_double(), C.c_double()
    lib().ora_sincos(float(t), C.byref(s), C.byref(c))
    return s.value, c.value


def rotating(spec) -> bool:
    """A spec with "moving": 2 turns its bodies' shapes with their angular velocities."""
    m = spec.get("moving", False)
    return not isinstance(m, bool) and m == 2


def rasterize(spec, step=None) -> np.ndarray:
    """Body-id mask uint8 [ny, nx] (0 = fluid) from the spec's shapes; with `step`, the
    mask of a moving domain at that step index (shapes translated with their bodies, and
    turned with them for a rotating domain)."""
    nx, ny = spec["nx"], spec["ny"]
    mask = np.zeros((ny, nx), dtype=np.uint8)
    arr, n = _shapes_of(spec)
    if step is None:
        lib().ora_rasterize(nx, ny, arr, n, mask.ctypes.data_as(C.POINTER(C.c_uint8)))
    else:
        bodies, nb = _bodies_of(spec)
        fn = lib().ora_rasterize_rot if rotating(spec) else lib().ora_rasterize_at
        fn(nx, ny, arr, n, bodies, nb, int(step), mask.ctypes.data_as(C.POINTER(C.c_uint8)))
    return mask


def _dynamics_of(spec):
    """Body dynamics of a spec (bodies with a "dynamics" entry respond to their force)."""
    bs = spec["bodies"]
    arr = (_Dynamics * max(1, len(bs)))()
    any_active = False
    for k, b in enumerate(bs):
        d = b.get("dynamics")
        if d:
            any_active = True
            arr[k] = _Dynamics(d["mass"], d["stiffness"][0], d["stiffness"][1], d["damping"][0],
                               d["damping"][1], int(d["free"][0]), int(d["free"][1]), 1)
    return arr, any_active


class Domain:
    """One simulation: post-collision populations g [9, ny, nx] in FP64. A spec with
    "moving": True has bodies that translate with their velocities (the mask and the
    body centres follow them, re-rasterised before every step); bodies with a
    "dynamics" entry move in response to their force (fluid-structure coupling)."""

    def __init__(self, spec, mask=None, g=None):
        self.spec = spec
        self.p = params_of(spec)
        self.moving = bool(spec.get("moving", False))
        self.rotating = rotating(spec)
        if self.moving and mask is not None:
            raise ValueError("a moving domain's mask follows its shapes")
        self.mask = np.ascontiguousarray(rasterize(spec) if mask is None else mask,
                                         dtype=np.uint8)
        self.bodies, self.nb = _bodies_of(spec)
        self.shapes, self.ns = _shapes_of(spec)
        self.dyn, self.fsi = _dynamics_of(spec)
        if self.fsi and not self.moving:
            raise ValueError("bodies with dynamics need a moving domain")
        if self.fsi and self.rotating:
            raise ValueError("coupled bodies do not turn their shapes (rotating domain)")
        deforming = any(b.get("deform") for b in spec["bodies"])
        if deforming and not self.moving:
            raise ValueError("deforming bodies need a moving domain")
        if deforming and self.fsi:
            raise ValueError("coupled bodies do not deform")
        # (x, y, vx, vy, Fx, Fy) of every body at the current step index (used by coupled
        # bodies; F is the force of the previous step, zero before the first)
        self.state = np.array([[b["cx"], b["cy"], b["vx"], b["vy"], 0.0, 0.0] for b in spec["bodies"]],
                              dtype=np.float64).reshape(-1, 6)
        nx, ny = spec["nx"], spec["ny"]
        if g is None:
            self.g = np.zeros((9, ny, nx))
            lib().ora_init(C.byref(self.p), spec["u0"][0], spec["u0"][1], _dp(self.g))
        else:
            self.g = np.ascontiguousarray(g, dtype=np.float64).copy()
        self.steps_done = 0

    def run(self, n: int, srt: bool = False, want_forces: bool = True, track=None) -> np.ndarray:
        """Advance n steps; returns the force on each body per step, [n, nbodies, 2].
        `track`, an array [n, nbodies, 4], receives the body state each step used."""
        forces = np.zeros((n, max(self.nb, 1), 2)) if want_forces else None
        if self.fsi:
            if srt:
                raise ValueError("coupled bodies are run with the TRT update")
            st = np.ascontiguousarray(self.state).copy()
            tr = None
            if track is not None:
                tr = np.zeros((n, max(self.nb, 1), 4))
            rc = lib().ora_run_fsi(C.byref(self.p), self.shapes, self.ns, self.bodies, self.dyn,
                                   self.nb, _dp(self.g), self.steps_done, n, _dp(st),
                                   _dp(forces) if want_forces else None,
                                   _dp(tr) if tr is not None else None)
            if rc != 0:
                raise MemoryError("oracle run failed to allocate")
            self.state = st
            if tr is not None:
                track[...] = tr[:, : self.nb]
            self.steps_done += n
            self.mask = self._mask_now()
            return forces[:, : self.nb] if want_forces else None
        if self.moving:
            rc = lib().ora_run_moving_mode(C.byref(self.p), self.shapes, self.ns, self.bodies,
                                           self.nb, _dp(self.g), self.steps_done, n,
                                           _dp(forces) if want_forces else None, 1 if srt else 0,
                                           1 if self.rotating else 0)
        else:
            rc = lib().ora_run(C.byref(self.p), self.mask.ctypes.data_as(C.POINTER(C.c_uint8)),
                               self.bodies, self.nb, _dp(self.g), n,
                               _dp(forces) if want_forces else None, 1 if srt else 0)
        if rc != 0:
            raise MemoryError("oracle run failed to allocate")
        self.steps_done += n
        if self.moving:
            self.mask = rasterize(self.spec, self.steps_done)
        return forces[:, : self.nb] if want_forces else None

    def _bodies_now(self):
        """Body table at the current step index (centres moved for a moving domain)."""
        if not self.moving:
            return self.bodies
        out = (_Body * max(1, self.nb))()
        lib().ora_bodies_at(self.bodies, self.nb, self.steps_done, out)
        for k in range(self.nb):
            if self.dyn[k].active:
                out[k].cx, out[k].cy, out[k].vx, out[k].vy = (float(v) for v in self.state[k, :4])
        return out

    def _mask_now(self):
        """The mask at the current step index (coupled bodies at their current state)."""
        if not self.fsi:
            return rasterize(self.spec, self.steps_done)
        spec = dict(self.spec)
        shapes = []
        for s in self.spec["shapes"]:
            s = dict(s)
            k = s["body"] - 1
            if 0 <= k < self.nb and self.dyn[k].active:
                b = self.spec["bodies"][k]
                s["cx"] = s["cx"] + (float(self.state[k, 0]) - b["cx"])
                s["cy"] = s["cy"] + (float(self.state[k, 1]) - b["cy"])
            shapes.append(s)
        spec["shapes"] = shapes
        spec["bodies"] = [dict(b, vx=0.0, vy=0.0) if self.dyn[k].active else b
                          for k, b in enumerate(self.spec["bodies"])]
        return rasterize(spec, self.steps_done)

    def step_once(self, srt: bool = False):
        """One step returning (new g, forces [nbodies, 2]) without the run wrapper."""
        out = np.zeros_like(self.g)
        fb = np.zeros((max(self.nb, 1), 2))
        fn = lib().ora_step_srt if srt else lib().ora_step_trt
        fn(C.byref(self.p), self.mask.ctypes.data_as(C.POINTER(C.c_uint8)), self._bodies_now(),
           self.nb, _dp(self.g), _dp(out), _dp(fb))
        if self.fsi:
            raise ValueError("use run() for coupled bodies")
        self.g = out
        self.steps_done += 1
        if self.moving:
            self.mask = rasterize(self.spec, self.steps_done)
        return out, fb[: self.nb]

    def moments(self):
        nx, ny = self.spec["nx"], self.spec["ny"]
        rho, ux, uy = (np.zeros((ny, nx)) for _ in range(3))
        lib().ora_moments(C.byref(self.p), self.mask.ctypes.data_as(C.POINTER(C.c_uint8)),
                          self._bodies_now(), _dp(self.g), _dp(rho), _dp(ux), _dp(uy))
        return rho, ux, uy


# ---- diagnostics (Sec. 3: Re, C_d, C_l, St) ---------------------------------------------

def coefficients(forces, U, ref_length, rho0=1.0):
    """C_d = 2 F_x / (rho U^2 D), C_l = 2 F_y / (rho U^2 D) for a [n, 2] force series."""
    f = np.asarray(forces, dtype=np.float64)
    s = 2.0 / (rho0 * U * U * ref_length)
    return f[:, 0] * s, f[:, 1] * s


def strouhal(signal, ref_length, U, dt=1.0):
    """St = f_q D / U from the upward zero crossings of (signal - mean), linearly
    interpolated, over whole periods between the first and last crossing."""
    x = np.asarray(signal, dtype=np.float64)
    x = x - x.mean()
    t_cross = []
    for n in range(len(x) - 1):
        if x[n] < 0.0 <= x[n + 1]:
            t_cross.append((n + (-x[n]) / (x[n + 1] - x[n])) * dt)
    if len(t_cross) < 2:
        return 0.0
    periods = len(t_cross) - 1
    f = periods / (t_cross[-1] - t_cross[0])
    return f * ref_length / U


def strouhal_fft(signal, ref_length, U, dt=1.0):
    """St = f_q D / U with f_q the largest peak of the amplitude spectrum of the
    Hann-windowed (signal - mean), refined by a parabola through the log amplitudes of
    the peak bin and its two neighbours. Unlike zero crossings it is not disturbed by a
    weaker oscillation at another frequency (the channel's acoustic standing wave)."""
    x = np.asarray(signal, dtype=np.float64)
    n = len(x)
    if n < 8:
        return 0.0
    x = x - x.mean()
    win = 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(n) / n)
    amp = np.abs(np.fft.rfft(x * win))
    k = 1 + int(np.argmax(amp[1:-1]))
    a, b, c = np.log(amp[k - 1] + 1e-300), np.log(amp[k] + 1e-300), np.log(amp[k + 1] + 1e-300)
    den = a - 2.0 * b + c
    shift = 0.5 * (a - c) / den if den != 0.0 else 0.0
    f = (k + shift) / (n * dt)
    return f * ref_length / U


def rms(signal):
    x = np.asarray(signal, dtype=np.float64)
    return float(np.sqrt(np.mean((x - x.mean()) ** 2)))
