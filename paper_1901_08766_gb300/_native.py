"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every computation runs in the CUDA library; this module converts problem descriptions
into the ABI's structs, hands PyTorch's caching allocator and current stream to the
library, and raises on any non-OK status. There is no CPU fallback: loading fails
loudly if the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import _compile as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_EBUSY, LBM_ENOTFOUND = range(8)
STORAGE = {"f64": 0, "f32": 1, "f16s": 2, "bf16s": 3}
STORAGE_DTYPE = {"f64": np.float64, "f32": np.float32, "f16s": np.float16, "bf16s": np.uint16}
ELEM_SIZE = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}
EDGE = {"periodic": 0, "inlet": 1, "outflow": 2, "free_slip": 3}
SHAPE = {"circle": 0, "annulus_outside": 1, "naca4": 2}


class LbmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nu", C.c_double),
                ("tau_plus", C.c_double), ("magic_lambda", C.c_double), ("eta", C.c_double),
                ("rho0", C.c_double), ("u_in_x", C.c_double), ("u_in_y", C.c_double),
                ("u0_x", C.c_double), ("u0_y", C.c_double), ("west", C.c_int32),
                ("east", C.c_int32), ("south", C.c_int32), ("north", C.c_int32),
                ("storage", C.c_int32), ("force_every", C.c_int32),
                ("force_capacity", C.c_int32), ("moving", C.c_int32), ("x_origin", C.c_int32)]


class Body(C.Structure):
    _fields_ = [("cx", C.c_double), ("cy", C.c_double), ("vx", C.c_double),
                ("vy", C.c_double), ("omega", C.c_double), ("ref_length", C.c_double)]


class Shape(C.Structure):
    _fields_ = [("kind", C.c_int32), ("body", C.c_int32), ("cx", C.c_double),
                ("cy", C.c_double), ("radius", C.c_double), ("chord", C.c_double),
                ("thickness", C.c_double), ("aoa_rad", C.c_double)]


class Geometry(C.Structure):
    _fields_ = [("shapes", C.POINTER(Shape)), ("nshapes", C.c_int32)]


class BodyDynamics(C.Structure):
    _fields_ = [("mass", C.c_double), ("stiffness", C.c_double * 2), ("damping", C.c_double * 2),
                ("free_axis", C.c_int32 * 2)]


def dynamics_from(d) -> BodyDynamics:
    return BodyDynamics(d["mass"], (C.c_double * 2)(*d["stiffness"]), (C.c_double * 2)(*d["damping"]),
                        (C.c_int32 * 2)(*[int(v) for v in d["free"]]))


class BodyDynamics3(C.Structure):
    _fields_ = [("mass", C.c_double), ("stiffness", C.c_double * 3), ("damping", C.c_double * 3),
                ("free_axis", C.c_int32 * 3)]


def dynamics3_from(d) -> BodyDynamics3:
    return BodyDynamics3(d["mass"], (C.c_double * 3)(*d["stiffness"]), (C.c_double * 3)(*d["damping"]),
                         (C.c_int32 * 3)(*[int(v) for v in d["free"]]))


def moving_mode(spec) -> int:
    """0 fixed, 1 translating bodies ("moving": True), 2 bodies that also turn their shapes
    ("moving": 2)."""
    m = spec.get("moving", False)
    if isinstance(m, bool) or m in (0, 1):
        return 1 if m else 0
    return int(m)


class Params3(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nu", C.c_double),
                ("tau_plus", C.c_double), ("magic_lambda", C.c_double), ("eta", C.c_double),
                ("rho0", C.c_double), ("u_in", C.c_double * 3), ("u0", C.c_double * 3),
                ("west", C.c_int32), ("east", C.c_int32), ("south", C.c_int32),
                ("north", C.c_int32), ("bottom", C.c_int32), ("top", C.c_int32),
                ("storage", C.c_int32), ("force_every", C.c_int32),
                ("force_capacity", C.c_int32), ("lattice", C.c_int32), ("moving", C.c_int32)]


class Body3(C.Structure):
    _fields_ = [("c", C.c_double * 3), ("v", C.c_double * 3), ("w", C.c_double * 3),
                ("ref_length", C.c_double)]


class Shape3(C.Structure):
    _fields_ = [("kind", C.c_int32), ("body", C.c_int32), ("c", C.c_double * 3),
                ("radius", C.c_double)]


SHAPE3 = {"sphere": 0, "cylinder_z": 1}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

# Every symbol the header declares, with (restype, argtypes).
_VP, _I32, _I64, _SZ, _D = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.c_double
_DP = C.POINTER(C.c_double)
SIGNATURES = {
    "lbm_params_default": (None, [C.POINTER(Params)]),
    "lbm_status_string": (C.c_char_p, [C.c_int]),
    "lbm_last_error": (C.c_char_p, []),
    "lbm_domain_bytes": (_SZ, [C.POINTER(Params), _I32]),
    "lbm_domain_create": (C.c_int, [C.POINTER(Params), C.c_void_p, C.POINTER(Geometry),
                                    C.POINTER(Body), _I32, _VP, ALLOC_FN, FREE_FN, _VP,
                                    C.POINTER(_VP)]),
    "lbm_step": (C.c_int, [_VP, _I64]),
    "lbm_forces": (C.c_int, [_VP, _DP, _I64, C.POINTER(_I64)]),
    "lbm_moments": (C.c_int, [_VP, _VP, _VP, _VP]),
    "lbm_moments_noalloc": (C.c_int, [_VP, _VP, _VP, _VP]),
    "lbm_get_populations": (C.c_int, [_VP, _VP, _SZ]),
    "lbm_set_populations": (C.c_int, [_VP, _VP, _SZ]),
    "lbm_steps_done": (C.c_int, [_VP, C.POINTER(_I64)]),
    "lbm_set_steps_done": (C.c_int, [_VP, _I64]),
    "lbm_get_mask": (C.c_int, [_VP, _VP]),
    "lbm_batch_get_mask": (C.c_int, [_VP, _I32, _VP]),
    "lbm_domain_destroy": (C.c_int, [_VP]),
    "lbm_batch_create": (C.c_int, [_I32, _SZ, _I32, _I32, _VP, ALLOC_FN, FREE_FN, _VP,
                                   C.POINTER(_VP)]),
    "lbm_batch_admit": (C.c_int, [_VP, C.POINTER(Params), C.c_void_p, C.POINTER(Geometry),
                                  C.POINTER(Body), _I32, _I64, C.POINTER(_I32)]),
    "lbm_batch_run": (C.c_int, [_VP, _I64, C.POINTER(_I64)]),
    "lbm_batch_admit_many": (C.c_int, [_VP, _I32, C.POINTER(Params), C.POINTER(Geometry),
                                       C.POINTER(C.POINTER(Body)), C.POINTER(_I32), C.POINTER(_I64),
                                       C.POINTER(_I32)]),
    "lbm_batch_poll": (C.c_int, [_VP, _I32, _DP, _I64, C.POINTER(_I64), C.POINTER(_I32)]),
    "lbm_batch_moments": (C.c_int, [_VP, _I32, _VP, _VP, _VP]),
    "lbm_batch_poll_many": (C.c_int, [_VP, _I32, C.POINTER(_I32), C.POINTER(_DP), C.POINTER(_I64),
                                      C.POINTER(_I64), C.POINTER(_I32), C.POINTER(_I32)]),
    "lbm_batch_get_populations": (C.c_int, [_VP, _I32, _VP, _SZ]),
    "lbm_batch_set_populations": (C.c_int, [_VP, _I32, _VP, _SZ]),
    "lbm_batch_steps_done": (C.c_int, [_VP, _I32, C.POINTER(_I64)]),
    "lbm_batch_link_x": (C.c_int, [_VP, _I32, _I32]),
    "lbm_batch_set_steps_done": (C.c_int, [_VP, _I32, _I64]),
    "lbm_batch_profile": (C.c_int, [_VP, _I32, _DP, _DP, C.POINTER(_I64)]),
    "lbm_batch_evict": (C.c_int, [_VP, _I32]),
    "lbm_batch_inject": (C.c_int, [_VP, _I32, _I32]),
    "lbm_batch_set_halo": (C.c_int, [_VP, _I32, _I32, _VP, _VP]),
    "lbm_batch_pack_halos": (C.c_int, [_VP]),
    "lbm_batch_capture": (C.c_int, [_VP]),
    "lbm_batch_autotune": (C.c_int, [_VP, _I32, _DP]),
    "lbm_batch_set_tile": (C.c_int, [_VP, _I32, _I32, _I32, _I32]),
    "lbm_batch_set_grouped_admission": (C.c_int, [_VP, _I32]),
    "lbm_batch_get_tile": (C.c_int, [_VP, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32),
                                     C.POINTER(_I32)]),
    "lbm_batch_info": (C.c_int, [_VP, C.POINTER(_I32), C.POINTER(_I64), C.POINTER(_I64),
                                 C.POINTER(_SZ)]),
    "lbm_batch_destroy": (C.c_int, [_VP]),
    "lbm_batch_set_dynamics": (C.c_int, [_VP, _I32, _I32, C.POINTER(BodyDynamics)]),
    "lbm_set_dynamics": (C.c_int, [_VP, _I32, C.POINTER(BodyDynamics)]),
    "lbm_batch_set_deformation": (C.c_int, [_VP, _I32, _I32, C.c_double, C.c_double]),
    "lbm_set_deformation": (C.c_int, [_VP, _I32, C.c_double, C.c_double]),
    "lbm_batch_body_state": (C.c_int, [_VP, _I32, _DP]),
    "lbm_body_state": (C.c_int, [_VP, _DP]),
    "lbm_batch_coupled_state": (C.c_int, [_VP, _I32, _DP]),
    "lbm_coupled_state": (C.c_int, [_VP, _DP]),
    "lbm_batch_restore_coupled": (C.c_int, [_VP, _I32, _I64, _DP]),
    "lbm_restore_coupled": (C.c_int, [_VP, _I64, _DP]),
    "lbm3_params_default": (None, [C.POINTER(Params3)]),
    "lbm3_domain_bytes": (_SZ, [C.POINTER(Params3), _I32]),
    "lbm3_domain_create": (C.c_int, [C.POINTER(Params3), C.POINTER(Shape3), _I32,
                                     C.POINTER(Body3), _I32, _VP, ALLOC_FN, FREE_FN, _VP,
                                     C.POINTER(_VP)]),
    "lbm3_step": (C.c_int, [_VP, _I64]),
    "lbm3_forces": (C.c_int, [_VP, _DP, _I64, C.POINTER(_I64)]),
    "lbm3_moments": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "lbm3_get_populations": (C.c_int, [_VP, _VP, _SZ]),
    "lbm3_set_populations": (C.c_int, [_VP, _VP, _SZ]),
    "lbm3_get_mask": (C.c_int, [_VP, _VP]),
    "lbm3_steps_done": (C.c_int, [_VP, C.POINTER(_I64)]),
    "lbm3_set_steps_done": (C.c_int, [_VP, _I64]),
    "lbm3_set_dynamics": (C.c_int, [_VP, _I32, C.POINTER(BodyDynamics3)]),
    "lbm3_body_state": (C.c_int, [_VP, _DP]),
    "lbm3_set_deformation": (C.c_int, [_VP, _I32, C.c_double, C.c_double]),
    "lbm3_coupled_state": (C.c_int, [_VP, _DP]),
    "lbm3_restore_coupled": (C.c_int, [_VP, _I64, _DP]),
    "lbm3_profile": (C.c_int, [_VP, _I32, _DP, _DP]),
    "lbm3_set_tile": (C.c_int, [_VP, _I32]),
    "lbm3_get_tile": (C.c_int, [_VP, C.POINTER(_I32)]),
    "lbm3_autotune": (C.c_int, [_VP, _I32, _DP]),
    "lbm3_domain_destroy": (C.c_int, [_VP]),
    "lbm3_batch_create": (C.c_int, [_I32, C.c_size_t, _I32, _I32, _VP, ALLOC_FN, FREE_FN, _VP,
                                    C.POINTER(_VP)]),
    "lbm3_batch_admit": (C.c_int, [_VP, C.POINTER(Params3), C.POINTER(Shape3), _I32,
                                   C.POINTER(Body3), _I32, _I64, C.POINTER(_I32)]),
    "lbm3_batch_run": (C.c_int, [_VP, _I64, C.POINTER(_I64)]),
    "lbm3_batch_poll": (C.c_int, [_VP, _I32, _DP, _I64, C.POINTER(_I64), C.POINTER(_I32)]),
    "lbm3_batch_domain": (C.c_int, [_VP, _I32, C.POINTER(_VP)]),
    "lbm3_batch_evict": (C.c_int, [_VP, _I32]),
    "lbm3_batch_set_tile": (C.c_int, [_VP, _I32]),
    "lbm3_batch_info": (C.c_int, [_VP, C.POINTER(_I32), C.POINTER(_I64), C.POINTER(_I64),
                                  C.POINTER(C.c_size_t), C.POINTER(_I32)]),
    "lbm3_batch_destroy": (C.c_int, [_VP]),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB_PATH


def load(path: str | None = None):
    """Load the compiled library (built by __graft_entry__.build() or build.py)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or library_path()
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built ({p} missing); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def check(status: int, where: str):
    if status != LBM_OK:
        detail = _lib.lbm_last_error().decode(errors="replace") if _lib else ""
        raise LbmError(status, where, detail)


# ---- marshalling of problem descriptions ------------------------------------------------

def params_from_spec(spec, storage: str, force_every: int = 1, force_capacity: int = 8192) -> Params:
    e = spec["edges"]
    return Params(spec["nx"], spec["ny"], spec["nu"], 0.0, spec["magic_lambda"], spec["eta"],
                  spec["rho0"], spec["u_in"][0], spec["u_in"][1], spec["u0"][0], spec["u0"][1],
                  EDGE[e["west"]], EDGE[e["east"]], EDGE[e["south"]], EDGE[e["north"]],
                  STORAGE[storage], force_every, force_capacity, moving_mode(spec),
                  int(spec.get("x_origin", 0)))


def bodies_from_spec(spec):
    bs = spec["bodies"]
    arr = (Body * max(1, len(bs)))()
    for k, b in enumerate(bs):
        arr[k] = Body(b["cx"], b["cy"], b["vx"], b["vy"], b["omega"], b["ref_length"])
    return arr, len(bs)


def geometry_from_spec(spec):
    shp = spec["shapes"]
    arr = (Shape * max(1, len(shp)))()
    for k, s in enumerate(shp):
        arr[k] = Shape(SHAPE[s["kind"]], s["body"], s["cx"], s["cy"], s.get("radius", 0.0),
                       s.get("chord", 0.0), s.get("thickness", 0.0), s.get("aoa_rad", 0.0))
    g = Geometry(arr, len(shp))
    return g, arr


class ManyDomains:
    """The admission arguments of many domains, built in one pass into numpy arrays laid
    out as the C structures (the same bytes as params_from_spec, geometry_from_spec and
    bodies_from_spec per domain, without a ctypes object per field)."""

    def __init__(self, specs, storage: str, force_every: int, force_capacity: int, nsteps):
        pd, sd, bd = np.dtype(Params), np.dtype(Shape), np.dtype(Body)
        gd = np.dtype({"names": ["shapes", "nshapes"], "formats": [np.uintp, np.int32],
                       "offsets": [0, 8], "itemsize": C.sizeof(Geometry)})
        st = STORAGE[storage]
        self.params = np.array(
            [(sp["nx"], sp["ny"], sp["nu"], 0.0, sp["magic_lambda"], sp["eta"], sp["rho0"],
              sp["u_in"][0], sp["u_in"][1], sp["u0"][0], sp["u0"][1],
              EDGE[sp["edges"]["west"]], EDGE[sp["edges"]["east"]], EDGE[sp["edges"]["south"]],
              EDGE[sp["edges"]["north"]], st, force_every, force_capacity, moving_mode(sp),
              int(sp.get("x_origin", 0))) for sp in specs], dtype=pd)
        shapes = [(SHAPE[s["kind"]], s["body"], s["cx"], s["cy"], s.get("radius", 0.0),
                   s.get("chord", 0.0), s.get("thickness", 0.0), s.get("aoa_rad", 0.0))
                  for sp in specs for s in sp["shapes"]]
        self.shapes = np.array(shapes or [(0, 0) + (0.0,) * 6], dtype=sd)
        bodies = [(b["cx"], b["cy"], b["vx"], b["vy"], b["omega"], b["ref_length"])
                  for sp in specs for b in sp["bodies"]]
        self.bodies = np.array(bodies or [(0.0,) * 6], dtype=bd)
        ns = np.array([len(sp["shapes"]) for sp in specs], dtype=np.int64)
        self.nbodies = np.array([len(sp["bodies"]) for sp in specs], dtype=np.int32)
        self.geometry = np.zeros(len(specs), dtype=gd)
        self.geometry["shapes"] = self.shapes.ctypes.data + sd.itemsize * (np.cumsum(ns) - ns)
        self.geometry["nshapes"] = ns
        nb = self.nbodies.astype(np.int64)
        self.body_ptrs = (self.bodies.ctypes.data + bd.itemsize * (np.cumsum(nb) - nb)).astype(np.uintp)
        self.nsteps = np.array(nsteps, dtype=np.int64)

    def args(self):
        """(params, geometries, body pointers, body counts, step counts) as the pointers
        lbm_batch_admit_many takes; valid while this object lives."""
        return (self.params.ctypes.data_as(C.POINTER(Params)),
                self.geometry.ctypes.data_as(C.POINTER(Geometry)),
                self.body_ptrs.ctypes.data_as(C.POINTER(C.POINTER(Body))),
                self.nbodies.ctypes.data_as(C.POINTER(_I32)),
                self.nsteps.ctypes.data_as(C.POINTER(_I64)))


def params3_from_spec(spec, storage: str, force_every: int = 1,
                      force_capacity: int = 8192) -> Params3:
    e = spec["edges"]
    return Params3(spec["nx"], spec["ny"], spec["nz"], spec["nu"], 0.0, spec["magic_lambda"],
                   spec["eta"], spec["rho0"], (C.c_double * 3)(*spec["u_in"]),
                   (C.c_double * 3)(*spec["u0"]), EDGE[e["west"]], EDGE[e["east"]],
                   EDGE[e["south"]], EDGE[e["north"]], EDGE[e["bottom"]], EDGE[e["top"]],
                   STORAGE[storage], force_every, force_capacity, int(spec.get("lattice", 19)),
                   moving_mode(spec))


def bodies3_from_spec(spec):
    bs = spec["bodies"]
    arr = (Body3 * max(1, len(bs)))()
    for k, b in enumerate(bs):
        arr[k] = Body3((C.c_double * 3)(*b["c"]), (C.c_double * 3)(*b["v"]),
                       (C.c_double * 3)(*b["w"]), b["ref_length"])
    return arr, len(bs)


def shapes3_from_spec(spec):
    shp = spec["shapes"]
    arr = (Shape3 * max(1, len(shp)))()
    for k, s in enumerate(shp):
        arr[k] = Shape3(SHAPE3[s["kind"]], s["body"], (C.c_double * 3)(*s["c"]), s["radius"])
    return arr, len(shp)


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.live = {}
        self.c_alloc = ALLOC_FN(self._alloc)
        self.c_free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:  # out of memory: the library reports LBM_ENOMEM
            return None
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, ctx):
        self.live.pop(ptr, None)


def current_stream_handle():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)
