"""GB300-native TRT-LBM-VP (arXiv:1901.08766): flows past obstacles with the coupled
two-relaxation-time lattice Boltzmann / volume-penalization method.

The compute path is the CUDA library built from ``csrc/`` (C ABI in include/lbm.h);
this package marshals arguments to it and provides host-side helpers (force
coefficients and Strouhal number, the request server). PyTorch supplies device memory
and the CUDA stream.

    import paper_1901_08766_gb300 as lbm
    dom = lbm.Domain(spec, storage="f16s")   # spec: see the synth module's description
    dom.step(1000)
    forces = dom.forces()                    # [steps, nbodies, 2], force on each body
    rho, ux, uy = dom.moments()
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native
from ._native import (ELEM_SIZE, LBM_EBUSY, LBM_EUNSTABLE, LbmError, STORAGE, STORAGE_DTYPE,
                      check, load)
from ._compile import build

__all__ = ["Domain", "Domain3", "Batch", "load", "build", "LbmError", "STORAGE", "domain_bytes"]


def _mask_arg(mask):
    if mask is None:
        return None, None
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    return m, m.ctypes.data_as(C.c_void_p)


def _allocator(allocator):
    """"torch": PyTorch's caching allocator; None: the library's own stream-ordered
    allocation; otherwise an object with ctypes callbacks `c_alloc` and `c_free`."""
    if allocator == "torch":
        return _native.TorchAllocator()
    return allocator


def domain_bytes(spec, storage="f32", force_every=1, force_capacity=8192) -> int:
    L = load()
    p = _native.params_from_spec(spec, storage, force_every, force_capacity)
    return int(L.lbm_domain_bytes(C.byref(p), len(spec["bodies"])))


class Domain:
    """One simulation domain on the current CUDA device (lbm_domain_* calls)."""

    def __init__(self, spec, storage="f32", force_every=1, force_capacity=8192, mask=None,
                 stream=None, allocator="torch"):
        import torch
        L = load()
        self.spec, self.storage = spec, storage
        self.nx, self.ny = spec["nx"], spec["ny"]
        self.nbodies = len(spec["bodies"])
        self._params = _native.params_from_spec(spec, storage, force_every, force_capacity)
        self._bodies, nb = _native.bodies_from_spec(spec)
        self._geom, self._shapes = _native.geometry_from_spec(spec)
        m, mp = _mask_arg(mask)
        self._alloc = _allocator(allocator)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        check(L.lbm_domain_create(C.byref(self._params), mp, C.byref(self._geom), self._bodies,
                                  nb, C.c_void_p(self._stream.cuda_stream),
                                  self._alloc.c_alloc if self._alloc else _native.ALLOC_FN(),
                                  self._alloc.c_free if self._alloc else _native.FREE_FN(),
                                  None, C.byref(h)), "lbm_domain_create")
        self._h = h
        for k, b in enumerate(spec["bodies"]):
            if b.get("dynamics"):
                dyn = _native.dynamics_from(b["dynamics"])
                check(L.lbm_set_dynamics(h, k + 1, C.byref(dyn)), "lbm_set_dynamics")
            if b.get("deform"):  # a pulsating body
                check(L.lbm_set_deformation(h, k + 1, float(b["deform"]["amplitude"]),
                                            float(b["deform"]["rate"])), "lbm_set_deformation")

    def body_state(self) -> np.ndarray:
        """Body table of the current step: [nbodies, 5] (cx, cy, vx, vy, omega); coupled
        bodies report their integrated state."""
        out = np.zeros((max(self.nbodies, 1), 5))
        check(load().lbm_body_state(self._handle(), out.ctypes.data_as(C.POINTER(C.c_double))),
              "lbm_body_state")
        return out[: self.nbodies]

    def coupled_state(self) -> np.ndarray:
        """Checkpoint of coupled bodies: [nbodies, 6] (x, y, vx, vy, previous Fx, Fy)."""
        out = np.zeros((max(self.nbodies, 1), 6))
        check(load().lbm_coupled_state(self._handle(), out.ctypes.data_as(C.POINTER(C.c_double))),
              "lbm_coupled_state")
        return out[: self.nbodies]

    def restore_coupled(self, steps: int, state):
        """Resume a domain with coupled bodies at a step index with a saved coupled state
        (set the populations first)."""
        a = np.ascontiguousarray(state, dtype=np.float64).reshape(self.nbodies, 6)
        check(load().lbm_restore_coupled(self._handle(), int(steps), a.ctypes.data_as(C.POINTER(C.c_double))),
              "lbm_restore_coupled")

    def _handle(self):
        if self._h is None:
            raise RuntimeError("domain destroyed")
        return self._h

    def step(self, n: int):
        check(load().lbm_step(self._handle(), int(n)), "lbm_step")

    def run(self, n: int, chunk: int = 4096):
        """Advance n steps, draining the force ring between chunks; returns the forces."""
        out = []
        left = int(n)
        while left > 0:
            k = min(chunk, left)
            self.step(k)
            out.append(self.forces())
            left -= k
        if not out:
            return np.zeros((0, self.nbodies, 2))
        return np.concatenate(out, axis=0)

    def forces(self, max_entries: int | None = None) -> np.ndarray:
        L = load()
        cap = self._params.force_capacity if max_entries is None else int(max_entries)
        buf = np.zeros((cap, max(self.nbodies, 1), 2))
        w = C.c_int64()
        check(L.lbm_forces(self._handle(), buf.ctypes.data_as(C.POINTER(C.c_double)), cap,
                           C.byref(w)), "lbm_forces")
        return buf[: w.value, : self.nbodies].copy()

    def moments(self):
        rho, ux, uy = (np.zeros((self.ny, self.nx)) for _ in range(3))
        check(load().lbm_moments(self._handle(), rho.ctypes.data_as(C.c_void_p),
                                 ux.ctypes.data_as(C.c_void_p), uy.ctypes.data_as(C.c_void_p)),
              "lbm_moments")
        return rho, ux, uy

    def get_populations(self) -> np.ndarray:
        out = np.zeros((9, self.ny, self.nx), dtype=STORAGE_DTYPE[self.storage])
        check(load().lbm_get_populations(self._handle(), out.ctypes.data_as(C.c_void_p),
                                         out.nbytes), "lbm_get_populations")
        return out

    def set_populations(self, arr: np.ndarray):
        a = np.ascontiguousarray(arr, dtype=STORAGE_DTYPE[self.storage])
        if a.shape != (9, self.ny, self.nx):
            raise ValueError(f"populations must have shape (9, {self.ny}, {self.nx})")
        check(load().lbm_set_populations(self._handle(), a.ctypes.data_as(C.c_void_p), a.nbytes),
              "lbm_set_populations")

    def steps_done(self) -> int:
        v = C.c_int64()
        check(load().lbm_steps_done(self._handle(), C.byref(v)), "lbm_steps_done")
        return v.value

    def set_steps_done(self, steps: int):
        """Restore the step index with saved populations (it keys the 16-bit rounding)."""
        check(load().lbm_set_steps_done(self._handle(), int(steps)), "lbm_set_steps_done")

    def mask(self) -> np.ndarray:
        out = np.zeros((self.ny, self.nx), dtype=np.uint8)
        check(load().lbm_get_mask(self._handle(), out.ctypes.data_as(C.c_void_p)), "lbm_get_mask")
        return out

    def close(self):
        if self._h is not None:
            load().lbm_domain_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Domain3:
    """One 3D simulation domain (D3Q19, or D3Q15 with spec["lattice"] = 15) on the current
    CUDA device (lbm3_* calls). Populations are [Q, nz, ny, nx]; forces are
    [entries, nbodies, 3]."""

    def __init__(self, spec, storage="f32", force_every=1, force_capacity=8192, stream=None,
                 allocator="torch"):
        import torch
        L = load()
        self.spec, self.storage = spec, storage
        self.nx, self.ny, self.nz = spec["nx"], spec["ny"], spec["nz"]
        self.q = 15 if spec.get("lattice", 19) == 15 else 19
        self.nbodies = len(spec["bodies"])
        self._params = _native.params3_from_spec(spec, storage, force_every, force_capacity)
        self._bodies, nb = _native.bodies3_from_spec(spec)
        self._shapes, ns = _native.shapes3_from_spec(spec)
        self._alloc = _allocator(allocator)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        check(L.lbm3_domain_create(C.byref(self._params), self._shapes, ns, self._bodies, nb,
                                   C.c_void_p(self._stream.cuda_stream),
                                   self._alloc.c_alloc if self._alloc else _native.ALLOC_FN(),
                                   self._alloc.c_free if self._alloc else _native.FREE_FN(),
                                   None, C.byref(h)), "lbm3_domain_create")
        self._h = h
        for k, b in enumerate(spec["bodies"]):  # coupled bodies (fluid-structure coupling)
            if b.get("dynamics"):
                dyn = _native.dynamics3_from(b["dynamics"])
                rc = L.lbm3_set_dynamics(h, k + 1, C.byref(dyn))
                if rc != 0:
                    self.close()
                    check(rc, "lbm3_set_dynamics")
            if b.get("deform"):  # a pulsating body
                rc = L.lbm3_set_deformation(h, k + 1, float(b["deform"]["amplitude"]), float(b["deform"]["rate"]))
                if rc != 0:
                    self.close()
                    check(rc, "lbm3_set_deformation")

    def _handle(self):
        if self._h is None:
            raise RuntimeError("domain destroyed")
        return self._h

    def step(self, n: int):
        check(load().lbm3_step(self._handle(), int(n)), "lbm3_step")

    def run(self, n: int, chunk: int = 4096):
        """Advance n steps, draining the force ring between chunks; returns the forces."""
        out = []
        left = int(n)
        while left > 0:
            k = min(chunk, left)
            self.step(k)
            out.append(self.forces())
            left -= k
        if not out:
            return np.zeros((0, self.nbodies, 3))
        return np.concatenate(out, axis=0)

    def forces(self, max_entries: int | None = None) -> np.ndarray:
        cap = self._params.force_capacity if max_entries is None else int(max_entries)
        buf = np.zeros((cap, max(self.nbodies, 1), 3))
        w = C.c_int64()
        check(load().lbm3_forces(self._handle(), buf.ctypes.data_as(C.POINTER(C.c_double)), cap,
                                 C.byref(w)), "lbm3_forces")
        return buf[: w.value, : self.nbodies].copy()

    def moments(self):
        out = [np.zeros((self.nz, self.ny, self.nx)) for _ in range(4)]
        check(load().lbm3_moments(self._handle(), *(o.ctypes.data_as(C.c_void_p) for o in out)),
              "lbm3_moments")
        return tuple(out)

    def get_populations(self) -> np.ndarray:
        out = np.zeros((self.q, self.nz, self.ny, self.nx), dtype=STORAGE_DTYPE[self.storage])
        check(load().lbm3_get_populations(self._handle(), out.ctypes.data_as(C.c_void_p),
                                          out.nbytes), "lbm3_get_populations")
        return out

    def set_populations(self, arr: np.ndarray):
        a = np.ascontiguousarray(arr, dtype=STORAGE_DTYPE[self.storage])
        if a.shape != (self.q, self.nz, self.ny, self.nx):
            raise ValueError(f"populations must have shape ({self.q}, {self.nz}, {self.ny}, {self.nx})")
        check(load().lbm3_set_populations(self._handle(), a.ctypes.data_as(C.c_void_p), a.nbytes),
              "lbm3_set_populations")

    def steps_done(self) -> int:
        v = C.c_int64()
        check(load().lbm3_steps_done(self._handle(), C.byref(v)), "lbm3_steps_done")
        return v.value

    def set_steps_done(self, steps: int):
        """Restore the step index with saved populations (it keys the 16-bit rounding)."""
        check(load().lbm3_set_steps_done(self._handle(), int(steps)), "lbm3_set_steps_done")

    def body_state(self) -> np.ndarray:
        """Body table of the current step, [nbodies, 9]: centre, velocity, angular velocity."""
        out = np.zeros((max(self.nbodies, 1), 9))
        check(load().lbm3_body_state(self._handle(), out.ctypes.data_as(C.POINTER(C.c_double))),
              "lbm3_body_state")
        return out[: self.nbodies]

    def coupled_state(self) -> np.ndarray:
        """Checkpoint of the coupled bodies, [nbodies, 9]: x, v and the previous force."""
        out = np.zeros((max(self.nbodies, 1), 9))
        check(load().lbm3_coupled_state(self._handle(), out.ctypes.data_as(C.POINTER(C.c_double))),
              "lbm3_coupled_state")
        return out[: self.nbodies]

    def restore_coupled(self, steps: int, state: np.ndarray):
        """Resume at step index `steps` with a coupled_state() taken there (populations set
        separately)."""
        a = np.ascontiguousarray(state, dtype=np.float64)
        if a.shape != (self.nbodies, 9):
            raise ValueError(f"state must have shape ({self.nbodies}, 9)")
        check(load().lbm3_restore_coupled(self._handle(), int(steps), a.ctypes.data_as(C.POINTER(C.c_double))),
              "lbm3_restore_coupled")

    def mask(self) -> np.ndarray:
        out = np.zeros((self.nz, self.ny, self.nx), dtype=np.uint8)
        check(load().lbm3_get_mask(self._handle(), out.ctypes.data_as(C.c_void_p)), "lbm3_get_mask")
        return out

    def profile(self, steps: int):
        """Advance `steps` steps, timing each launch; returns (sweep us, force us) per step."""
        a, b = C.c_double(), C.c_double()
        check(load().lbm3_profile(self._handle(), int(steps), C.byref(a), C.byref(b)),
              "lbm3_profile")
        return a.value, b.value

    def set_tile(self, pipeline: int):
        """The sweep's register budget: 0, or 3 / 4 (20 / 24 resident warps per SM, 16-bit
        storage only). Results do not depend on it."""
        check(load().lbm3_set_tile(self._handle(), int(pipeline)), "lbm3_set_tile")

    def get_tile(self) -> int:
        p = C.c_int32()
        check(load().lbm3_get_tile(self._handle(), C.byref(p)), "lbm3_get_tile")
        return p.value

    def autotune(self, reps: int = 10) -> float:
        """Time each register budget on this domain (state untouched), keep the fastest;
        returns its time per sweep launch in microseconds."""
        us = C.c_double()
        check(load().lbm3_autotune(self._handle(), int(reps), C.byref(us)), "lbm3_autotune")
        return us.value

    def close(self):
        if self._h is not None:
            load().lbm3_domain_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _BatchDomain3(Domain3):
    """A resident domain of a Batch3, for its populations, moments, mask and step index.
    The batch owns it: it is not stepped or destroyed through this view."""

    def __init__(self, batch, slot, spec, storage, force_capacity):
        self.spec, self.storage = spec, storage
        self.nx, self.ny, self.nz = spec["nx"], spec["ny"], spec["nz"]
        self.q = 15 if spec.get("lattice", 19) == 15 else 19
        self.nbodies = len(spec["bodies"])
        self._params = _native.params3_from_spec(spec, storage, 1, force_capacity)
        h = C.c_void_p()
        check(load().lbm3_batch_domain(batch._h, int(slot), C.byref(h)), "lbm3_batch_domain")
        self._h = h

    def step(self, n: int):
        raise RuntimeError("a batch's domain is stepped by Batch3.run")

    def set_steps_done(self, steps: int):
        raise RuntimeError("a batch's domain keeps the batch's step index")

    def close(self):
        self._h = None  # owned by the batch


class Batch3:
    """Many fixed-geometry 3D domains of one storage and lattice advanced together: one
    persistent sweep launch per step over every resident domain (lbm3_batch_* calls)."""

    def __init__(self, storage="f16s", lattice=19, max_domains=16, hbm_budget=0, stream=None,
                 allocator="torch"):
        import torch
        self.storage, self.lattice = storage, int(lattice)
        self._alloc = _allocator(allocator)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        check(load().lbm3_batch_create(int(max_domains), int(hbm_budget), STORAGE[storage], self.lattice,
                                       C.c_void_p(self._stream.cuda_stream),
                                       self._alloc.c_alloc if self._alloc else _native.ALLOC_FN(),
                                       self._alloc.c_free if self._alloc else _native.FREE_FN(),
                                       None, C.byref(h)), "lbm3_batch_create")
        self._h = h
        self._meta = {}  # slot -> (spec, force_capacity)

    def admit(self, spec, nsteps=None, force_every=1, force_capacity=8192) -> int:
        """Admit a fixed-geometry domain; returns its slot. Raises LbmError(LBM_EBUSY) when
        the slots or the memory budget are used up."""
        sp = dict(spec, lattice=spec.get("lattice", self.lattice))
        params = _native.params3_from_spec(sp, self.storage, force_every, force_capacity)
        bodies, nb = _native.bodies3_from_spec(sp)
        shapes, ns = _native.shapes3_from_spec(sp)
        slot = C.c_int32()
        n = sp["steps"] if nsteps is None else int(nsteps)
        check(load().lbm3_batch_admit(self._h, C.byref(params), shapes, ns, bodies, nb, n, C.byref(slot)),
              "lbm3_batch_admit")
        self._meta[slot.value] = (sp, force_capacity)
        return slot.value

    def run(self, max_steps: int) -> int:
        """Enqueue up to max_steps steps of every domain with steps left; returns the steps
        enqueued (0: every domain reached its target)."""
        n = C.c_int64()
        check(load().lbm3_batch_run(self._h, int(max_steps), C.byref(n)), "lbm3_batch_run")
        return n.value

    def poll(self, slot: int):
        """(forces [entries, nbodies, 3] since the last poll, done)."""
        sp, cap = self._meta[slot]
        nb = len(sp["bodies"])
        buf = np.zeros((cap, max(nb, 1), 3))
        w, d = C.c_int64(), C.c_int32()
        check(load().lbm3_batch_poll(self._h, int(slot), buf.ctypes.data_as(C.POINTER(C.c_double)), cap,
                                     C.byref(w), C.byref(d)), "lbm3_batch_poll")
        return buf[: w.value, :nb].copy(), bool(d.value)

    def domain(self, slot: int) -> Domain3:
        """The slot's domain (populations, moments, mask, steps_done)."""
        sp, cap = self._meta[slot]
        return _BatchDomain3(self, slot, sp, self.storage, cap)

    def evict(self, slot: int):
        check(load().lbm3_batch_evict(self._h, int(slot)), "lbm3_batch_evict")
        self._meta.pop(slot, None)

    def set_tile(self, pipeline: int):
        check(load().lbm3_batch_set_tile(self._h, int(pipeline)), "lbm3_batch_set_tile")

    def info(self):
        r, c, k, b, p = C.c_int32(), C.c_int64(), C.c_int64(), C.c_size_t(), C.c_int32()
        check(load().lbm3_batch_info(self._h, C.byref(r), C.byref(c), C.byref(k), C.byref(b), C.byref(p)),
              "lbm3_batch_info")
        return {"resident": r.value, "cells": c.value, "kernel_launches": k.value,
                "bytes_in_use": b.value, "pipeline": p.value}

    def close(self):
        if self._h is not None:
            load().lbm3_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many uneven domains of one storage type advanced together (lbm_batch_* calls)."""

    def __init__(self, storage="f16s", max_domains=64, hbm_budget=0, graph_steps=32,
                 stream=None, allocator="torch"):
        import torch
        L = load()
        self.storage = storage
        self._alloc = _allocator(allocator)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        check(L.lbm_batch_create(max_domains, int(hbm_budget), STORAGE[storage], graph_steps,
                                 C.c_void_p(self._stream.cuda_stream),
                                 self._alloc.c_alloc if self._alloc else _native.ALLOC_FN(),
                                 self._alloc.c_free if self._alloc else _native.FREE_FN(),
                                 None, C.byref(h)), "lbm_batch_create")
        self._h = h
        self._meta = {}
        self._deform = set()  # slots with pulsating bodies (another sweep variant)

    def admit(self, spec, nsteps=None, force_every=1, force_capacity=8192, mask=None) -> int:
        """Admit a domain; returns its slot. Raises LbmError(LBM_EBUSY) when full."""
        p = _native.params_from_spec(spec, self.storage, force_every, force_capacity)
        bodies, nb = _native.bodies_from_spec(spec)
        geom, shapes = _native.geometry_from_spec(spec)
        m, mp = _mask_arg(mask)
        slot = C.c_int32()
        n = spec["steps"] if nsteps is None else int(nsteps)
        check(load().lbm_batch_admit(self._h, C.byref(p), mp, C.byref(geom), bodies, nb, n,
                                     C.byref(slot)), "lbm_batch_admit")
        self._meta[slot.value] = (spec["nx"], spec["ny"], len(spec["bodies"]), force_capacity)
        for k, b in enumerate(spec["bodies"]):
            if b.get("dynamics"):
                dyn = _native.dynamics_from(b["dynamics"])
                rc = load().lbm_batch_set_dynamics(self._h, slot.value, k + 1, C.byref(dyn))
                if rc != _native.LBM_OK:
                    err = LbmError(rc, "lbm_batch_set_dynamics", load().lbm_last_error().decode())
                    self.evict(slot.value)
                    raise err
            if b.get("deform"):  # a pulsating body
                self._deform.add(slot.value)
                rc = load().lbm_batch_set_deformation(self._h, slot.value, k + 1,
                                                      float(b["deform"]["amplitude"]),
                                                      float(b["deform"]["rate"]))
                if rc != _native.LBM_OK:
                    err = LbmError(rc, "lbm_batch_set_deformation", load().lbm_last_error().decode())
                    self.evict(slot.value)
                    raise err
        return slot.value

    def admit_many(self, specs, nsteps=None, force_every=1, force_capacity=8192) -> list:
        """Admit many domains; returns their slots in order (`nsteps`: one count for all,
        a list of per-domain counts, or None for each spec's own). Fixed-geometry domains are
        admitted together by one lbm_batch_admit_many call (one batched rasterise, solid
        list and initial-state pass, two synchronisations); moving or coupled ones one by
        one. Raises LbmError (nothing of the batched group admitted) on failure."""
        specs = list(specs)
        plain = [k for k, sp in enumerate(specs)
                 if not sp.get("moving") and not any(b.get("dynamics") or b.get("deform")
                                                     for b in sp["bodies"])]
        out = [None] * len(specs)
        if plain:
            n = len(plain)
            group = [specs[k] for k in plain]
            steps = [int(sp["steps"] if nsteps is None else
                         (nsteps[k] if isinstance(nsteps, (list, tuple)) else nsteps))
                     for k, sp in zip(plain, group)]
            many = _native.ManyDomains(group, self.storage, force_every, force_capacity, steps)
            S = (C.c_int32 * n)()
            check(load().lbm_batch_admit_many(self._h, n, *many.args(), S), "lbm_batch_admit_many")
            for q, k in enumerate(plain):
                sp = specs[k]
                self._meta[S[q]] = (sp["nx"], sp["ny"], len(sp["bodies"]), force_capacity)
                out[k] = S[q]
        for k, sp in enumerate(specs):
            if out[k] is None:
                n_k = nsteps[k] if isinstance(nsteps, (list, tuple)) else nsteps
                out[k] = self.admit(sp, nsteps=n_k, force_every=force_every, force_capacity=force_capacity)
        return out

    def body_state(self, slot: int) -> np.ndarray:
        """Body table of the slot's current step: [nbodies, 5] (cx, cy, vx, vy, omega)."""
        nb = self._meta[slot][2]
        out = np.zeros((max(nb, 1), 5))
        check(load().lbm_batch_body_state(self._h, int(slot), out.ctypes.data_as(C.POINTER(C.c_double))),
              "lbm_batch_body_state")
        return out[:nb]

    def try_admit(self, spec, **kw):
        try:
            return self.admit(spec, **kw)
        except LbmError as e:
            if e.status == LBM_EBUSY:
                return None
            raise

    def run(self, max_steps: int) -> int:
        n = C.c_int64()
        check(load().lbm_batch_run(self._h, int(max_steps), C.byref(n)), "lbm_batch_run")
        return n.value

    def poll(self, slot: int, raise_unstable=True):
        """Drain a slot's forces: returns (forces [n, nbodies, 2], done)."""
        nx, ny, nb, cap = self._meta[slot]
        buf = np.zeros((cap, max(nb, 1), 2))
        w, d = C.c_int64(), C.c_int32()
        st = load().lbm_batch_poll(self._h, slot, buf.ctypes.data_as(C.POINTER(C.c_double)),
                                   cap, C.byref(w), C.byref(d))
        if st != 0 and (raise_unstable or st != LBM_EUNSTABLE):
            check(st, "lbm_batch_poll")
        return buf[: w.value, :nb].copy(), bool(d.value)

    def poll_many(self, slots, raise_unstable=True):
        """poll() for many slots with one synchronisation; a list of (forces, done)."""
        out = []
        for k, (f, done, st) in zip(slots, self.poll_many_status(slots)):
            if st != 0 and (raise_unstable or st != LBM_EUNSTABLE):
                raise LbmError(st, "lbm_batch_poll_many", f"slot {k}")
            out.append((f, done))
        return out

    def poll_many_status(self, slots):
        """poll_many without raising: a list of (forces, done, status) with each slot's own
        status (0 ok, LBM_EUNSTABLE, LBM_ETIMEOUT)."""
        slots = list(slots)
        n = len(slots)
        if n == 0:
            return []
        meta = [self._meta[k] for k in slots]
        # one host buffer for every slot's entries: slot q's [cap][max(nb, 1)][2] at off[q]
        per = np.array([2 * max(m[2], 1) for m in meta], dtype=np.int64)
        cap = np.array([m[3] for m in meta], dtype=np.int64)
        off = np.cumsum(per * cap) - per * cap
        buf = np.empty(int((per * cap).sum()))
        ptrs = (buf.ctypes.data + 8 * off).astype(np.uintp)
        S = np.array(slots, dtype=np.int32)
        W, D, ST = np.zeros(n, np.int64), np.zeros(n, np.int32), np.zeros(n, np.int32)
        _i32, _i64 = C.POINTER(C.c_int32), C.POINTER(C.c_int64)
        check(load().lbm_batch_poll_many(self._h, n, S.ctypes.data_as(_i32),
                                         ptrs.ctypes.data_as(C.POINTER(_native._DP)),
                                         cap.ctypes.data_as(_i64), W.ctypes.data_as(_i64),
                                         D.ctypes.data_as(_i32), ST.ctypes.data_as(_i32)),
              "lbm_batch_poll_many")
        out = []
        for q, m in enumerate(meta):
            w, o, nb = int(W[q]), int(off[q]), max(m[2], 1)
            f = buf[o: o + w * 2 * nb].reshape(w, nb, 2)[:, : m[2]].copy()
            out.append((f, bool(D[q]), int(ST[q])))
        return out

    def moments(self, slot: int):
        nx, ny, nb, cap = self._meta[slot]
        rho, ux, uy = (np.zeros((ny, nx)) for _ in range(3))
        check(load().lbm_batch_moments(self._h, slot, rho.ctypes.data_as(C.c_void_p),
                                       ux.ctypes.data_as(C.c_void_p),
                                       uy.ctypes.data_as(C.c_void_p)), "lbm_batch_moments")
        return rho, ux, uy

    def get_populations(self, slot: int) -> np.ndarray:
        nx, ny, nb, cap = self._meta[slot]
        out = np.zeros((9, ny, nx), dtype=STORAGE_DTYPE[self.storage])
        check(load().lbm_batch_get_populations(self._h, slot, out.ctypes.data_as(C.c_void_p),
                                               out.nbytes), "lbm_batch_get_populations")
        return out

    def set_populations(self, slot: int, arr):
        a = np.ascontiguousarray(arr, dtype=STORAGE_DTYPE[self.storage])
        check(load().lbm_batch_set_populations(self._h, slot, a.ctypes.data_as(C.c_void_p),
                                               a.nbytes), "lbm_batch_set_populations")

    def steps_done(self, slot: int) -> int:
        v = C.c_int64()
        check(load().lbm_batch_steps_done(self._h, slot, C.byref(v)), "lbm_batch_steps_done")
        return v.value

    def set_steps_done(self, slot: int, steps: int):
        check(load().lbm_batch_set_steps_done(self._h, slot, int(steps)), "lbm_batch_set_steps_done")

    def link_x(self, west_slot: int, east_slot: int):
        """Link two resident slabs of one grid across their x edges (see slabs.py)."""
        check(load().lbm_batch_link_x(self._h, int(west_slot), int(east_slot)), "lbm_batch_link_x")

    def mask(self, slot: int) -> np.ndarray:
        nx, ny, nb, cap = self._meta[slot]
        out = np.zeros((ny, nx), dtype=np.uint8)
        check(load().lbm_batch_get_mask(self._h, slot, out.ctypes.data_as(C.c_void_p)),
              "lbm_batch_get_mask")
        return out

    def evict(self, slot: int):
        check(load().lbm_batch_evict(self._h, slot), "lbm_batch_evict")
        self._meta.pop(slot, None)
        self._deform.discard(slot)

    def set_halo(self, slot: int, side: int, recv=None, send=None):
        """Make x edge `side` (0 west, 1 east) of a slot a halo edge fed from `recv` and
        packed into `send`: device tensors of [9, ny] storage elements that the caller
        keeps alive (None, None restores the admitted edge). See slabs.HaloGrid."""
        rp = C.c_void_p(recv.data_ptr()) if recv is not None else None
        sp = C.c_void_p(send.data_ptr()) if send is not None else None
        check(load().lbm_batch_set_halo(self._h, int(slot), int(side), rp, sp), "lbm_batch_set_halo")

    def pack_halos(self):
        """Enqueue the packing of every halo edge's send buffer from the current state."""
        check(load().lbm_batch_pack_halos(self._h), "lbm_batch_pack_halos")

    def capture(self):
        """Build the work lists and capture the step graph now (no steps run), so that the
        next run replays it without capturing."""
        check(load().lbm_batch_capture(self._h), "lbm_batch_capture")

    INJECT = {"none": 0, "unstable": 1, "wait_timeout": 2}

    def inject(self, kind: str, slot: int = -1):
        """Host-side failure injection for tests of the error paths (no GPU fault):
        "unstable" marks a slot as diverged, "wait_timeout" makes later launches of the
        shared-memory-staged sweep report a timed-out wait, "none" clears the latter."""
        check(load().lbm_batch_inject(self._h, int(slot), self.INJECT[kind]), "lbm_batch_inject")

    def profile(self, steps: int):
        """Run `steps` real steps one kernel at a time; returns (sweep_us, force_us,
        steps_run), the mean event-timed duration of each launch."""
        a, b, n = C.c_double(), C.c_double(), C.c_int64()
        check(load().lbm_batch_profile(self._h, int(steps), C.byref(a), C.byref(b), C.byref(n)),
              "lbm_batch_profile")
        return a.value, b.value, n.value

    def workload_key(self) -> str:
        """The class of the resident workload that tuned tile shapes are cached under
        (device, storage, kernel variant, cells and width classes: `tuning.workload_key`)."""
        import torch
        from .tuning import workload_key
        prop = torch.cuda.get_device_properties(self._stream.device)
        return workload_key(prop.name, prop.multi_processor_count, self.storage,
                            bool(self._deform), [m[:2] for m in self._meta.values()])

    def autotune(self, reps: int = 10, cache=None) -> float:
        """Time the tile shapes on the resident domains and keep the fastest; returns
        its time per sweep launch in microseconds. With a `tuning.TuneCache`, a shape
        already tuned for this workload class is set without timing (and the time it
        was tuned at is returned), and a newly tuned one is stored."""
        def tune():
            us = C.c_double()
            check(load().lbm_batch_autotune(self._h, reps, C.byref(us)), "lbm_batch_autotune")
            return us.value
        if cache is None:
            return tune()
        from .tuning import cached_autotune
        return cached_autotune(cache, self.workload_key(), tune, self.set_tile, self.get_tile)

    def set_grouped_admission(self, on: bool):
        """admit_many with two allocations for all of its domains (True, the default; a
        group's memory returns with its last domain) or two per domain (False)."""
        check(load().lbm_batch_set_grouped_admission(self._h, int(bool(on))),
              "lbm_batch_set_grouped_admission")

    def set_tile(self, vec: int, warps: int, rows: int, pipeline: int = 0):
        check(load().lbm_batch_set_tile(self._h, vec, warps, rows, pipeline), "lbm_batch_set_tile")

    def get_tile(self):
        """(cells per thread, warps per block, rows per warp, pipeline)."""
        v, w, r, p = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        check(load().lbm_batch_get_tile(self._h, C.byref(v), C.byref(w), C.byref(r), C.byref(p)),
              "lbm_batch_get_tile")
        return v.value, w.value, r.value, p.value

    def info(self):
        r, c, k, b = C.c_int32(), C.c_int64(), C.c_int64(), C.c_size_t()
        check(load().lbm_batch_info(self._h, C.byref(r), C.byref(c), C.byref(k), C.byref(b)),
              "lbm_batch_info")
        return {"resident": r.value, "cells": c.value, "kernel_launches": k.value,
                "bytes_in_use": b.value}

    def close(self):
        if self._h is not None:
            load().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
