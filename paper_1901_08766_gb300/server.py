"""Continuous-batching request server for TRT-LBM-VP simulations.

Requests (a problem description with geometry, Re, grid size and step count) arrive at
any time. The server keeps their populations resident in one batch on the GPU
(lbm_batch_* calls) and advances all resident domains together in chunks of steps, one
persistent sweep launch per step. Between chunks it streams each request's new
force-series slice back, retires finished requests (evicting their device memory) and
admits waiting requests in arrival order as slots and memory budget free up, so that
requests arriving while others run join the running batch.

Each result is the same whether the request ran alone or in a mix: the per-node
arithmetic and the force-sum order do not depend on the batch composition.

    srv = Server(storage="f16s", hbm_budget=40 << 30)
    fut = srv.submit(spec)                  # spec as produced by the synth module
    srv.run_until_idle()                    # or srv.start() for a background loop
    res = fut.result()                      # Result: forces, latency, status
"""
from __future__ import annotations

import collections
import heapq
import itertools
import os
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np
import torch


def _nvtx(name):
    """A named NVTX range (seen by profilers that record NVTX; inert otherwise). The
    library's own entry points (lbm_batch_run, lbm_batch_admit_many, lbm_batch_poll_many,
    ...) push ranges of their own inside these."""
    return torch.cuda.nvtx.range(name)

from . import diagnostics
from .tuning import TuneCache


@dataclass
class Result:
    request_id: int
    name: str
    status: str                      # "ok", "unstable", "failed", "cancelled" or "rejected"
    forces: np.ndarray               # [steps, nbodies, 2]: force on each body per step
    steps: int
    cells: int
    arrival: float
    admitted: float | None
    done: float
    detail: str = ""
    coefficients: dict = field(default_factory=dict)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Req:
    rid: int
    spec: dict
    nsteps: int
    arrival: float
    future: Future
    on_forces: object = None
    slot: int | None = None
    admitted: float | None = None
    chunks: list = field(default_factory=list)
    cancelled: bool = False


class Server:
    """Admission by memory budget, FIFO order, chunked stepping of all resident domains."""

    def __init__(self, storage="f16s", max_domains=256, hbm_budget=0, chunk_steps=256,
                 graph_steps=32, force_every=1, backend=None, clock=time.perf_counter,
                 autotune=True, tune_cache=None, max_resident=None):
        if backend is None:
            from . import Batch
            backend = Batch(storage, max_domains=max_domains, hbm_budget=hbm_budget,
                            graph_steps=graph_steps)
        self.backend = backend
        self.max_domains = max_domains
        self.storage = storage
        self.hbm_budget = hbm_budget
        if hbm_budget > 0 and hasattr(backend, "set_grouped_admission"):
            # requests admitted together end at different times: under a memory budget
            # each one's memory must return at its own eviction
            backend.set_grouped_admission(False)
        self.chunk_steps = int(chunk_steps)
        self.force_every = int(force_every)
        self.force_capacity = self.chunk_steps + 8  # force entries of one chunk per request
        self.clock = clock
        # the tile shape is retuned whenever the resident workload changes class
        # (tuning.workload_key); shapes tuned once per class come from the cache, which
        # persists in a JSON file when `tune_cache` is a path
        self.autotune = autotune
        if isinstance(tune_cache, (str, bytes, os.PathLike)):
            tune_cache = TuneCache(os.fsdecode(tune_cache))
        self.tune_cache = tune_cache if tune_cache is not None else TuneCache()
        self._tuned_key = None
        # at most this many requests share the GPU at once (None: as many as memory holds);
        # fewer residents finish each sooner, the others wait in the FIFO queue
        self.max_resident = max_resident
        self._ids = itertools.count()
        self._lock = threading.Lock()
        self._pending = []                      # heap of (arrival, rid, req) not yet arrived
        self._queue = collections.deque()       # arrived, waiting for admission (FIFO)
        self._resident = {}                     # slot -> req
        self._cancel = set()
        self._thread = None
        self._stop = threading.Event()
        self.completed = []
        self.cell_updates = 0
        self.t_start = None
        self.chunks_run = 0
        self.max_queue = 0
        # host time per part of the loop (seconds): admission, enqueueing the chunk, draining
        # (which waits for the chunk on the GPU)
        self.host_s = {"admit": 0.0, "tune": 0.0, "run": 0.0, "drain": 0.0}
        self.retunes = 0

    # ---- client side ---------------------------------------------------------------
    def submit(self, spec, nsteps=None, arrival=None, on_forces=None) -> Future:
        """Queue a request; `arrival` (server clock) defaults to now. Returns a Future
        resolving to a Result. `on_forces(request_id, chunk)` receives each new slice."""
        fut = Future()
        n = int(spec["steps"] if nsteps is None else nsteps)
        t = self.clock() if arrival is None else float(arrival)
        req = _Req(next(self._ids), spec, n, t, fut, on_forces)
        fut.request_id = req.rid
        with self._lock:
            heapq.heappush(self._pending, (t, req.rid, req))
        return fut

    def cancel(self, request_id: int):
        with self._lock:
            self._cancel.add(request_id)

    # ---- server loop ---------------------------------------------------------------
    def _finish(self, req, status, detail=""):
        forces = np.concatenate(req.chunks) if req.chunks else np.zeros((0, len(req.spec["bodies"]), 2))
        res = Result(req.rid, req.spec.get("name", ""), status, forces, len(forces),
                     req.spec["nx"] * req.spec["ny"], req.arrival, req.admitted, self.clock(), detail)
        if status == "ok" and len(forces) and req.spec["bodies"]:
            b = req.spec["bodies"][0]
            res.coefficients = diagnostics.summary(forces[:, 0], req.spec["U"], b["ref_length"],
                                                   req.spec["rho0"])
        if status == "ok":
            self.cell_updates += res.cells * res.steps
        self.completed.append(res)
        req.future.set_result(res)

    def _arrivals(self, now):
        with self._lock:
            while self._pending and self._pending[0][0] <= now:
                self._queue.append(heapq.heappop(self._pending)[2])
            cancel, self._cancel = self._cancel, set()
        if cancel:
            for q in [q for q in self._queue if q.rid in cancel]:
                self._queue.remove(q)
                self._finish(q, "cancelled")
            for slot, q in list(self._resident.items()):
                if q.rid in cancel:
                    self.backend.evict(slot)
                    del self._resident[slot]
                    self._finish(q, "cancelled")

    def _admit_group(self):
        """Admit the longest FIFO prefix of the queue that fits the free slots and the
        memory budget with one batched admission (backends that offer it). False when
        nothing was admitted that way (the one-by-one path then decides)."""
        from . import domain_bytes
        from ._native import LbmError
        if not hasattr(self.backend, "admit_many") or len(self._queue) < 2:
            return False
        info = self.backend.info()
        room = self.max_domains - info["resident"]
        if self.max_resident is not None:
            room = min(room, self.max_resident - len(self._resident))
        left = self.hbm_budget - info["bytes_in_use"] if self.hbm_budget > 0 else None
        group = []
        for req in self._queue:
            if len(group) >= room:
                break
            if req.spec.get("moving") or any(b.get("dynamics") or b.get("deform") for b in req.spec["bodies"]):
                break
            need = domain_bytes(req.spec, self.storage, self.force_every, self.force_capacity)
            if left is not None:
                if need > left:
                    break
                left -= need
            group.append(req)
        if len(group) < 2:
            return False
        try:
            slots = self.backend.admit_many([r.spec for r in group], nsteps=[r.nsteps for r in group],
                                            force_every=self.force_every,
                                            force_capacity=self.force_capacity)
        except LbmError:
            return False  # nothing admitted: the one-by-one path finds the culprit
        now = self.clock()
        for req, slot in zip(group, slots):
            self._queue.popleft()
            req.slot = slot
            req.admitted = now
            self._resident[slot] = req
        return True

    def _admit(self):
        from ._native import LbmError
        self._admit_group()
        while self._queue:
            if self.max_resident is not None and len(self._resident) >= self.max_resident:
                break
            req = self._queue[0]
            try:
                slot = self.backend.try_admit(req.spec, nsteps=req.nsteps, force_every=self.force_every,
                                              force_capacity=self.force_capacity)
            except LbmError as e:  # invalid request
                self._queue.popleft()
                self._finish(req, "rejected", str(e))
                continue
            if slot is None:
                if not self._resident:  # can never fit: nothing left to free
                    self._queue.popleft()
                    self._finish(req, "rejected", "larger than the memory budget")
                    continue
                break  # FIFO: wait for memory to free up
            self._queue.popleft()
            req.slot = slot
            req.admitted = self.clock()
            self._resident[slot] = req
        self.max_queue = max(self.max_queue, len(self._queue))

    def _drain(self):
        from ._native import LBM_EUNSTABLE, LbmError
        if hasattr(self.backend, "poll_many_status"):
            # every resident's new force slice with one synchronisation
            items = list(self._resident.items())
            for (slot, req), (f, done, st) in zip(items, self.backend.poll_many_status([s for s, _ in items])):
                if len(f):
                    req.chunks.append(f)
                    if req.on_forces is not None:
                        req.on_forces(req.rid, f)
                if st != 0:
                    self.backend.evict(slot)
                    del self._resident[slot]
                    self._finish(req, "unstable" if st == LBM_EUNSTABLE else "failed",
                                 f"device status {st}")
                elif done:
                    self.backend.evict(slot)
                    del self._resident[slot]
                    self._finish(req, "ok")
            return
        for slot, req in list(self._resident.items()):
            try:
                f, done = self.backend.poll(slot)
            except LbmError as e:
                if e.status != LBM_EUNSTABLE:
                    raise
                self.backend.evict(slot)
                del self._resident[slot]
                self._finish(req, "unstable", str(e))
                continue
            if len(f):
                req.chunks.append(f)
                if req.on_forces is not None:
                    req.on_forces(req.rid, f)
            if done:
                self.backend.evict(slot)
                del self._resident[slot]
                self._finish(req, "ok")

    def pump(self) -> bool:
        """One scheduling round. Returns True while requests remain anywhere."""
        now = self.clock()
        if self.t_start is None:
            self.t_start = now
        self._arrivals(now)
        t0 = time.perf_counter()
        with _nvtx("server.admit"):
            self._admit()
        t1 = time.perf_counter()
        self.host_s["admit"] += t1 - t0
        if self._resident:
            if self.autotune:
                key = self.backend.workload_key()
                if key != self._tuned_key:
                    with _nvtx("server.autotune"):
                        self.backend.autotune(reps=3, cache=self.tune_cache)
                    self._tuned_key = key
                    self.retunes += 1
                t_tune = time.perf_counter()
                self.host_s["tune"] += t_tune - t1
                t1 = t_tune
            with _nvtx(f"server.chunk {self.chunks_run}"):
                ran = self.backend.run(self.chunk_steps)
            t2 = time.perf_counter()
            self.chunks_run += 1
            with _nvtx("server.drain"):
                self._drain()
                if ran == 0:
                    self._drain()
            self.host_s["run"] += t2 - t1
            self.host_s["drain"] += time.perf_counter() - t2
        with self._lock:
            pending = bool(self._pending)
            next_arrival = self._pending[0][0] if pending else None
        if not self._resident and not self._queue and pending:
            delay = next_arrival - self.clock()
            if delay > 0:
                time.sleep(min(delay, 0.05))
        return bool(self._resident or self._queue or pending)

    def run_until_idle(self, timeout=None):
        t0 = self.clock()
        while self.pump():
            if timeout is not None and self.clock() - t0 > timeout:
                raise TimeoutError("server did not drain within the timeout")

    def start(self):
        """Run the loop in a background thread until stop()."""
        def loop():
            while not self._stop.is_set():
                if not self.pump():
                    time.sleep(0.001)
        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()

    def stop(self):
        self._stop.set()
        if self._thread is not None:
            self._thread.join()

    # ---- reporting -----------------------------------------------------------------
    def stats(self) -> dict:
        ok = [r for r in self.completed if r.status == "ok"]
        lat = np.array([r.latency for r in ok]) if ok else np.zeros(0)
        wall = (max(r.done for r in ok) - self.t_start) if ok else 0.0
        return {"completed": len(ok), "failed": len(self.completed) - len(ok),
                "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
                "glups": self.cell_updates / wall / 1e9 if wall > 0 else None,
                "wall_s": wall, "chunks": self.chunks_run, "max_queue": self.max_queue,
                "host_s": dict(self.host_s), "retunes": self.retunes,
                "tune_cache": {"hits": self.tune_cache.hits, "misses": self.tune_cache.misses}}
