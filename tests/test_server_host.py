"""Host logic of the request server, on a fake batch backend (no GPU): FIFO admission by
memory budget, continuous batching, force streaming, cancellation, rejection and
divergence handling, latency statistics."""
import numpy as np
import pytest

import synth
from paper_1901_08766_gb300 import server as srvmod
from paper_1901_08766_gb300 import tuning
from paper_1901_08766_gb300._native import LBM_EBUSY, LBM_EINVAL, LBM_EUNSTABLE, LbmError


@pytest.fixture(autouse=True)
def _library(built_library):
    # the server sizes requests under a memory budget with lbm_domain_bytes
    return built_library


class FakeBatch:
    """Mimics lbm.Batch: a slot runs until its own step target; each step records a force
    that depends only on (request name, step), like the real library's results."""

    def __init__(self, budget_cells, max_slots=64, unstable_names=(), clock=None):
        self.budget = budget_cells
        self.max_slots = max_slots
        self.slots = {}
        self.unstable = set(unstable_names)
        self.clock = clock
        self.runs = []

    def try_admit(self, spec, nsteps, force_every=1, force_capacity=0):
        if spec["nx"] < 3:
            raise LbmError(LBM_EINVAL, "lbm_batch_admit", "nx must be >= 3")
        cells = spec["nx"] * spec["ny"]
        used = sum(s["cells"] for s in self.slots.values())
        if used + cells > self.budget or len(self.slots) >= self.max_slots:
            return None
        k = next(i for i in range(self.max_slots) if i not in self.slots)
        self.slots[k] = {"spec": spec, "cells": cells, "target": nsteps, "done": 0, "drained": 0,
                         "cap": force_capacity, "nb": len(spec["bodies"])}
        return k

    def run(self, max_steps):
        rem = [s["target"] - s["done"] for s in self.slots.values() if s["done"] < s["target"]]
        n = min(max_steps, max(rem)) if rem else 0
        for s in self.slots.values():
            adv = min(n, s["target"] - s["done"])
            assert s["done"] + adv - s["drained"] <= s["cap"], "force ring overflow"
            s["done"] += adv
        self.runs.append(n)
        if self.clock is not None:
            self.clock.t += 0.001 * n
        return n

    def poll(self, slot):
        s = self.slots[slot]
        if s["spec"]["name"] in self.unstable and s["done"] > 0:
            raise LbmError(LBM_EUNSTABLE, "lbm_batch_poll", "diverged")
        steps = np.arange(s["drained"], s["done"])
        h = sum(map(ord, s["spec"]["name"]))
        f = np.stack([np.stack([np.sin(h + 0.01 * steps), np.cos(h + 0.02 * steps)], -1)] * s["nb"], 1)
        s["drained"] = s["done"]
        return f, s["done"] >= s["target"]

    def evict(self, slot):
        del self.slots[slot]

    # tile tuning: the fake's "best" tile depends on the resident cells, like a real batch
    tile = (8, 16, 1, 0)
    timed = 0

    def workload_key(self):
        return tuning.workload_key("fake", 2, "f16s", False,
                                   [(s["spec"]["nx"], s["spec"]["ny"]) for s in self.slots.values()])

    def set_tile(self, *t):
        self.tile = tuple(t)

    def get_tile(self):
        return self.tile

    def autotune(self, reps=3, cache=None):
        def tune():
            self.timed += 1
            cells = sum(s["cells"] for s in self.slots.values())
            self.tile = (8, 12 if cells > 4000 else 8, 4, 4)
            return 100.0 + cells
        if cache is None:
            return tune()
        return tuning.cached_autotune(cache, self.workload_key(), tune, self.set_tile, self.get_tile)


class FakeBatchMany(FakeBatch):
    """FakeBatch with the batched calls: all-or-none admission of many requests and one
    poll for many slots that reports each slot's status instead of raising."""

    def info(self):
        return {"resident": len(self.slots), "bytes_in_use": 0}

    def admit_many(self, specs, nsteps, force_every=1, force_capacity=0):
        used = sum(s["cells"] for s in self.slots.values())
        for sp in specs:
            if sp["nx"] < 3:
                raise LbmError(LBM_EINVAL, "lbm_batch_admit_many", "nx must be >= 3")
            used += sp["nx"] * sp["ny"]
        if used > self.budget or len(self.slots) + len(specs) > self.max_slots:
            raise LbmError(LBM_EBUSY, "lbm_batch_admit_many", "does not fit")
        self.groups = getattr(self, "groups", 0) + 1
        return [self.try_admit(sp, n, force_every, force_capacity) for sp, n in zip(specs, nsteps)]

    def poll_many_status(self, slots):
        out = []
        for k in slots:
            try:
                f, done = self.poll(k)
                out.append((f, done, 0))
            except LbmError as e:
                out.append((np.zeros((0, self.slots[k]["nb"], 2)), False, e.status))
        return out


FAKES = [FakeBatch, FakeBatchMany]


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def _spec(name, n=100, steps=50):
    sp = synth.parity_case("channel_97x61")
    return dict(sp, name=name, nx=n, ny=n // 2, steps=steps)


@pytest.mark.parametrize("Fake", FAKES)
def test_fifo_admission_under_budget_and_streaming(Fake):
    clock = Clock()
    fb = Fake(budget_cells=2 * 100 * 50, clock=clock)
    srv = srvmod.Server(backend=fb, chunk_steps=16, clock=clock)
    seen = {}
    futs = [srv.submit(_spec(f"r{i}", steps=40 + 10 * i), arrival=0.0,
                       on_forces=lambda rid, f: seen.setdefault(rid, []).append(len(f)))
            for i in range(4)]
    srv.pump()
    assert len(fb.slots) == 2 and len(srv._queue) == 2  # budget holds two
    srv.run_until_idle()
    res = [f.result() for f in futs]
    assert [r.status for r in res] == ["ok"] * 4
    assert [r.steps for r in res] == [40, 50, 60, 70]
    # FIFO: admission times follow arrival order
    adm = [r.admitted for r in res]
    assert adm == sorted(adm)
    # the streamed slices add up to the whole series
    for r, f in zip(res, futs):
        assert sum(seen[f.request_id]) == r.steps
    st = srv.stats()
    assert st["completed"] == 4 and st["p99_latency_s"] >= st["p50_latency_s"] > 0


@pytest.mark.parametrize("Fake", FAKES)
def test_resident_cap_keeps_fifo_and_limits_sharing(Fake):
    clock = Clock()
    fb = Fake(budget_cells=10 ** 9, clock=clock)
    srv = srvmod.Server(backend=fb, chunk_steps=10, clock=clock, max_resident=2)
    futs = [srv.submit(_spec(f"r{i}", steps=30), arrival=0.0) for i in range(5)]
    peak = 0
    while srv.pump():
        peak = max(peak, len(fb.slots))
    assert peak == 2
    res = [f.result() for f in futs]
    assert all(r.status == "ok" and r.steps == 30 for r in res)
    adm = [r.admitted for r in res]
    assert adm == sorted(adm)
    # pairs finish together: the first two long before the last one
    assert res[1].done < res[4].admitted


@pytest.mark.parametrize("Fake", FAKES)
def test_late_arrival_joins_running_batch(Fake):
    clock = Clock()
    fb = Fake(budget_cells=10 ** 9, clock=clock)
    srv = srvmod.Server(backend=fb, chunk_steps=10, clock=clock)
    a = srv.submit(_spec("long", steps=200), arrival=0.0)
    b = srv.submit(_spec("late", steps=30), arrival=0.05)
    while not b.done():
        srv.pump()
    assert not a.done()  # the late request finished while the long one kept running
    srv.run_until_idle()
    ra, rb = a.result(), b.result()
    assert rb.admitted < ra.done and rb.done < ra.done


@pytest.mark.parametrize("Fake", FAKES)
def test_cancel_reject_and_unstable(Fake):
    clock = Clock()
    fb = Fake(budget_cells=100 * 50, unstable_names={"bad"}, clock=clock)
    srv = srvmod.Server(backend=fb, chunk_steps=8, clock=clock)
    big = srv.submit(_spec("huge", n=400), arrival=0.0)          # can never fit
    bad = srv.submit(_spec("bad", steps=30), arrival=0.0)
    queued = srv.submit(_spec("queued", steps=30), arrival=0.0)  # waits behind "bad"
    inval = srv.submit(dict(_spec("tiny"), nx=2), arrival=0.0)
    srv.pump()
    srv.cancel(queued.request_id)
    srv.run_until_idle()
    assert big.result().status == "rejected"
    assert bad.result().status == "unstable"
    assert queued.result().status == "cancelled"
    assert inval.result().status == "rejected"
    assert not fb.slots  # everything evicted


@pytest.mark.parametrize("Fake", FAKES)
def test_background_thread_serves_submissions(Fake):
    fb = Fake(budget_cells=10 ** 9)
    srv = srvmod.Server(backend=fb, chunk_steps=32)
    srv.start()
    futs = [srv.submit(_spec(f"t{i}", steps=64)) for i in range(5)]
    res = [f.result(timeout=30) for f in futs]
    srv.stop()
    assert all(r.status == "ok" and r.forces.shape == (64, 2, 2) for r in res)


def test_group_admission_is_fifo_and_used():
    clock = Clock()
    fb = FakeBatchMany(budget_cells=10 ** 9, clock=clock)
    srv = srvmod.Server(backend=fb, chunk_steps=16, clock=clock)
    futs = [srv.submit(_spec(f"g{i}", steps=20 + i), arrival=0.0) for i in range(6)]
    srv.run_until_idle()
    assert getattr(fb, "groups", 0) >= 1  # the arrived requests went in as one group
    res = [f.result() for f in futs]
    assert all(r.status == "ok" for r in res) and [r.steps for r in res] == [20 + i for i in range(6)]
    assert [r.admitted for r in res] == sorted(r.admitted for r in res)


class FakeBatchGrouping(FakeBatchMany):
    """FakeBatchMany that records the grouped-admission setting it is given."""

    def set_grouped_admission(self, on):
        self.grouped = bool(on)


@pytest.mark.parametrize("budget,grouped", [(0, None), (1 << 30, False)])
def test_server_under_a_budget_admits_groups_per_domain(budget, grouped):
    # requests admitted together end at different times: under a memory budget the
    # server turns grouped admission off, so each request's memory returns at its own
    # eviction; without a budget the batch keeps its default
    fb = FakeBatchGrouping(budget_cells=10 ** 9, clock=Clock())
    srvmod.Server(backend=fb, hbm_budget=budget, chunk_steps=16, clock=fb.clock)
    assert getattr(fb, "grouped", None) is grouped


def test_server_retunes_per_workload_class_and_persists(tmp_path):
    # autotuning is on by default: the server tunes when the resident workload changes
    # class, takes shapes it has tuned before from the cache, and a second server reading
    # the same JSON file times nothing
    path = tmp_path / "tune.json"
    runs = []
    for _ in range(2):
        clock = Clock()
        fb = FakeBatch(budget_cells=10 ** 9, clock=clock)
        srv = srvmod.Server(backend=fb, chunk_steps=10, clock=clock, tune_cache=str(path))
        futs = [srv.submit(_spec("small", n=40, steps=30), arrival=0.0),
                srv.submit(_spec("big", n=200, steps=60), arrival=0.015),
                srv.submit(_spec("small2", n=40, steps=60), arrival=0.05)]
        srv.run_until_idle()
        assert all(f.result().status == "ok" for f in futs)
        runs.append((fb.timed, srv.retunes, srv.stats()["tune_cache"]))
    (timed1, retunes1, c1), (timed2, retunes2, c2) = runs
    # classes seen: small alone; small + big (big alone and big + small2 are the same
    # class: the small domains hold under a quarter of the cells); small2 alone, the
    # first class again, so from the cache
    assert retunes1 == retunes2 == 3
    assert timed1 == c1["misses"] and c1["hits"] == retunes1 - timed1 and timed1 < retunes1
    assert timed2 == 0 and c2["hits"] == retunes2
    saved = tuning.TuneCache(str(path)).entries
    assert len(saved) == timed1 and all(len(e["tile"]) == 4 for e in saved.values())


def test_server_without_autotune_keeps_the_tile():
    clock = Clock()
    fb = FakeBatch(budget_cells=10 ** 9, clock=clock)
    srv = srvmod.Server(backend=fb, chunk_steps=10, clock=clock, autotune=False)
    srv.submit(_spec("a", steps=20), arrival=0.0)
    srv.run_until_idle()
    assert fb.timed == 0 and srv.retunes == 0 and fb.tile == (8, 16, 1, 0)
