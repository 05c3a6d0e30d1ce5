"""Failure paths of the library, exercised without any GPU fault, trap or hang: the
failures are made on the host.

- An allocator callback that returns NULL at the k-th request, for every k a domain's
  life makes: the call that needed the memory returns LBM_ENOMEM and every block the
  library took is given back (nothing leaks).
- Guard bands: every allocation is padded on both sides with a byte pattern that the
  library must never touch; ragged grid sizes in every storage are created, stepped,
  read and written back, and the bands are checked on every free and at the end (in
  place of a device sanitizer).
- Host-side injection (lbm_batch_inject): a slot marked unstable reports LBM_EUNSTABLE
  while its neighbours carry on; the shared-memory-staged sweep takes its timeout path
  after its row copies completed and the slots report LBM_ETIMEOUT, also through the
  moments export; afterwards the device is still usable.
"""
import numpy as np
import pytest

import codec
import synth

pytestmark = pytest.mark.gpu

LBM_ENOMEM, LBM_EUNSTABLE, LBM_ETIMEOUT = 2, 4, 5


class GuardedAllocator:
    """Device memory from PyTorch with guard bands of a fixed pattern before and after
    each block; optionally refuses (returns NULL) from the `fail_at`-th request on."""

    GUARD = 4096  # bytes on each side (a multiple of 256 keeps the blocks' alignment)
    PATTERN = 0xA5

    def __init__(self, fail_at=None):
        import torch
        from paper_1901_08766_gb300 import _native
        self.torch = torch
        self.fail_at = fail_at
        self.requests = 0
        self.live = {}
        self.violations = []
        self.c_alloc = _native.ALLOC_FN(self._alloc)
        self.c_free = _native.FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        k = self.requests
        self.requests += 1
        if self.fail_at is not None and k >= self.fail_at:
            return None
        t = self.torch.empty(int(nbytes) + 2 * self.GUARD, dtype=self.torch.uint8, device="cuda")
        # only the bands are written here: the block itself belongs to the library's stream
        t[: self.GUARD].fill_(self.PATTERN)
        t[self.GUARD + int(nbytes):].fill_(self.PATTERN)
        self.torch.cuda.synchronize()
        ptr = t.data_ptr() + self.GUARD
        self.live[ptr] = (t, int(nbytes))
        return ptr

    def _check(self, ptr, t, n):
        self.torch.cuda.synchronize()
        head = t[: self.GUARD]
        tail = t[self.GUARD + n:]
        if not bool((head == self.PATTERN).all()) or not bool((tail == self.PATTERN).all()):
            self.violations.append((ptr, n))

    def _free(self, ptr, ctx):
        ent = self.live.pop(ptr, None)
        if ent is None:
            self.violations.append((ptr, "freed twice or never allocated"))
        else:
            self._check(ptr, *ent)

    def check_all(self):
        for ptr, (t, n) in list(self.live.items()):
            self._check(ptr, t, n)


def _small_channel():
    return synth.parity_case("channel_97x61")


def test_allocator_null_gives_enomem_and_leaks_nothing(lbm):
    spec = _small_channel()
    # requests made by a domain's creation, its first steps and one moments export
    probe = GuardedAllocator()
    dom = lbm.Domain(spec, storage="f32", allocator=probe)
    created = probe.requests
    dom.step(2)
    dom.moments()
    total = probe.requests
    dom.close()
    assert not probe.live and not probe.violations
    assert created >= 4 and total > created
    for k in range(total):
        a = GuardedAllocator(fail_at=k)
        with pytest.raises(lbm.LbmError) as ei:
            d = lbm.Domain(spec, storage="f32", allocator=a)
            try:
                d.step(2)
                d.moments()
            finally:
                d.close()
        assert ei.value.status == LBM_ENOMEM, (k, ei.value)
        assert not a.live, f"refusing request {k} leaked {len(a.live)} blocks"
        assert not a.violations


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
def test_guard_bands_untouched_on_ragged_sizes(lbm, storage):
    a = GuardedAllocator()
    sizes = [(3, 3), (5, 4), (64, 3), (65, 7), (130, 5), (257, 9), (513, 4)]
    for nx, ny in sizes:
        for e in (synth._edges(), synth._edges("inlet", "outflow", "free_slip", "free_slip")):
            shapes = [synth._circle(1, nx / 3.0, ny / 2.0, max(1.0, min(nx, ny) / 4.0))]
            bodies = [synth._body(nx / 3.0, ny / 2.0, 2.0, omega=1e-3)]
            spec = synth._spec("edge", nx, ny, 0.05, shapes, bodies, 0, 0.02, e, u_in=(0.02, 0.0))
            d = lbm.Domain(spec, storage=storage, allocator=a)
            d.set_populations(codec.encode(synth.random_populations(nx + ny, nx, ny, 0.05), storage))
            d.step(7)
            d.forces()
            d.moments()
            d.get_populations()
            a.check_all()
            d.close()
    # a batch of all the sizes at once, each tile shape the autotuner may pick
    b = lbm.Batch(storage, max_domains=len(sizes), graph_steps=4, allocator=a)
    slots = []
    for nx, ny in sizes:
        spec = synth._spec("edge", nx, ny, 0.05, [], [], 0, 0.02, synth._edges())
        slots.append(b.admit(spec, nsteps=100))
    vecs = {"f64": (1, 2), "f32": (2, 4)}.get(storage, (4, 8))
    for vec in vecs:
        for pipe in (0, 1, 2, 3, 4):
            b.set_tile(vec, 8 if pipe != 3 else 5, 2, pipe)
            b.run(5)
    for k in slots:
        b.poll(k)
    a.check_all()
    b.close()
    assert not a.live, "blocks not given back"
    assert not a.violations, a.violations


@pytest.mark.parametrize("grouped", [True, False])
def test_batched_admission_refused_allocations_and_guard_bands(lbm, grouped):
    # lbm_batch_admit_many with its shared allocations (grouped) or two per domain: every
    # allocator request it makes refused in turn gives LBM_ENOMEM, admits nothing and
    # keeps nothing; a successful admission steps with the guard bands intact
    specs = [synth._spec("edge", nx, ny, 0.05, [synth._circle(1, nx / 3.0, ny / 2.0, max(1.0, min(nx, ny) / 4.0))],
                         [synth._body(nx / 3.0, ny / 2.0, 2.0)], 0, 0.02,
                         synth._edges("inlet", "outflow", "free_slip", "free_slip"), u_in=(0.02, 0.0))
             for nx, ny in [(65, 7), (130, 5), (257, 9), (97, 61), (3, 3)]]
    probe = GuardedAllocator()
    b = lbm.Batch("f16s", max_domains=8, graph_steps=0, allocator=probe)
    b.set_grouped_admission(grouped)
    before = probe.requests
    slots = b.admit_many(specs, nsteps=20)
    n_admit = probe.requests - before
    assert n_admit == (3 if grouped else 2 * len(specs) + 1)
    for pipe in (0, 3, 4):
        b.set_tile(8, 8 if pipe != 3 else 5, 2, pipe)
        b.run(5)
    b.poll_many(slots)
    probe.check_all()
    b.close()
    assert not probe.live and not probe.violations, probe.violations
    for k in range(n_admit):
        a = GuardedAllocator(fail_at=before + k)
        b = lbm.Batch("f16s", max_domains=8, graph_steps=0, allocator=a)
        b.set_grouped_admission(grouped)
        with pytest.raises(lbm.LbmError) as ei:
            b.admit_many(specs, nsteps=20)
        assert ei.value.status == LBM_ENOMEM, (k, ei.value)
        info = b.info()
        assert info["resident"] == 0 and info["bytes_in_use"] == 0
        a.check_all()
        b.close()
        assert not a.live, f"refusing request {k} leaked {len(a.live)} blocks"
        assert not a.violations


def test_injected_unstable_slot_is_reported_alone(lbm):
    spec = _small_channel()
    b = lbm.Batch("f32", max_domains=2, graph_steps=0)
    s0 = b.admit(spec, nsteps=50)
    s1 = b.admit(spec, nsteps=50)
    b.run(5)
    b.inject("unstable", s0)
    b.run(5)
    with pytest.raises(lbm.LbmError) as ei:
        b.poll(s0)
    assert ei.value.status == LBM_EUNSTABLE
    f1, _ = b.poll(s1)
    assert f1.shape[0] == 10 and np.all(np.isfinite(f1))
    b.evict(s0)  # as the server does with a failed request
    b.run(5)
    f1, _ = b.poll(s1)
    assert f1.shape[0] == 5
    b.close()
    with pytest.raises(lbm.LbmError):
        lbm.Batch("f32", max_domains=1).inject("unstable", 0)  # free slot: LBM_ENOTFOUND


@pytest.mark.parametrize("storage", ["f16s", "f32"])
def test_injected_wait_timeout_reports_etimeout(lbm, storage):
    spec = _small_channel()
    vec = 8 if storage == "f16s" else 4
    b = lbm.Batch(storage, max_domains=2, graph_steps=0)
    slots = [b.admit(spec, nsteps=50), b.admit(spec, nsteps=50)]
    b.set_tile(vec, 8, 2, 1)  # the shared-memory-staged sweep
    b.run(2)
    for k in slots:
        b.poll(k)  # clean so far
    b.inject("wait_timeout")
    b.run(2)
    for k in slots:
        with pytest.raises(lbm.LbmError) as ei:
            b.poll(k)
        assert ei.value.status == LBM_ETIMEOUT
        with pytest.raises(lbm.LbmError) as ei:
            b.moments(k)
        assert ei.value.status == LBM_ETIMEOUT
    b.inject("none")
    b.close()
    # the device is still usable: a fresh batch on the same pipeline matches the direct one
    outs = []
    for pipe in (1, 0):
        b = lbm.Batch(storage, max_domains=1, graph_steps=0)
        k = b.admit(spec, nsteps=20)
        b.set_tile(vec, 8, 2, pipe)
        b.run(20)
        b.poll(k)
        outs.append(b.get_populations(k))
        b.close()
    assert np.array_equal(outs[0], outs[1])
