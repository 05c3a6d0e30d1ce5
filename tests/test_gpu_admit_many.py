"""Batched admission (lbm_batch_admit_many) against admitting the same domains one by one
(lbm_batch_admit): the same masks, solid-node lists (seen through the force series),
initial states and, after stepping, the same populations bit for bit, for every storage
type, ragged sizes, NACA sections and domains without bodies. Failures admit nothing."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

LBM_EINVAL, LBM_EBUSY = 1, 6


def _mixed_specs():
    specs = synth.batched_domains(6)
    specs.append(synth.naca0012(7.0, 800.0, chord=60.0, U=0.05, nx=301, ny=133, steps=100))
    specs.append(synth._spec("empty", 65, 7, 0.05, [], [], 0, 0.02,
                             synth._edges("inlet", "outflow", "free_slip", "free_slip"), u_in=(0.02, 0.0)))
    specs.append(synth.parity_case("periodic_97x61"))
    specs.append(synth.couette(n=70, r_inner=12.0, r_outer=30.0))
    specs.append(_thick_and_many())
    return specs


def _thick_and_many():
    # a NACA section whose thickness ratio (2.6) takes it beyond one chord of its quarter
    # chord across the chord line, tilted; and 70 small circles on three bodies (more
    # shapes than the rasteriser culls per row)
    sh = [{"kind": "naca4", "body": 1, "cx": 60.3, "cy": 50.2, "chord": 16.0, "thickness": 2.6,
           "aoa_rad": 1.2}]
    for q in range(70):
        sh.append(synth._circle(2 + q % 3, 110.0 + 7.3 * (q % 10), 12.0 + 11.1 * (q // 10), 2.6 + 0.1 * (q % 4)))
    bodies = [synth._body(60.3, 50.2, 16.0)] + [synth._body(140.0, 50.0, 10.0) for _ in range(3)]
    return synth._spec("thick_many", 197, 101, 0.05, sh, bodies, 0, 0.02,
                       synth._edges("inlet", "outflow", "free_slip", "free_slip"), u_in=(0.02, 0.0))


def test_admit_many_masks_equal_the_oracle(lbm):
    import oracle
    specs = _mixed_specs()
    b = lbm.Batch("f16s", max_domains=len(specs), graph_steps=0)
    slots = b.admit_many(specs, nsteps=1)
    for sp, k in zip(specs, slots):
        ref = oracle.rasterize(sp)
        assert np.array_equal(b.mask(k), ref), sp["name"]
    # the thick section reaches beyond one chord across its chord line
    m = oracle.rasterize(specs[-1])
    ys, xs = np.nonzero(m == 1)
    assert np.hypot(xs - 60.3, ys - 50.2).max() > 16.0 + 2.0
    b.close()


def _run(lbm, storage, specs, batched, steps=23):
    b = lbm.Batch(storage, max_domains=len(specs) + 2, graph_steps=8)
    if batched:
        slots = b.admit_many(specs, nsteps=steps + 5, force_capacity=64)
    else:
        slots = [b.admit(sp, nsteps=steps + 5, force_capacity=64) for sp in specs]
    masks = [b.mask(k) for k in slots]
    init = [b.get_populations(k) for k in slots]
    b.run(steps)
    out = [(b.get_populations(k), b.poll(k)[0]) for k in slots]
    info = b.info()
    b.close()
    return slots, masks, init, out, info


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
def test_admit_many_equals_one_by_one(lbm, storage):
    specs = _mixed_specs()
    s1, m1, i1, o1, info1 = _run(lbm, storage, specs, False)
    s2, m2, i2, o2, info2 = _run(lbm, storage, specs, True)
    assert s1 == s2
    assert info1["bytes_in_use"] == info2["bytes_in_use"] and info1["cells"] == info2["cells"]
    for a, b in zip(m1, m2):
        assert np.array_equal(a, b)
    for a, b in zip(i1, i2):
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    for (pa, fa), (pb, fb) in zip(o1, o2):
        assert np.array_equal(pa.view(np.uint8), pb.view(np.uint8))
        assert np.array_equal(fa, fb)


def test_admit_many_into_a_batch_with_residents_and_mixed_kinds(lbm):
    # slots already taken, then a batched group that also holds a moving domain (admitted
    # on its own); the whole batch steps as when every domain was admitted one by one
    specs = _mixed_specs()
    moving = dict(synth.parity_case("channel_97x61"), moving=True)
    b = lbm.Batch("f16s", max_domains=16, graph_steps=0)
    first = b.admit(specs[0], nsteps=30)
    rest = b.admit_many(specs[1:] + [moving], nsteps=30)
    assert first not in rest and len(set(rest)) == len(rest)
    b.run(30)
    got = [b.get_populations(k) for k in [first] + rest]
    b.close()
    ref = lbm.Batch("f16s", max_domains=16, graph_steps=0)
    ks = [ref.admit(sp, nsteps=30) for sp in specs + [moving]]
    ref.run(30)
    want = [ref.get_populations(k) for k in ks]
    ref.close()
    for g, w in zip(got, want):
        assert np.array_equal(g.view(np.uint16), w.view(np.uint16))


def test_admit_many_failures_admit_nothing(lbm):
    specs = synth.batched_domains(4)
    b = lbm.Batch("f16s", max_domains=8, graph_steps=0)
    k0 = b.admit(specs[0], nsteps=10)
    before = b.info()
    # a shape naming a body that does not exist
    bad = dict(specs[2], shapes=[dict(s, body=3) for s in specs[2]["shapes"]])
    with pytest.raises(lbm.LbmError) as ei:
        b.admit_many([specs[1], bad], nsteps=10)
    assert ei.value.status == LBM_EINVAL
    assert b.info() == before
    # more domains than free slots
    with pytest.raises(lbm.LbmError) as ei:
        b.admit_many(synth.batched_domains(8), nsteps=10)
    assert ei.value.status == LBM_EBUSY
    assert b.info() == before
    b.close()
    # over the memory budget
    need = sum(lbm.domain_bytes(sp, "f16s") for sp in specs)
    c = lbm.Batch("f16s", max_domains=8, hbm_budget=need // 2, graph_steps=0)
    with pytest.raises(lbm.LbmError) as ei:
        c.admit_many(specs, nsteps=10)
    assert ei.value.status == LBM_EBUSY
    assert c.info()["resident"] == 0 and c.info()["bytes_in_use"] == 0
    c.close()
    del k0


@pytest.mark.parametrize("n,cap", [(6, 32), (6, 7), (3, 7)])
def test_poll_many_equals_polls(lbm, n, cap):
    # from four slots on poll_many gathers every slot's status word and ring entries on the
    # device and reads them back at once; with a ring of 7 entries the reads wrap around it
    specs = synth.batched_domains(n)
    got, want = [], []
    for many in (True, False):
        b = lbm.Batch("f16s", max_domains=8, graph_steps=0)
        slots = b.admit_many(specs, nsteps=[11 + k for k in range(len(specs))], force_capacity=cap)
        for _ in range(3):
            b.run(5)
            out = b.poll_many(slots) if many else [b.poll(k) for k in slots]
            (got if many else want).append(out)
        b.close()
    for ga, wa in zip(got, want):
        for (fa, da), (fb, db) in zip(ga, wa):
            assert da == db and np.array_equal(fa, fb)
    # nsteps 11, 12, ... after 15 steps
    assert [d for _, d in got[-1]] == [11 + k <= 15 for k in range(n)]
    assert all(len(f) == 5 for f, _ in got[0])


def test_batched_admission_memory_returns_with_its_last_domain(lbm):
    # the domains of one batched admission share its allocations: their memory stays
    # counted until the last of them leaves; the others step on unchanged meanwhile
    specs = synth.batched_domains(4)
    b = lbm.Batch("f16s", max_domains=8, graph_steps=0)
    slots = b.admit_many(specs, nsteps=20, force_capacity=32)
    held = b.info()["bytes_in_use"]
    assert held >= sum(lbm.domain_bytes(sp, "f16s", force_capacity=32) for sp in specs)
    b.run(4)
    b.evict(slots[0])
    b.evict(slots[2])
    assert b.info()["bytes_in_use"] == held and b.info()["resident"] == 2
    b.run(16)
    got = [(b.get_populations(k), b.poll(k)[0]) for k in (slots[1], slots[3])]
    # a domain admitted alone returns its memory at once
    k = b.admit(specs[0], nsteps=5)
    assert b.info()["bytes_in_use"] > held
    b.evict(k)
    assert b.info()["bytes_in_use"] == held
    b.evict(slots[1])
    assert b.info()["bytes_in_use"] == held
    b.evict(slots[3])
    assert b.info()["bytes_in_use"] == 0 and b.info()["resident"] == 0
    # the freed group entry serves the next batched admission
    again = b.admit_many(specs[:2], nsteps=3)
    b.run(3)
    assert all(d for _, d in b.poll_many(again))
    b.close()
    # with grouped admission off, each domain's memory returns at its eviction
    c = lbm.Batch("f16s", max_domains=8, graph_steps=0)
    c.set_grouped_admission(False)
    ks = c.admit_many(specs, nsteps=5, force_capacity=32)
    assert c.info()["bytes_in_use"] == held
    c.evict(ks[0])
    assert c.info()["bytes_in_use"] < held
    for k in ks[1:]:
        c.evict(k)
    assert c.info()["bytes_in_use"] == 0
    c.close()
    for (pa, fa), sp in zip(got, (specs[1], specs[3])):
        ref = lbm.Batch("f16s", max_domains=1, graph_steps=0)
        r = ref.admit(sp, nsteps=20, force_capacity=32)
        ref.run(20)
        assert np.array_equal(pa.view(np.uint16), ref.get_populations(r).view(np.uint16))
        assert np.array_equal(fa, ref.poll(r)[0])
        ref.close()


@pytest.mark.parametrize("moving", [True, 2])
def test_thick_section_moving_masks_equal_the_oracle(lbm, moving):
    # the per-row column culling of moving and rotating domains reaches the thick section
    sp = _thick_and_many()
    sp = dict(sp, shapes=sp["shapes"][:1], bodies=[dict(sp["bodies"][0], vx=0.05, vy=-0.02, omega=0.01)],
              moving=moving)
    import oracle
    d = lbm.Domain(sp, storage="f32")
    assert np.array_equal(d.mask(), oracle.rasterize(sp, 0))
    d.run(40)
    assert np.array_equal(d.mask(), oracle.rasterize(sp, 40))
    d.close()
