"""Batches of 3D domains (lbm3_batch_*): every domain of a batch steps exactly as it does
alone (populations and force series bit for bit, every storage, both lattices, every
register budget), through uneven step targets, evictions and admissions mid-run; the
FP64 batch matches the 3D oracle; the guards."""
import numpy as np
import pytest

import codec
import synth
import test_gpu_3d as t3
from oracle import d3 as ora3

pytestmark = pytest.mark.gpu

CASES = ["sphere_channel_150x20x12", "periodic_bodies_97x18x14", "slip_y_periodic_z_70x16x22"]


def _pops(spec, storage, seed):
    g0 = synth.random_populations3(seed, spec["nx"], spec["ny"], spec["nz"], 0.05, q=ora3.nq(spec))
    return codec.encode(g0, storage)


def _alone(lbm, spec, storage, raw0, steps):
    d = lbm.Domain3(spec, storage=storage, force_capacity=512)
    d.set_populations(raw0)
    f = d.run(steps)
    out = d.get_populations().view(np.uint8).copy()
    d.close()
    return out, f


def _batched(lbm, specs, storage, raws, targets, q, pipeline=None, chunk=25):
    b = lbm.Batch3(storage, lattice=q, max_domains=len(specs) + 1)
    if pipeline is not None:
        b.set_tile(pipeline)
    slots = [b.admit(sp, nsteps=n, force_capacity=512) for sp, n in zip(specs, targets)]
    for k, raw in zip(slots, raws):
        b.domain(k).set_populations(raw)
    forces = {k: [] for k in slots}
    while b.run(chunk):
        for k in slots:
            forces[k].append(b.poll(k)[0])
    out = []
    for k, n in zip(slots, targets):
        f, done = b.poll(k)
        assert done
        dom = b.domain(k)
        assert dom.steps_done() == n
        out.append((dom.get_populations().view(np.uint8).copy(), np.concatenate(forces[k] + [f])))
    info = b.info()
    b.close()
    return out, info


@pytest.mark.parametrize("q", [19, 15])
@pytest.mark.parametrize("storage", ["f16s", "bf16s", "f32", "f64"])
def test_batch3_equals_alone(lbm, storage, q):
    specs = [t3._case(c, q) for c in CASES]
    targets = [70, 45, 90]  # uneven: domains finish mid-chunk
    raws = [_pops(sp, storage, 31 + i) for i, sp in enumerate(specs)]
    got, info = _batched(lbm, specs, storage, raws, targets, q)
    assert info["resident"] == 3 and info["kernel_launches"] > 0
    for sp, raw, n, (pops, f) in zip(specs, raws, targets, got):
        ref_pops, ref_f = _alone(lbm, sp, storage, raw, n)
        assert np.array_equal(pops, ref_pops), sp["name"]
        assert f.shape == ref_f.shape and np.array_equal(f, ref_f), sp["name"]


@pytest.mark.parametrize("q", [19, 15])
@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_batch3_register_budgets_give_the_same_bits(lbm, storage, q):
    specs = [t3._case(c, q) for c in CASES[:2]]
    raws = [_pops(sp, storage, 7 + i) for i, sp in enumerate(specs)]
    runs = [_batched(lbm, specs, storage, raws, [40, 33], q, pipeline=p, chunk=16)[0] for p in (0, 3, 4)]
    for r in runs[1:]:
        for (a, fa), (b, fb) in zip(r, runs[0]):
            assert np.array_equal(a, b) and np.array_equal(fa, fb)


def test_batch3_evict_and_admit_mid_run(lbm):
    # a domain evicted after 30 steps and a new one admitted into its slot leave the
    # others' results as they are alone
    storage, q = "f16s", 19
    a, b_, c = (t3._case(n, q) for n in CASES)
    raws = {n: _pops(sp, storage, 11 + i) for i, (n, sp) in enumerate(zip("abc", (a, b_, c)))}
    b = lbm.Batch3(storage, lattice=q, max_domains=2)
    ka = b.admit(a, nsteps=80, force_capacity=512)
    kb = b.admit(b_, nsteps=80, force_capacity=512)
    b.domain(ka).set_populations(raws["a"])
    b.domain(kb).set_populations(raws["b"])
    with pytest.raises(lbm.LbmError):  # both slots taken
        b.admit(c, nsteps=10)
    assert b.run(30) == 30
    fa = [b.poll(ka)[0]]
    b.evict(kb)
    kc = b.admit(c, nsteps=50, force_capacity=512)
    assert kc == kb
    b.domain(kc).set_populations(raws["c"])
    while b.run(20):
        fa.append(b.poll(ka)[0])
    fa.append(b.poll(ka)[0])
    fc, done = b.poll(kc)
    assert done
    pa = b.domain(ka).get_populations().view(np.uint8).copy()
    pc = b.domain(kc).get_populations().view(np.uint8).copy()
    b.close()
    ra, rfa = _alone(lbm, a, storage, raws["a"], 80)
    rc, rfc = _alone(lbm, c, storage, raws["c"], 50)
    assert np.array_equal(pa, ra) and np.array_equal(np.concatenate(fa), rfa)
    assert np.array_equal(pc, rc) and np.array_equal(fc, rfc)


def test_batch3_fp64_matches_the_oracle(lbm):
    q = 19
    spec = t3._case("periodic_bodies_97x18x14", q)
    g0 = synth.random_populations3(5, spec["nx"], spec["ny"], spec["nz"], 0.1, q=q)
    b = lbm.Batch3("f64", lattice=q, max_domains=2)
    k = b.admit(spec, nsteps=300, force_capacity=512)
    k2 = b.admit(t3._case("sphere_channel_150x20x12", q), nsteps=120, force_capacity=512)
    b.domain(k).set_populations(g0)
    f = []
    while b.run(100):
        f.append(b.poll(k)[0])
        b.poll(k2)
    f.append(b.poll(k)[0])
    g = b.domain(k).get_populations()
    b.close()
    ora = ora3.Domain(spec, g=g0)
    fo = ora.run(300)
    assert (np.abs(g - ora.g) / np.abs(ora.g)).max() <= 1e-12
    f = np.concatenate(f)
    assert np.abs(f - fo).max() <= 1e-10 * np.abs(fo).max() + 1e-14


def test_batch3_guards(lbm):
    q = 19
    spec = t3._case("sphere_channel_150x20x12", q)
    b = lbm.Batch3("f32", lattice=q, max_domains=4,
                   hbm_budget=int(1.5 * lbm.load().lbm3_domain_bytes(*_bytes_args(spec, "f32"))))
    with pytest.raises(lbm.LbmError):  # another lattice
        b.admit(dict(spec, lattice=15))
    with pytest.raises(lbm.LbmError):  # a moving domain
        b.admit(dict(spec, moving=True))
    k = b.admit(spec, nsteps=100, force_capacity=16)
    with pytest.raises(lbm.LbmError) as e:  # over the memory budget
        b.admit(spec, nsteps=10)
    assert e.value.status == 6
    with pytest.raises(lbm.LbmError) as e:  # the force ring holds 16 entries
        b.run(40)
    assert e.value.status == 6
    assert b.run(16) == 16
    f, done = b.poll(k)
    assert f.shape == (16, 1, 3) and not done
    with pytest.raises(RuntimeError):
        b.domain(k).step(1)
    with pytest.raises(lbm.LbmError):
        b.evict(3)
    with pytest.raises(lbm.LbmError):
        b.set_tile(3)  # FP32 has one register budget
    b.evict(k)
    assert b.info()["resident"] == 0 and b.run(10) == 0
    b.close()
    # another storage than the batch's, through the C call (the binding converts specs to
    # the batch's storage)
    import ctypes as C
    from paper_1901_08766_gb300 import _native
    b2 = lbm.Batch3("f16s", lattice=q, max_domains=1)
    p = _native.params3_from_spec(spec, "f32")
    sh, ns = _native.shapes3_from_spec(spec)
    bd, nb = _native.bodies3_from_spec(spec)
    slot = C.c_int32()
    assert lbm.load().lbm3_batch_admit(b2._h, C.byref(p), sh, ns, bd, nb, 10, C.byref(slot)) == 1
    b2.close()


def _bytes_args(spec, storage):
    import ctypes as C
    from paper_1901_08766_gb300 import _native
    p = _native.params3_from_spec(spec, storage, 1, 16)
    return C.byref(p), len(spec["bodies"])


def test_batch3_two_groups_and_a_domain_without_bodies(lbm):
    # 19 domains: two launch groups per step (16 + 3, then fewer as domains finish); one
    # domain has no bodies, one a body without solid nodes
    q, storage = 15, "f16s"
    specs = []
    for i in range(17):
        c = (10.5 + i % 5, 8.25, 6.5)
        specs.append(synth.spec3(f"g{i}", 24 + 4 * (i % 6), 16 + (i % 3), 12 + (i % 4), 0.05,
                                 [synth.sphere(1, c, 2.5 + 0.2 * (i % 3))], [synth.body3(c, 5.0)], 0, 0.02,
                                 synth.channel_edges3(), u_in=(0.02, 0.0, 0.0), u0=(0.02, 0.0, 0.0), lattice=q))
    specs.append(synth.spec3("nobody", 40, 12, 10, 0.05, [], [], 0, 0.02, synth.channel_edges3(),
                             u_in=(0.02, 0.0, 0.0), u0=(0.02, 0.0, 0.0), lattice=q))
    far = (200.0, 6.0, 5.0)  # a body whose sphere lies outside the grid: zero force entries
    specs.append(synth.spec3("nosolid", 36, 12, 10, 0.05, [synth.sphere(1, far, 3.0)], [synth.body3(far, 6.0)],
                             0, 0.02, synth.channel_edges3(), u_in=(0.02, 0.0, 0.0), u0=(0.02, 0.0, 0.0),
                             lattice=q))
    targets = [20 + 3 * (i % 7) for i in range(len(specs))]
    raws = [_pops(sp, storage, 50 + i) for i, sp in enumerate(specs)]
    b = lbm.Batch3(storage, lattice=q, max_domains=len(specs))
    slots = [b.admit(sp, nsteps=n, force_capacity=64) for sp, n in zip(specs, targets)]
    for k, raw in zip(slots, raws):
        b.domain(k).set_populations(raw)
    while b.run(10):
        pass
    got = []
    for k in slots:
        f, done = b.poll(k)
        assert done
        got.append((b.domain(k).get_populations().view(np.uint8).copy(), f))
    b.close()
    for sp, raw, n, (pops, f) in zip(specs, raws, targets, got):
        ref_pops, ref_f = _alone(lbm, sp, storage, raw, n)
        assert np.array_equal(pops, ref_pops), sp["name"]
        assert np.array_equal(f, ref_f), sp["name"]
