"""Batched uneven domains: results do not depend on the batch composition, the tile
shape, graph replay or the autotuner; admission respects the memory budget."""
import numpy as np
import pytest

import codec
import oracle
import synth

pytestmark = pytest.mark.gpu


def _specs():
    a = synth.parity_case("channel_256x128")
    b = synth.parity_case("mixed_edges_61x47")
    c = synth.batched_domains(3)[2]
    c = dict(c, nx=420, ny=210, shapes=[synth._circle(1, 105, 105, 20), synth._circle(2, 200, 95, 20)],
             bodies=[synth._body(105, 105, 40), synth._body(200, 95, 40)])
    return [a, b, c]


@pytest.mark.parametrize("storage", ["f16s", "f32"])
def test_batch_equals_alone(lbm, storage):
    specs = _specs()
    steps = [300, 170, 250]  # uneven step targets: domains finish mid-run
    batch = lbm.Batch(storage, max_domains=8, graph_steps=16)
    slots = [batch.admit(s, nsteps=n) for s, n in zip(specs, steps)]
    forces = {k: [] for k in slots}
    while True:
        ran = batch.run(64)
        for k in slots:
            f, _ = batch.poll(k)
            forces[k].append(f)
        if ran == 0:
            break
    for k, s, n in zip(slots, specs, steps):
        assert batch.steps_done(k) == n
        alone = lbm.Domain(s, storage=storage)
        fa = alone.run(n)
        assert np.array_equal(np.concatenate(forces[k]), fa)
        pa, pb = alone.get_populations(), batch.get_populations(k)
        assert np.array_equal(pa, pb) if storage == "f32" else np.array_equal(pa.view(np.uint16), pb.view(np.uint16))
        alone.close()
    batch.close()


def test_tile_shape_and_graphs_do_not_change_results(lbm):
    spec = synth.parity_case("channel_256x128")
    g0 = codec.encode(synth.random_populations(8, 256, 128, 0.05), "f16s")
    ref = None
    for vec, warps, rows, pipe, graph in [(8, 8, 2, 0, 16), (4, 4, 1, 0, 0), (8, 16, 4, 1, 7),
                                          (4, 2, 3, 1, 32), (8, 4, 4, 1, 0), (8, 8, 3, 2, 16),
                                          (4, 2, 4, 2, 0), (8, 10, 2, 3, 16), (4, 5, 3, 3, 0),
                                          (8, 12, 4, 4, 7), (8, 6, 1, 4, 0)]:
        batch = lbm.Batch("f16s", max_domains=2, graph_steps=graph)
        k = batch.admit(spec, nsteps=100)
        batch.set_tile(vec, warps, rows, pipe)
        batch.set_populations(k, g0)
        while batch.run(45):
            pass
        f, done = batch.poll(k)
        out = (batch.get_populations(k).view(np.uint16), f)
        assert done
        if ref is None:
            ref = out
        else:
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
        batch.close()


def test_autotune_keeps_state_and_results(lbm):
    specs = _specs()
    batch = lbm.Batch("f16s", max_domains=4, graph_steps=16)
    slots = [batch.admit(s, nsteps=60) for s in specs]
    batch.run(20)
    before = [batch.get_populations(k).view(np.uint16).copy() for k in slots]
    us = batch.autotune(reps=3)
    assert us > 0
    after = [batch.get_populations(k).view(np.uint16) for k in slots]
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    vec, warps, rows, pipe = batch.get_tile()
    assert vec in (4, 8) and 1 <= warps <= 16 and 1 <= rows <= 16 and pipe in (0, 1, 2, 3, 4)
    batch.run(40)
    ref = lbm.Domain(specs[0], storage="f16s")
    ref.step(60)
    assert np.array_equal(ref.get_populations().view(np.uint16), batch.get_populations(slots[0]).view(np.uint16))
    ref.close()
    batch.close()


def test_autotune_cache_reuses_shapes_per_workload_class(lbm, tmp_path):
    from paper_1901_08766_gb300.tuning import TuneCache
    specs = _specs()
    path = str(tmp_path / "tune.json")
    cache = TuneCache(path)
    a = lbm.Batch("f16s", max_domains=4, graph_steps=0)
    for s in specs:
        a.admit(s, nsteps=40)
    us = a.autotune(reps=2, cache=cache)
    tile = a.get_tile()
    assert cache.misses == 1 and us > 0
    # a second batch of the same workload class takes the stored shape without timing
    b = lbm.Batch("f16s", max_domains=4, graph_steps=0)
    slots = [b.admit(s, nsteps=40) for s in specs]
    b.set_tile(4, 4, 1, 0)
    n0 = b.info()["kernel_launches"]
    assert b.workload_key() == a.workload_key()
    assert b.autotune(reps=2, cache=TuneCache(path)) == us
    assert b.get_tile() == tile and b.info()["kernel_launches"] == n0
    # and steps as the tuned batch does, bit for bit
    b.run(40)
    a.run(40)
    for k in slots:
        assert np.array_equal(a.get_populations(k).view(np.uint16), b.get_populations(k).view(np.uint16))
    a.close()
    b.close()


def test_admission_budget_and_eviction(lbm):
    spec = synth.parity_case("channel_97x61")
    need = lbm.domain_bytes(spec, "f16s")
    batch = lbm.Batch("f16s", max_domains=8, hbm_budget=int(2.5 * need) + 4096)
    a = batch.admit(spec, nsteps=10)
    b = batch.admit(spec, nsteps=10)
    assert batch.try_admit(spec, nsteps=10) is None  # over budget
    batch.run(10)
    f, done = batch.poll(a)
    assert done and f.shape == (10, 2, 2)
    batch.evict(a)
    c = batch.try_admit(spec, nsteps=5)
    assert c is not None
    assert batch.run(100) == 5  # only the new domain still has steps to run
    info = batch.info()
    assert info["resident"] == 2 and info["kernel_launches"] > 0
    batch.close()


def test_full_size_batch_one_step_sampled_parity(lbm):
    # The batched workload at full size in the benchmark's launch configuration: every
    # domain starts from seeded FP16-shifted populations and takes one step on the GPU;
    # each domain's result is compared with the oracle's step of the same decoded state.
    specs = synth.batched_domains(64)
    batch = lbm.Batch("f16s", max_domains=64, graph_steps=32)
    sample = range(0, 64, 9)  # domains of every size class; the others start at rest flow
    slots = []
    for d, s in enumerate(specs):
        k = batch.admit(s, nsteps=1)
        if d in sample:
            batch.set_populations(k, codec.encode(
                synth.random_populations(1000 + d, s["nx"], s["ny"], 0.05), "f16s"))
        slots.append(k)
    batch.autotune(reps=3)
    batch.run(1)
    for d in sample:
        s = specs[d]
        raw0 = codec.encode(synth.random_populations(1000 + d, s["nx"], s["ny"], 0.05), "f16s")
        ora = oracle.Domain(s, g=codec.decode(raw0, "f16s"))
        f_ora = ora.run(1)
        got = codec.decode(batch.get_populations(slots[d]), "f16s")
        tol = codec.step_tol(ora.g, "f16s", s)
        assert np.all(np.abs(got - ora.g) <= tol)
        f_gpu, _ = batch.poll(slots[d])
        assert np.allclose(f_gpu, f_ora, rtol=1e-4, atol=1e-5)
    batch.close()


def test_randomised_membership_tiles_and_graphs_equal_alone(lbm):
    # domains admitted and evicted at random chunk boundaries while the tile shape and
    # register budget change (and sometimes are set to the current one again), graphs of
    # 8 steps replayed: each domain's populations and force series equal its run alone
    rng = np.random.default_rng(190108766)
    base = [synth.parity_case(n) for n in ("channel_97x61", "periodic_97x61", "mixed_edges_61x47")]
    tiles = [(8, 12, 4, 4), (8, 6, 4, 4), (8, 10, 2, 3), (4, 8, 1, 0), (8, 16, 4, 0), (8, 8, 2, 1)]
    b = lbm.Batch("f16s", max_domains=5, graph_steps=8)
    live, done, specs, raws, forces = {}, {}, {}, {}, {}
    admitted = 0
    tile = tiles[0]
    b.set_tile(*tile)
    for chunk in range(40):
        if admitted < 9 and len(live) < 5 and rng.random() < 0.6:
            sp = dict(base[admitted % 3], name=f"r{admitted}")
            n = int(rng.integers(20, 90))
            raw = codec.encode(synth.random_populations(300 + admitted, sp["nx"], sp["ny"], 0.05), "f16s")
            k = b.admit(sp, nsteps=n)
            b.set_populations(k, raw)
            live[k] = admitted
            specs[admitted], raws[admitted], forces[admitted] = (sp, n), raw, []
            admitted += 1
        if rng.random() < 0.3:
            tile = tiles[int(rng.integers(len(tiles)))] if rng.random() < 0.7 else tile
            b.set_tile(*tile)
        b.run(int(rng.integers(3, 20)))
        for k in list(live):
            f, fin = b.poll(k)
            forces[live[k]].append(f)
            if fin:
                done[live[k]] = b.get_populations(k).view(np.uint16).copy()
                b.evict(k)
                del live[k]
    while b.run(50):
        pass
    for k in list(live):
        f, fin = b.poll(k)
        assert fin
        forces[live[k]].append(f)
        done[live[k]] = b.get_populations(k).view(np.uint16).copy()
    b.close()
    assert len(done) == admitted >= 5
    for r, pops in done.items():
        sp, n = specs[r]
        d = lbm.Domain(sp, storage="f16s")
        d.set_populations(raws[r])
        f = d.run(n)
        assert np.array_equal(d.get_populations().view(np.uint16), pops), sp["name"]
        assert np.array_equal(np.concatenate(forces[r]), f), sp["name"]
        d.close()
