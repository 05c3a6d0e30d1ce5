"""GPU path vs the FP64 oracle, element by element, through the C ABI.

FP64 storage must match the oracle to 1e-12 relative per population after 1000 steps
on seeded inputs; the reduced-precision storages are checked one step at a time to
within one unit of their stored type, and over many steps against drift bounds
derived in the design notes. The mask rasteriser must be bit-exact.
"""
import math

import numpy as np
import pytest

import codec
import oracle
import synth

pytestmark = pytest.mark.gpu


def _run_pair(lbm, spec, storage, steps, seed=1, amp=0.1):
    g0 = synth.random_populations(seed, spec["nx"], spec["ny"], amp)
    raw0 = codec.encode(g0, storage)
    dom = lbm.Domain(spec, storage=storage)
    dom.set_populations(raw0)
    f_gpu = dom.run(steps)
    raw = dom.get_populations()
    ora = oracle.Domain(spec, g=codec.decode(raw0, storage))
    f_ora = ora.run(steps)
    dom.close()
    return raw, f_gpu, ora, f_ora


@pytest.mark.parametrize("case", synth.PARITY_CASES)
def test_fp64_matches_oracle_1000_steps(lbm, case):
    spec = synth.parity_case(case)
    raw, f_gpu, ora, f_ora = _run_pair(lbm, spec, "f64", 1000)
    rel = np.abs(raw - ora.g) / np.abs(ora.g)
    assert rel.max() <= 1e-12, f"max relative population difference {rel.max():.3e}"
    # force series: every step, every body
    assert f_gpu.shape == f_ora.shape == (1000, len(spec["bodies"]), 2)
    scale = np.abs(f_ora).max()
    assert np.abs(f_gpu - f_ora).max() <= 1e-10 * scale + 1e-14


@pytest.mark.parametrize("case", ["channel_97x61", "mixed_edges_61x47"])
def test_fp64_srt_mode_matches_oracle_srt(lbm, case):
    # SRT-LBM-VP on the GPU is the TRT sweep with Lambda = (tau_s - 1/2)^2, i.e.
    # tau_a = tau_s (Sec. 2.1); it must match the oracle's separately written SRT update
    # (single relaxation time, unsplit Guo term) to the FP64 parity bound.
    spec = synth.parity_case(case)
    spec = dict(spec, magic_lambda=(3.0 * spec["nu"]) ** 2)
    g0 = synth.random_populations(7, spec["nx"], spec["ny"], 0.1)
    dom = lbm.Domain(spec, storage="f64")
    dom.set_populations(g0)
    f_gpu = dom.run(1000)
    raw = dom.get_populations()
    dom.close()
    ora = oracle.Domain(spec, g=g0)
    f_ora = ora.run(1000, srt=True)
    rel = np.abs(raw - ora.g) / np.abs(ora.g)
    assert rel.max() <= 1e-12, f"max relative population difference {rel.max():.3e}"
    assert np.abs(f_gpu - f_ora).max() <= 1e-10 * np.abs(f_ora).max() + 1e-14


@pytest.mark.parametrize("nx,ny", [(3, 3), (5, 4), (64, 3), (65, 7), (130, 5), (257, 9), (513, 4)])
@pytest.mark.parametrize("edges", ["periodic", "channel"])
def test_fp64_edge_sizes(lbm, nx, ny, edges):
    # ragged tails, a strip narrower than one warp, grids smaller than a tile
    e = synth._edges() if edges == "periodic" else synth._edges("inlet", "outflow", "free_slip", "free_slip")
    shapes = [synth._circle(1, nx / 3.0, ny / 2.0, max(1.0, min(nx, ny) / 4.0))]
    bodies = [synth._body(nx / 3.0, ny / 2.0, 2.0, omega=1e-3)]
    spec = synth._spec("edge", nx, ny, 0.05, shapes, bodies, 0, 0.02, e, u_in=(0.02, 0.0))
    raw, f_gpu, ora, f_ora = _run_pair(lbm, spec, "f64", 40, seed=nx * 1000 + ny)
    assert np.max(np.abs(raw - ora.g) / np.abs(ora.g)) <= 1e-13
    assert np.abs(f_gpu - f_ora).max() <= 1e-11 * max(np.abs(f_ora).max(), 1e-30) + 1e-15


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("case", ["channel_97x61", "mixed_edges_61x47"])
def test_reduced_precision_one_step_within_one_unit(lbm, storage, case):
    # Same decoded input on both sides; the GPU computes in FP32 and rounds to the
    # stored type (to nearest for FP32, stochastically for the 16-bit types), so each
    # stored value is within one unit of the oracle's FP64 result; the 16-bit rest
    # population also carries the moving populations' rounding residuals (mass kept).
    spec = synth.parity_case(case)
    raw, _, ora, _ = _run_pair(lbm, spec, storage, 1, seed=3)
    got = codec.decode(raw, storage)
    tol = codec.step_tol(ora.g, storage, spec)
    assert np.all(np.abs(got - ora.g) <= tol)


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_reduced_precision_mass_kept(lbm, storage):
    # 16-bit storages store the rest population as the pulled mass minus the rounded
    # moving populations: after one step, each node's stored mass equals its pulled mass
    # (computed by the oracle's pull from the same decoded state) within one unit of
    # the stored rest population (stochastic rounding), plus FP32 arithmetic (periodic
    # box: no ghost inflow).
    spec = synth.parity_case("mixed_edges_61x47")
    spec = dict(spec, edges=synth._edges())
    raw, _, ora, _ = _run_pair(lbm, spec, storage, 1, seed=5, amp=0.05)
    got = codec.decode(raw, storage)
    g0 = codec.decode(codec.encode(synth.random_populations(5, spec["nx"], spec["ny"], 0.05), storage), storage)
    pulled = oracle.stream(spec, g0).sum(axis=0)
    ulp0 = codec.stored_ulp(got[0] - codec.W[0], storage)
    err = np.abs(got.sum(axis=0) - pulled)
    assert np.all(err <= ulp0 + 1e-7), err.max()


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
def test_reduced_precision_drift(lbm, storage):
    # Each step adds at most one storage rounding (one unit of the largest stored
    # magnitude) plus the FP32 arithmetic error (a few units of 2^-24 on values of
    # order one); the collision does not amplify them, so after n steps the population
    # error is below n * (ulp_store + 4 * 2^-24). The 16-bit rest population takes the
    # eight moving populations' residuals as well: n * (9 ulp_store + 4 * 2^-24).
    steps = 200
    spec = synth.parity_case("channel_256x128")
    raw, f_gpu, ora, f_ora = _run_pair(lbm, spec, storage, steps, seed=4, amp=0.05)
    got = codec.decode(raw, storage)
    stored = np.abs(ora.g - (0.0 if storage == "f32" else codec.W)).max()
    ulp = float(codec.stored_ulp(np.array([stored]), storage)[0])
    tol = steps * (ulp + 4 * 2.0 ** -24)
    err = np.abs(got - ora.g)
    assert err[1:].max() <= tol, f"{storage}: drift {err[1:].max():.3e} > bound {tol:.3e}"
    tol0 = steps * ((9 if storage != "f32" else 1) * ulp + 4 * 2.0 ** -24)
    assert err[0].max() <= tol0, f"{storage}: rest drift {err[0].max():.3e} > bound {tol0:.3e}"


@pytest.mark.parametrize("spec_fn", [
    lambda: synth.couette(),
    lambda: synth.parity_case("mixed_edges_61x47"),
    lambda: synth.naca0012(10.0, 1000.0),
    lambda: synth.naca0012(3.7, 700.0, chord=57.3, nx=300, ny=160),
    lambda: synth.counter_rotating_pair(1.3),
    lambda: synth.batched_domains(4)[3],
    lambda: synth.precision_cylinder(large=False),
], ids=["couette", "mixed", "naca10", "naca_odd", "rotating", "side_by_side", "cyl600"])
def test_rasterizer_bit_exact(lbm, spec_fn):
    spec = spec_fn()
    dom = lbm.Domain(spec, storage="f16s", force_every=0)
    m_gpu = dom.mask()
    dom.close()
    m_ora = oracle.rasterize(spec)
    assert np.array_equal(m_gpu, m_ora), f"{(m_gpu != m_ora).sum()} nodes differ"


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
def test_initial_state_and_moments(lbm, storage):
    # Step (1): g = f^eq(rho0, u0); the moments of the initial state reproduce rho0 and
    # u0 away from obstacles and edges.
    spec = synth.parity_case("channel_97x61")
    dom = lbm.Domain(spec, storage=storage)
    raw = dom.get_populations()
    ora = oracle.Domain(spec)
    want = ora.g if storage in ("f64", "f32") else ora.g - codec.W
    got = codec.decode(raw, storage) - (0.0 if storage in ("f64", "f32") else codec.W)
    tol = codec.stored_ulp(want, storage) * 0.5 + 1e-17
    assert np.all(np.abs(got - want) <= tol)
    # moments of a random state vs the oracle's moments of the same decoded state
    g0 = synth.random_populations(9, spec["nx"], spec["ny"])
    raw0 = codec.encode(g0, storage)
    dom.set_populations(raw0)
    rho, ux, uy = dom.moments()
    o = oracle.Domain(spec, g=codec.decode(raw0, storage))
    r2, x2, y2 = o.moments()
    t = np.full(rho.shape, 1e-14 if storage == "f64" else 2e-6)
    t[:, 0] += 3 * codec.ghost_ulp(spec, storage)  # three ghost populations enter column 0
    assert np.all(np.abs(rho - r2) <= t) and np.all(np.abs(ux - x2) <= t) and np.all(np.abs(uy - y2) <= t)
    dom.close()


def test_checkpoint_resume_bit_identical(lbm):
    spec = synth.parity_case("channel_256x128")
    a = lbm.Domain(spec, storage="f16s")
    fa = a.run(200)
    pa = a.get_populations()
    b = lbm.Domain(spec, storage="f16s")
    fb1 = b.run(100)
    snap = b.get_populations()
    b.close()
    c = lbm.Domain(spec, storage="f16s")
    c.set_populations(snap)
    c.set_steps_done(100)  # the step index keys the 16-bit rounding's random bits
    with pytest.raises(lbm.LbmError):
        c.set_steps_done(-1)
    fb2 = c.run(100)
    assert np.array_equal(c.get_populations().view(np.uint16), pa.view(np.uint16))
    assert np.array_equal(np.concatenate([fb1, fb2]), fa)
    a.close()
    c.close()


def test_unstable_state_is_reported(lbm):
    spec = synth.parity_case("periodic_97x61")
    dom = lbm.Domain(spec, storage="f32")
    g = synth.random_populations(2, spec["nx"], spec["ny"]).astype(np.float32)
    g[:, 10, 10] = -1.0  # negative density at one node
    dom.set_populations(g)
    dom.step(3)
    with pytest.raises(lbm.LbmError) as ei:
        dom.forces()
    assert ei.value.status == 4  # LBM_EUNSTABLE
    dom.close()


def test_invalid_mask_body_id_rejected(lbm):
    spec = synth.parity_case("periodic_97x61")
    mask = oracle.rasterize(spec)
    mask[5, 5] = 7  # only 2 bodies given
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Domain(spec, storage="f32", mask=mask)
    assert ei.value.status == 1  # LBM_EINVAL


def test_host_mask_equals_geometry(lbm):
    spec = synth.parity_case("channel_97x61")
    g0 = synth.random_populations(5, spec["nx"], spec["ny"])
    a = lbm.Domain(spec, storage="f64")
    b = lbm.Domain(spec, storage="f64", mask=oracle.rasterize(spec))
    a.set_populations(g0)
    b.set_populations(g0)
    assert np.array_equal(a.run(30), b.run(30))
    assert np.array_equal(a.get_populations(), b.get_populations())
    a.close()
    b.close()


@pytest.mark.parametrize("storage,vec", [("f64", 1), ("f64", 2), ("f32", 2), ("f32", 4),
                                         ("f16s", 4), ("f16s", 8), ("bf16s", 8)])
@pytest.mark.parametrize("nx,ny,edges", [(5, 4, "periodic"), (65, 7, "channel"), (257, 9, "periodic"),
                                         (600, 11, "channel")])
def test_tma_pipeline_matches_direct_and_oracle(lbm, storage, vec, nx, ny, edges):
    # The TMA-staged and the register-prefetched sweeps, and the direct one compiled for
    # 20 and 24 resident warps, perform the same arithmetic as the direct one: identical
    # results for every storage and strip width, and FP64 within 1e-13 of the oracle.
    e = synth._edges() if edges == "periodic" else synth._edges("inlet", "outflow", "free_slip", "free_slip")
    shapes = [synth._circle(1, nx / 3.0, ny / 2.0, max(1.0, min(nx, ny) / 4.0))]
    bodies = [synth._body(nx / 3.0, ny / 2.0, 2.0, omega=1e-3)]
    spec = synth._spec("tma", nx, ny, 0.05, shapes, bodies, 0, 0.02, e, u_in=(0.02, 0.0))
    g0 = codec.encode(synth.random_populations(77 + nx, nx, ny, 0.05), storage)
    out = []
    for pipe in (0, 1, 2, 3, 4):
        b = lbm.Batch(storage, max_domains=1, graph_steps=0)
        k = b.admit(spec, nsteps=30)
        b.set_tile(vec, 4, 3, pipe)
        b.set_populations(k, g0)
        b.run(30)
        f, _ = b.poll(k)
        out.append((b.get_populations(k), f))
        b.close()
    for o in out[1:]:
        assert np.array_equal(out[0][0].view(np.uint8), o[0].view(np.uint8))
        assert np.array_equal(out[0][1], o[1])
    if storage == "f64":
        ora = oracle.Domain(spec, g=codec.decode(g0, storage))
        ora.run(30)
        assert np.max(np.abs(out[1][0] - ora.g) / np.abs(ora.g)) <= 1e-13
