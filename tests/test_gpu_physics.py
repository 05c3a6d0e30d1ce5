"""Physics of the GPU path on the paper's workloads.

- Cylindrical Couette flow (Sec. 3.1), FP64: matches the oracle after 20 000 steps and
  the closed form u_theta = A r + B/r; FP32 and FP16-shifted storage stay within a
  velocity-field relative L2 of 1e-3 of FP64. BF16-shifted storage is not claimed to meet
  that bound: its rounding floor alone (8 mantissa bits) is above it, which one test
  records; another keeps its measured level as a regression check.
- A shear wave whose per-step change is below half a unit of the 16-bit storages decays
  as in FP64 (stochastic rounding keeps sub-unit increments).
- Single cylinder (Sec. 3.2), FP32: C_d and St close to Table (high-Re) / (low-Re) of
  the paper (plausibility only: domain and edges differ from the paper's).
- Precision sweep at the oracle's size (600x300, D = 30, Re = 200): mean C_d, C_l rms and
  St of FP64, FP32 and FP16-shifted storage within 1 % of the stored FP64 oracle values
  (BF16-shifted: measured level only, as for Couette).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from paper_1901_08766_gb300 import diagnostics as dg

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _couette_fields(lbm, storage, steps=20000):
    spec = synth.couette(steps=steps)
    dom = lbm.Domain(spec, storage=storage, force_every=0)
    dom.step(steps)
    rho, ux, uy = dom.moments()
    pops = dom.get_populations()
    dom.close()
    return spec, ux, uy, pops


def _utheta(ux, uy, n=128):
    c = n / 2.0
    j, i = np.mgrid[0:n, 0:n]
    x, y = i - c, j - c
    r = np.hypot(x, y)
    rr = np.where(r > 0, r, 1.0)
    return (-y * ux + x * uy) / rr, r


def test_couette_fp64_matches_oracle_and_closed_form(lbm):
    spec, ux, uy, pops = _couette_fields(lbm, "f64")
    ora = oracle.Domain(spec)
    ora.run(spec["steps"], want_forces=False)
    assert np.max(np.abs(pops - ora.g) / np.abs(ora.g)) <= 1e-10
    ut, r = _utheta(ux, uy)
    sel = (r >= 21) & (r <= 49)
    ri, ro, u0 = 20.0, 50.0, 0.01
    A = -u0 * ri / (ro ** 2 - ri ** 2)
    B = u0 * ri * ro ** 2 / (ro ** 2 - ri ** 2)
    exact = A * r + B / np.where(r > 0, r, 1.0)
    err = math.sqrt(((ut - exact)[sel] ** 2).sum() / (exact[sel] ** 2).sum())
    assert err < 0.03


def _couette_l2_vs_fp64(ux, uy, ux64, uy64):
    num = np.sqrt(((ux - ux64) ** 2 + (uy - uy64) ** 2).sum())
    den = np.sqrt((ux64 ** 2 + uy64 ** 2).sum())
    return num / den


@pytest.mark.parametrize("storage,steps", [("f32", 20000), ("f16s", 20000), ("f16s", 100000)])
def test_couette_reduced_precision_velocity_l2(lbm, storage, steps):
    # The bound: velocity-field relative L2 against FP64 storage <= 1e-3 after the 20 000
    # steps of the workload (FP32 1.4e-5, FP16-shifted 3.1e-4: stochastic rounding keeps
    # the spin-up's sub-unit increments that rounding to nearest dropped, 2.2e-3 then),
    # and FP16 once more at 100 000 steps.
    bound = 1e-3
    _, ux64, uy64, _ = _couette_fields(lbm, "f64", steps=20000)
    _, ux, uy, _ = _couette_fields(lbm, storage, steps=steps)
    num = np.sqrt(((ux - ux64) ** 2 + (uy - uy64) ** 2).sum())
    den = np.sqrt((ux64 ** 2 + uy64 ** 2).sum())
    print(f"{storage} after {steps} steps: velocity relative L2 vs FP64 = {num / den:.3e}")
    assert num / den <= bound


def test_couette_bf16s_rounding_floor_is_above_the_bound(lbm):
    # Why BF16-shifted storage is excluded from the 1e-3 Couette bound: started from the
    # converged FP64 state itself, it stays 2.6e-3 away from it (measured 2.56e-3): the
    # stochastic-rounding noise of 8-mantissa-bit values that carry the velocity is above
    # the bound whatever the path to the steady state (FP16-shifted, 11 bits: 3.2e-4).
    import codec
    spec, ux64, uy64, pops = _couette_fields(lbm, "f64")
    dom = lbm.Domain(spec, storage="bf16s", force_every=0)
    dom.set_populations(codec.encode(pops, "bf16s"))
    dom.step(20000)
    _, ux, uy = dom.moments()
    dom.close()
    floor = _couette_l2_vs_fp64(ux, uy, ux64, uy64)
    print(f"bf16s from the converged FP64 state, 20000 steps: velocity relative L2 {floor:.3e}")
    assert 1e-3 < floor < 5e-3


def test_couette_bf16s_measured_level(lbm):
    # Regression check of BF16-shifted storage (not a bound: see the test above): the
    # velocity-field relative L2 against FP64 after the workload's 20 000 steps, measured
    # 2.6e-3, stays below 5e-3.
    _, ux64, uy64, _ = _couette_fields(lbm, "f64", steps=20000)
    _, ux, uy, _ = _couette_fields(lbm, "bf16s", steps=20000)
    level = _couette_l2_vs_fp64(ux, uy, ux64, uy64)
    print(f"bf16s after 20000 steps: velocity relative L2 vs FP64 = {level:.3e}")
    assert level <= 5e-3


def test_couette_fp16s_rounding_floor(lbm):
    # Started from the converged FP64 state, FP16-shifted storage stays within 5e-4 of it:
    # the rounding floor of the stored steady state (measured 2.5e-4).
    import codec
    spec, ux64, uy64, pops = _couette_fields(lbm, "f64")
    dom = lbm.Domain(spec, storage="f16s", force_every=0)
    dom.set_populations(codec.encode(pops, "f16s"))
    dom.step(20000)
    _, ux, uy = dom.moments()
    dom.close()
    num = np.sqrt(((ux - ux64) ** 2 + (uy - uy64) ** 2).sum())
    den = np.sqrt((ux64 ** 2 + uy64 ** 2).sum())
    print(f"f16s from the converged FP64 state, 20000 steps: velocity relative L2 {num / den:.3e}")
    assert num / den <= 5e-4


@pytest.mark.parametrize("storage,tol", [("f16s", 0.02), ("bf16s", 0.05)])
def test_sub_unit_decay_not_frozen(lbm, storage, tol):
    # A shear wave u_x = A sin(2 pi y / n) in a periodic box decays by viscosity as
    # exp(-nu k^2 t). With A = 1e-3 its per-step change of a population (about 3e-8) is
    # far below half a unit of the 16-bit storage (about 1.2e-7 for FP16 at 3e-4):
    # rounded to nearest the wave would stay frozen; rounded stochastically it decays as
    # in FP64 storage (projected amplitude after 1/(nu k^2) steps, about 0.38 A).
    import codec
    n, A, nu, steps = 64, 1e-3, 0.01, 10000
    spec = synth._spec("shear", n, n, nu, [], [], steps, A, synth._edges())
    col = np.stack([oracle.equilibrium(1.0, A * math.sin(2 * math.pi * j / n), 0.0)
                    for j in range(n)], axis=1)  # [9, ny]
    g0 = np.repeat(col[:, :, None], n, axis=2)
    sinj = np.sin(2 * math.pi * np.arange(n) / n)[:, None]
    amp = {}
    for st in ("f64", storage):
        dom = lbm.Domain(spec, storage=st, force_every=0)
        dom.set_populations(codec.encode(g0, st))
        dom.step(steps)
        _, ux, _ = dom.moments()
        dom.close()
        amp[st] = 2.0 * (ux * sinj).mean()
    decay = math.exp(-nu * (2 * math.pi / n) ** 2 * steps)
    print(f"{storage}: amplitude {amp[storage]:.4e} vs FP64 {amp['f64']:.4e} (A e^(-nu k^2 t) = {A * decay:.4e})")
    assert abs(amp["f64"] - A * decay) / (A * decay) < 0.01
    assert abs(amp[storage] - amp["f64"]) / amp["f64"] < tol


@pytest.mark.parametrize("re,cd,st,steps", [(100.0, 1.336, 0.169, 120000), (40.0, 1.55, None, 60000)])
def test_single_cylinder_against_paper_tables(lbm, re, cd, st, steps):
    # Table (high-Re): Re 100 gives C_d 1.336, St 0.169; Table (low-Re): Re 40 gives C_d 1.55.
    # The domain (1600x800, free-slip walls) differs from the paper's 2048x1024: 10 % on
    # C_d and 5 % on St are plausibility bands.
    # centre offset half a cell in y: shedding starts from the geometry instead of
    # waiting for roundoff to break the symmetry of a centred cylinder
    spec = synth.single_cylinder(re=re, steps=steps, cy=400.5)
    dom = lbm.Domain(spec, storage="f32")
    f = dom.run(steps, chunk=8000)[:, 0]
    dom.close()
    s = dg.summary(f, spec["U"], spec["bodies"][0]["ref_length"], window=0.3)
    print(f"Re {re}: {s}")
    assert abs(s["cd_mean"] - cd) / cd < 0.10
    if st is not None:
        assert abs(s["st"] - st) / st < 0.05
    else:
        assert s["cl_rms"] < 0.01  # steady wake


def _precision_sweep(lbm, storage):
    path = os.path.join(GOLDEN, "precision_cylinder_600x300.json")
    ref = json.load(open(path))
    spec = synth.precision_cylinder(large=False)
    dom = lbm.Domain(spec, storage=storage)
    f = dom.run(spec["steps"], chunk=8000)[:, 0]
    dom.close()
    D, U = spec["bodies"][0]["ref_length"], spec["U"]
    cd, cl = dg.coefficients(f, U, D)
    half = slice(len(cd) // 2, len(cd))
    got = {"cd_mean": cd[half].mean(), "cl_rms": dg.rms(cl[half]),
           "st": dg.strouhal_spectral(cl[half], D, U)}
    print(storage, got, {k: ref[k] for k in got})
    return got, ref


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_precision_sweep_against_oracle(lbm, storage):
    # The bound: mean C_d, C_l rms and St (lift spectral peak) over steps 40 000..80 000
    # within 1 % of the stored FP64 oracle values.
    got, ref = _precision_sweep(lbm, storage)
    for k in got:
        assert abs(got[k] - ref[k]) / abs(ref[k]) < 0.01, k


def test_precision_sweep_bf16s_measured_level(lbm):
    # Regression check of BF16-shifted storage, which is not claimed to meet the 1 % bound
    # (measured: C_d +1.4 %, St +1.0 %, C_l rms -1.0 %): each within 3 %.
    got, ref = _precision_sweep(lbm, "bf16s")
    for k in got:
        assert abs(got[k] - ref[k]) / abs(ref[k]) < 0.03, k
