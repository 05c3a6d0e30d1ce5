"""Product-side force diagnostics (paper_1901_08766_gb300.diagnostics) against the
oracle's estimators and closed forms (Sec. 3: C_d, C_l, St)."""
import math

import numpy as np
import pytest

import oracle
from paper_1901_08766_gb300 import diagnostics as dg


def _series(periods=6, D=40.0, U=0.05, st=0.169, cd=1.33, amp_d=0.008, amp_l=0.3, seed=0):
    rng = np.random.default_rng(seed)
    f = st * U / D
    n = int(round(periods / f))  # whole periods, so that the rms is unbiased
    t = np.arange(n)
    cdv = cd + amp_d * np.sin(4 * math.pi * f * t) + 1e-4 * rng.standard_normal(n)
    clv = amp_l * np.sin(2 * math.pi * f * t + 0.7) + 1e-4 * rng.standard_normal(n)
    q = 0.5 * U * U * D
    return np.stack([cdv * q, clv * q], -1), D, U


def test_coefficients_and_summary_closed_form():
    forces, D, U = _series()
    cd, cl = dg.coefficients(forces, U, D)
    s = dg.summary(forces, U, D, window=1.0)
    assert s["cd_mean"] == pytest.approx(1.33, abs=1e-3)
    assert s["cl_rms"] == pytest.approx(0.3 / math.sqrt(2), rel=2e-3)
    assert s["cl_amp"] == pytest.approx(0.3, rel=5e-3)
    assert s["st"] == pytest.approx(0.169, rel=3e-3)
    assert s["st_zero_crossing"] == pytest.approx(0.169, rel=1e-3)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_matches_oracle_estimators(seed):
    forces, D, U = _series(seed=seed, st=0.15 + 0.02 * seed)
    cd_p, cl_p = dg.coefficients(forces, U, D)
    cd_o, cl_o = oracle.coefficients(forces, U, D)
    assert np.allclose(cd_p, cd_o, rtol=1e-15) and np.allclose(cl_p, cl_o, rtol=1e-15)
    assert dg.strouhal(cl_p, D, U) == pytest.approx(oracle.strouhal(cl_o, D, U), rel=1e-12)
    assert dg.rms(cl_p) == pytest.approx(oracle.rms(cl_o), rel=1e-12)
    assert dg.strouhal_spectral(cl_p, D, U) == pytest.approx(oracle.strouhal_fft(cl_o, D, U), rel=1e-12)


def test_steady_signal_has_no_shedding():
    assert dg.strouhal(np.full(1000, 1.55), 40.0, 0.05) == 0.0
