"""Force coefficients and shedding frequency from body-force series (Sec. 3).

C_d = 2 F_x / (rho U^2 D), C_l = 2 F_y / (rho U^2 D); St = f_q D / U with the shedding
frequency f_q taken from the dominant peak of the lift spectrum (primary: a channel with
an equilibrium inlet and a zero-gradient outflow carries an acoustic standing wave that
adds zero crossings) or from the upward zero crossings of (signal - mean), interpolated
linearly over whole periods (secondary). The "C_l +- a" amplitude is half the
peak-to-peak value; the rms is that of signal - mean.
"""
from __future__ import annotations

import numpy as np


def coefficients(forces, U: float, ref_length: float, rho0: float = 1.0):
    """(C_d, C_l) series of one body from its force series [n, 2]."""
    f = np.asarray(forces, dtype=np.float64).reshape(-1, 2)
    scale = 2.0 / (rho0 * U * U * ref_length)
    return scale * f[:, 0], scale * f[:, 1]


def upward_crossings(signal, dt: float = 1.0) -> np.ndarray:
    """Times at which signal - mean crosses zero from below (linear interpolation)."""
    x = np.asarray(signal, dtype=np.float64)
    x = x - x.mean()
    lo, hi = x[:-1], x[1:]
    idx = np.nonzero((lo < 0.0) & (hi >= 0.0))[0]
    frac = -lo[idx] / (hi[idx] - lo[idx])
    return (idx + frac) * dt


def strouhal(signal, ref_length: float, U: float, dt: float = 1.0) -> float:
    t = upward_crossings(signal, dt)
    if len(t) < 2:
        return 0.0
    return (len(t) - 1) / (t[-1] - t[0]) * ref_length / U


def strouhal_spectral(signal, ref_length: float, U: float, dt: float = 1.0) -> float:
    """St from the dominant spectral peak: Hann window over (signal - mean), real FFT,
    the largest non-constant bin refined by the vertex of the parabola through the
    logarithms of its amplitude and its neighbours'. Robust to a weaker second tone."""
    x = np.asarray(signal, dtype=np.float64)
    n = x.size
    if n < 8:
        return 0.0
    w = np.hanning(n + 1)[:-1]  # periodic Hann window
    spec = np.abs(np.fft.rfft((x - x.mean()) * w))
    k = int(np.argmax(spec[1:-1])) + 1
    lm, l0, lp = np.log(np.maximum(spec[k - 1:k + 2], 1e-300))
    curv = lm - 2.0 * l0 + lp
    delta = 0.5 * (lm - lp) / curv if curv != 0.0 else 0.0
    return (k + delta) / (n * dt) * ref_length / U


def rms(signal) -> float:
    x = np.asarray(signal, dtype=np.float64)
    return float(np.sqrt(np.mean(np.square(x - x.mean()))))


def amplitude(signal) -> float:
    x = np.asarray(signal, dtype=np.float64)
    return 0.5 * float(x.max() - x.min())


def summary(forces, U: float, ref_length: float, rho0: float = 1.0, window: float = 0.5):
    """Mean C_d, C_l rms and amplitudes, and St of the lift (spectral peak, and from
    zero crossings), over the last `window` fraction of the series; St = 0 for a
    steady wake."""
    cd, cl = coefficients(forces, U, ref_length, rho0)
    n = len(cd)
    s = slice(int(n * (1.0 - window)), n)
    cdw, clw = cd[s], cl[s]
    steady = len(clw) == 0 or amplitude(clw) < 1e-6
    st = 0.0 if steady else strouhal_spectral(clw, ref_length, U)
    st_zc = 0.0 if steady else strouhal(clw, ref_length, U)
    return {"cd_mean": float(cdw.mean()) if len(cdw) else 0.0, "cl_rms": rms(clw) if len(clw) else 0.0,
            "cd_amp": amplitude(cdw) if len(cdw) else 0.0, "cl_amp": amplitude(clw) if len(clw) else 0.0,
            "st": st, "st_zero_crossing": st_zc}
