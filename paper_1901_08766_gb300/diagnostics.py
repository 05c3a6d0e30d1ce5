"""Force coefficients and shedding frequency from body-force series (Sec. 3).

C_d = 2 F_x / (rho U^2 D), C_l = 2 F_y / (rho U^2 D); St = f_q D / U with the shedding
frequency from the upward zero crossings of (signal - mean), interpolated linearly and
averaged over the whole periods between the first and the last crossing. The "C_l +- a"
amplitude is half the peak-to-peak value; the rms is that of signal - mean.
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


def rms(signal) -> float:
    x = np.asarray(signal, dtype=np.float64)
    return float(np.sqrt(np.mean(np.square(x - x.mean()))))


def amplitude(signal) -> float:
    x = np.asarray(signal, dtype=np.float64)
    return 0.5 * float(x.max() - x.min())


def summary(forces, U: float, ref_length: float, rho0: float = 1.0, window: float = 0.5):
    """Mean C_d, C_l rms and amplitude, and St (from C_l, else C_d) over the last
    `window` fraction of the series."""
    cd, cl = coefficients(forces, U, ref_length, rho0)
    n = len(cd)
    s = slice(int(n * (1.0 - window)), n)
    cdw, clw = cd[s], cl[s]
    st = strouhal(clw, ref_length, U)
    if st == 0.0:
        st = strouhal(cdw, ref_length, U)
    return {"cd_mean": float(cdw.mean()) if len(cdw) else 0.0, "cl_rms": rms(clw) if len(clw) else 0.0,
            "cd_amp": amplitude(cdw) if len(cdw) else 0.0, "cl_amp": amplitude(clw) if len(clw) else 0.0,
            "st": st}
