"""Test-side storage conversions: FP64 populations to and from the library's stored
types (F64, F32, F16S, BF16S), with the shift by w_alpha * rho0 for the 16-bit types.

The shift weights come from the oracle's own constants. Encoding is the test's choice
of inputs (any stored values are valid); decoding is exact, so the oracle receives
exactly the state the GPU starts from.
"""
import numpy as np

import oracle

W = oracle.W[:, None, None]


def f32_to_bf16_bits(x):
    """Round-to-nearest-even of float32 values to bfloat16, as uint16 bits."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def bf16_bits_to_f64(bits):
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def encode(g, storage, rho0=1.0):
    """FP64 populations [9, ny, nx] -> stored array in the library's layout."""
    if storage == "f64":
        return np.ascontiguousarray(g, dtype=np.float64)
    if storage == "f32":
        return np.ascontiguousarray(g, dtype=np.float32)
    s = g - W * rho0
    if storage == "f16s":
        return np.ascontiguousarray(s.astype(np.float32).astype(np.float16))
    if storage == "bf16s":
        return f32_to_bf16_bits(s.astype(np.float32))
    raise KeyError(storage)


def decode(raw, storage, rho0=1.0):
    """Stored array -> FP64 populations (exact)."""
    if storage in ("f64", "f32"):
        return np.asarray(raw, dtype=np.float64)
    if storage == "f16s":
        return np.asarray(raw, dtype=np.float16).astype(np.float64) + W * rho0
    if storage == "bf16s":
        return bf16_bits_to_f64(raw) + W * rho0
    raise KeyError(storage)


def stored_ulp(values_shifted, storage):
    """Spacing of the stored type at the given (shifted) magnitudes."""
    a = np.abs(np.asarray(values_shifted, dtype=np.float64))
    if storage == "f16s":
        return np.spacing(a.astype(np.float16)).astype(np.float64)
    if storage == "bf16s":
        e = np.floor(np.log2(np.maximum(a, 2.0 ** -126)))
        return 2.0 ** (e - 7)
    if storage == "f32":
        return np.spacing(a.astype(np.float32)).astype(np.float64)
    return np.spacing(a)


def ghost_ulp(spec, storage):
    """One unit of the stored type at the inlet ghost populations f^eq(rho0, u_in) (shifted
    for the 16-bit types): the library holds the ghost as the stored type would."""
    g = oracle.equilibrium(spec["rho0"], *spec["u_in"])
    if storage in ("f16s", "bf16s"):
        g = g - oracle.W
    if storage == "f64":
        return 0.0
    return float(stored_ulp(g, storage).max())


def step_tol(want, storage, spec=None, arith=None):
    """Per-population bound for one step of a reduced storage against the oracle's FP64
    result `want` (populations [9, ny, nx]) from the same decoded state.

    Every stored value is within one unit of the stored type of the FP64 result (ties can
    round either way; FP32 arithmetic adds `arith`). For the 16-bit storages the rest
    population is stored as the pulled mass minus the eight rounded moving populations,
    so it also carries their rounding residuals: half a unit of each. With an inlet, the
    library holds the ghost populations as the stored type would: one more unit of the
    ghost's magnitude at column 0 (three such units for the rest population, whose pulled
    mass includes the three ghost values)."""
    shift = W if storage != "f32" else 0.0
    ulp = stored_ulp(want - shift, storage)
    if arith is None:
        arith = 3e-7 if storage == "f32" else 2e-8
    tol = ulp + arith
    if storage in ("f16s", "bf16s"):
        tol[0] += 0.5 * ulp[1:].sum(axis=0)
    if spec is not None and spec["edges"]["west"] == "inlet":
        g = ghost_ulp(spec, storage)
        tol[:, :, 0] += g
        if storage in ("f16s", "bf16s"):
            tol[0, :, 0] += 2 * g + 0.5 * 3 * g
    return tol
