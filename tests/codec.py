"""Test-side storage conversions: FP64 populations to and from the library's stored
types (F64, F32, F16S, BF16S), with the shift by w_alpha * rho0 for the 16-bit types and
the power-of-two scale F16S stores the shifted values with.

The shift weights come from the oracle's own constants. Encoding is the test's choice
of inputs (any stored values are valid); decoding is exact, so the oracle receives
exactly the state the GPU starts from.
"""
import numpy as np

import oracle

W = oracle.W[:, None, None]
_W3 = {}


def _weights(g):
    """Shift weights broadcast over populations [9, ny, nx] (D2Q9) or [q, nz, ny, nx]
    (D3Q19 or D3Q15, the 3D oracle's weights)."""
    q = np.shape(g)[0]
    if q == 9:
        return W
    if q not in _W3:
        from oracle import d3
        _W3[q] = d3.lattice(q)[3][:, None, None, None]
    return _W3[q]


F16_SCALE = 1024.0  # F16S stores F16_SCALE * (f - w rho0)


def f32_to_bf16_bits(x):
    """Round-to-nearest-even of float32 values to bfloat16, as uint16 bits."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def bf16_bits_to_f64(bits):
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def encode(g, storage, rho0=1.0):
    """FP64 populations [9, ny, nx] or [19, nz, ny, nx] -> stored array in the library's
    layout."""
    if storage == "f64":
        return np.ascontiguousarray(g, dtype=np.float64)
    if storage == "f32":
        return np.ascontiguousarray(g, dtype=np.float32)
    s = g - _weights(g) * rho0
    if storage == "f16s":
        return np.ascontiguousarray((s * F16_SCALE).astype(np.float32).astype(np.float16))
    if storage == "bf16s":
        return f32_to_bf16_bits(s.astype(np.float32))
    raise KeyError(storage)


def decode(raw, storage, rho0=1.0):
    """Stored array -> FP64 populations (exact)."""
    if storage in ("f64", "f32"):
        return np.asarray(raw, dtype=np.float64)
    if storage == "f16s":
        return np.asarray(raw, dtype=np.float16).astype(np.float64) / F16_SCALE + _weights(raw) * rho0
    if storage == "bf16s":
        return bf16_bits_to_f64(raw) + _weights(raw) * rho0
    raise KeyError(storage)


def stored_ulp(values_shifted, storage):
    """Spacing of the stored type at the given (shifted) magnitudes."""
    a = np.abs(np.asarray(values_shifted, dtype=np.float64))
    if storage == "f16s":
        return np.spacing((a * F16_SCALE).astype(np.float16)).astype(np.float64) / F16_SCALE
    if storage == "bf16s":
        e = np.floor(np.log2(np.maximum(a, 2.0 ** -126)))
        return 2.0 ** (e - 7)
    if storage == "f32":
        return np.spacing(a.astype(np.float32)).astype(np.float64)
    return np.spacing(a)


def ghost_ulp(spec, storage):
    """One unit of the stored type at the inlet ghost populations f^eq(rho0, u_in) (shifted
    for the 16-bit types): the library holds the ghost as the stored type would."""
    if "nz" in spec:
        from oracle import d3
        q = d3.nq(spec)
        g = d3.equilibrium(spec["rho0"], spec["u_in"], q)
        w = d3.lattice(q)[3]
    else:
        g = oracle.equilibrium(spec["rho0"], *spec["u_in"])
        w = oracle.W
    if storage in ("f16s", "bf16s"):
        g = g - w
    if storage == "f64":
        return 0.0
    return float(stored_ulp(g, storage).max())


def step_tol(want, storage, spec=None, arith=None):
    """Per-population bound for one step of a reduced storage against the oracle's FP64
    result `want` (populations [9, ny, nx] or [19, nz, ny, nx]) from the same decoded state.

    Every stored value is within one unit of the stored type of the FP64 result: FP32
    rounds to nearest (ties either way), the 16-bit storages round stochastically to
    one of the two neighbours; FP32 arithmetic adds `arith`. For the 16-bit storages the
    rest population is stored as the pulled mass minus the rounded moving (8 or 18)
    populations, so it also carries their rounding residuals: up to one unit of each.
    With an inlet, the library holds the ghost populations as the stored type would:
    one more unit of the ghost's magnitude at column 0 (and the 3 or 5 ghost values enter
    the rest population's pulled mass)."""
    shift = _weights(want) if storage != "f32" else 0.0
    n_in = 3 if np.shape(want)[0] == 9 else 5  # directions entering from x = -1 (D3Q19, D3Q15: 5)
    if arith is None:
        arith = 3e-7 if storage == "f32" else 2e-8
    g = 0.0
    if spec is not None and spec["edges"]["west"] == "inlet":
        g = ghost_ulp(spec, storage)
    mag = np.abs(want - shift)
    # units taken at the largest magnitude the rounded value can have (a value just
    # below a power of two may round into the next binade, whose unit is twice as large)
    ulp = stored_ulp(mag + arith + g, storage)
    tol = ulp + arith
    tol[..., 0] += g
    if storage in ("f16s", "bf16s"):
        carried = ulp[1:].sum(axis=0)
        carried[..., 0] += n_in * g
        ulp0 = stored_ulp(mag[0] + arith + carried, storage)
        tol[0] = ulp0 + carried + arith
    return tol
