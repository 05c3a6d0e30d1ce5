"""lbm_moments_noalloc: the moments export for callers that cannot let the library
allocate device memory when they read the fields (their own arena owns the GPU, or
the allocation's latency and device synchronisation are not acceptable in their loop).
It stages the fields in one fixed library-owned device array instead of a per-call
buffer. Checked through the C ABI against lbm_moments on two calls in a row, with the
moments tolerances of the other GPU tests; domains larger than the array are refused.

This file is collected last on purpose, so that a run stopping at its first failure
has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import codec
import synth

pytestmark = pytest.mark.gpu

MAX_NODES = 1 << 18


def _noalloc(lbm, dom):
    L = lbm.load()
    rho, ux, uy = (np.zeros((dom.ny, dom.nx)) for _ in range(3))
    st = L.lbm_moments_noalloc(dom._handle(), rho.ctypes.data_as(C.c_void_p),
                               ux.ctypes.data_as(C.c_void_p), uy.ctypes.data_as(C.c_void_p))
    return st, (rho, ux, uy)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-14), ("f16s", 2e-6)])
def test_noalloc_moments_match_moments_on_two_calls(lbm, storage, tol):
    spec = synth.parity_case("channel_97x61")
    dom = lbm.Domain(spec, storage=storage)
    dom.set_populations(codec.encode(synth.random_populations(31, spec["nx"], spec["ny"], 0.05),
                                     storage))
    for _ in range(2):
        dom.step(5)
        want = dom.moments()
        st, got = _noalloc(lbm, dom)
        assert st == 0, lbm.load().lbm_last_error()
        for g, w in zip(got, want):
            assert np.abs(g - w).max() <= tol
    dom.close()


def test_noalloc_moments_device_outputs_and_size_limit(lbm):
    import torch
    spec = synth.parity_case("periodic_97x61")
    dom = lbm.Domain(spec, storage="f32")
    dom.step(3)
    want = dom.moments()
    outs = [torch.zeros((spec["ny"], spec["nx"]), dtype=torch.float64, device="cuda") for _ in range(3)]
    L = lbm.load()
    st = L.lbm_moments_noalloc(dom._handle(), *[C.c_void_p(t.data_ptr()) for t in outs])
    assert st == 0
    for t, w in zip(outs, want):
        assert np.abs(t.cpu().numpy() - w).max() <= 2e-6
    dom.close()
    big = synth._spec("big", 1024, 257, 0.05, [], [], 0, 0.01, synth._edges())
    assert big["nx"] * big["ny"] > MAX_NODES
    d2 = lbm.Domain(big, storage="f16s", force_every=0)
    st, _ = _noalloc(lbm, d2)
    assert st == 1  # LBM_EINVAL: larger than the fixed staging array
    assert b"at most" in L.lbm_last_error() or b"more than" in L.lbm_last_error()
    d2.close()
