"""lbm_moments_noalloc: the moments export for callers that cannot let the library
allocate device memory when they read the fields (their own arena owns the GPU, or
the allocation's latency and device synchronisation are not acceptable in their loop).
It stages the fields in one fixed library-owned device array instead of a per-call
buffer. Checked through the C ABI against lbm_moments on two calls in a row: both run
the same kernel on the same stream, so the outputs must agree bit for bit. Between
the compared calls a domain of another size uses the shared array, and the first call
on a fresh domain must not change the device's free memory (the array was resolved
when the domain was created). Domains larger than the array are refused.

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


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
def test_noalloc_moments_match_moments_on_two_calls(lbm, storage):
    import torch
    spec = synth.parity_case("channel_97x61")
    dom = lbm.Domain(spec, storage=storage)
    dom.set_populations(codec.encode(synth.random_populations(31, spec["nx"], spec["ny"], 0.05),
                                     storage))
    # a second domain of another size shares the staging array between the compared calls
    other = synth._spec("other", 203, 131, 0.05, [], [], 0, 0.01, synth._edges())
    dom2 = lbm.Domain(other, storage=storage, force_every=0)
    dom2.step(2)
    for call in range(2):
        dom.step(5)
        want = dom.moments()  # also loads the moments kernel before the first measurement
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        st, got = _noalloc(lbm, dom)
        free1, _ = torch.cuda.mem_get_info()
        assert st == 0, lbm.load().lbm_last_error()
        assert free1 == free0, f"device memory changed by {free0 - free1} bytes"
        for g, w in zip(got, want):
            assert np.array_equal(g, w)
        st2, got2 = _noalloc(lbm, dom2)
        assert st2 == 0, lbm.load().lbm_last_error()
        for g, w in zip(got2, dom2.moments()):
            assert np.array_equal(g, w)
        # the first domain again after the other one used the array
        st, again = _noalloc(lbm, dom)
        assert st == 0
        for g, w in zip(again, want):
            assert np.array_equal(g, w)
    dom2.close()
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
        assert np.array_equal(t.cpu().numpy(), w)
    dom.close()
    big = synth._spec("big", 1024, 257, 0.05, [], [], 0, 0.01, synth._edges())
    assert big["nx"] * big["ny"] > MAX_NODES
    d2 = lbm.Domain(big, storage="f16s", force_every=0)
    st, _ = _noalloc(lbm, d2)
    assert st == 1  # LBM_EINVAL: larger than the fixed staging array
    assert b"at most" in L.lbm_last_error() or b"more than" in L.lbm_last_error()
    d2.close()
