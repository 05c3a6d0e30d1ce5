"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
function include/lbm.h declares, validates parameters before touching CUDA, and fails
loudly (no CPU fallback) when no device is present or the library is missing."""
import ctypes as C
import os
import re

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^LBM_API [^(]*?\b(lbm3?_\w+)\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import paper_1901_08766_gb300 as pkg
    pkg.build()
    return pkg


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = _declared()
    assert len(names) >= 28
    L = lib.load()
    for n in names:
        assert hasattr(L, n), f"{n} declared in lbm.h but not exported"
    from paper_1901_08766_gb300 import _native
    assert sorted(_native.SIGNATURES) == names
    # only the ABI is exported
    out = os.popen(f"nm -D --defined-only {_native.library_path()}").read()
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == set(names)


def test_status_strings_and_defaults(lib):
    from paper_1901_08766_gb300 import _native
    L = lib.load()
    assert L.lbm_status_string(0) == b"ok"
    assert L.lbm_status_string(4) == b"simulation diverged"
    p = _native.Params()
    L.lbm_params_default(C.byref(p))
    assert (p.nx, p.ny, p.storage, p.force_every, p.force_capacity) == (64, 64, 1, 1, 8192)
    assert p.magic_lambda == 3 / 16 and p.eta == 1e-4 and p.rho0 == 1.0


def test_domain_bytes(lib):
    spec = synth.parity_case("channel_97x61")
    b16 = lib.domain_bytes(spec, "f16s")
    b64 = lib.domain_bytes(spec, "f64")
    pitch = 128  # 97 rounded up to 64
    lat16 = 9 * 61 * pitch * 2
    assert b16 >= 2 * lat16 + 61 * pitch + 8192 * 2 * 2 * 8
    # populations 8 vs 2 bytes (x2 lattices), F_VP fields (one per lattice parity) 16 vs
    # 8 bytes per node
    assert b64 - b16 == pytest.approx(2 * 9 * 61 * pitch * 6 + 2 * 61 * pitch * 8, abs=1024)


BAD = [
    ("nx", 2), ("ny", 1), ("nu", -1.0), ("magic_lambda", 0.0), ("eta", 0.0), ("rho0", -1.0),
    ("west", 2), ("east", 1), ("south", 1), ("north", 2), ("storage", 9), ("force_every", -1),
    ("moving", 3), ("moving", -1),
]


@pytest.mark.parametrize("field,value", BAD)
def test_invalid_parameters_rejected_before_cuda(lib, field, value):
    from paper_1901_08766_gb300 import _native
    L = lib.load()
    spec = synth.parity_case("periodic_97x61")
    p = _native.params_from_spec(spec, "f32")
    setattr(p, field, value)
    if field == "nu":
        p.tau_plus = 0.4
    bodies, nb = _native.bodies_from_spec(spec)
    geom, _ = _native.geometry_from_spec(spec)
    h = C.c_void_p()
    st = L.lbm_domain_create(C.byref(p), None, C.byref(geom), bodies, nb, None,
                             _native.ALLOC_FN(), _native.FREE_FN(), None, C.byref(h))
    assert st == 1, L.lbm_last_error()
    assert h.value is None
    assert len(L.lbm_last_error()) > 0


def test_mixed_periodic_axis_rejected(lib):
    from paper_1901_08766_gb300 import _native
    L = lib.load()
    spec = synth.parity_case("periodic_97x61")
    p = _native.params_from_spec(spec, "f32")
    p.west = 1  # inlet with a periodic east edge
    h = C.c_void_p()
    st = L.lbm_domain_create(C.byref(p), None, None, None, 0, None, _native.ALLOC_FN(),
                             _native.FREE_FN(), None, C.byref(h))
    assert st == 1 and b"both periodic" in L.lbm_last_error()


def test_no_cpu_fallback(lib):
    import torch
    from paper_1901_08766_gb300 import _native
    L = lib.load()
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    spec = synth.parity_case("periodic_97x61")
    p = _native.params_from_spec(spec, "f32")
    bodies, nb = _native.bodies_from_spec(spec)
    geom, _ = _native.geometry_from_spec(spec)
    h = C.c_void_p()
    st = L.lbm_domain_create(C.byref(p), None, C.byref(geom), bodies, nb, None,
                             _native.ALLOC_FN(), _native.FREE_FN(), None, C.byref(h))
    assert st == 3  # LBM_ECUDA: there is no CPU path
    with pytest.raises(RuntimeError):
        _native.load.__wrapped__ if hasattr(_native.load, "__wrapped__") else None
        saved = _native._lib
        try:
            _native._lib = None
            _native.load(os.path.join(ROOT, "does_not_exist.so"))
        finally:
            _native._lib = saved


# ---- 3D (D3Q19) ABI ---------------------------------------------------------------------

def _sphere_spec3():
    return synth.spec3("sphere_40x24x20", 40, 24, 20, 0.05, [synth.sphere(1, (12.3, 11.6, 9.7), 4.2)],
                       [synth.body3((12.3, 11.6, 9.7), 8.4)], 10, 0.05, synth.channel_edges3(),
                       u_in=(0.05, 0.0, 0.0), u0=(0.05, 0.0, 0.0))


def test_params3_default_and_bytes(lib):
    from paper_1901_08766_gb300 import _native
    L = lib.load()
    p = _native.Params3()
    L.lbm3_params_default(C.byref(p))
    assert (p.nx, p.ny, p.nz, p.storage, p.force_every, p.force_capacity, p.lattice) == (32, 32, 32, 1, 1, 8192, 19)
    assert p.magic_lambda == 3 / 16 and p.eta == 1e-4 and p.rho0 == 1.0 and p.nu == 0.1
    spec = _sphere_spec3()
    sizes = {}
    for st in ("f64", "f32", "f16s"):
        q = _native.params3_from_spec(spec, st)
        sizes[st] = L.lbm3_domain_bytes(C.byref(q), 1)
    pitch, nodes = 64, 24 * 20
    lat = {st: 2 * 19 * nodes * pitch * e for st, e in (("f64", 8), ("f32", 4), ("f16s", 2))}
    for st in sizes:
        assert sizes[st] >= lat[st] + nodes * pitch + 8192 * 3 * 8
    # lattices x2 and the F_VP field (3 doubles vs 3 floats per node) differ
    assert sizes["f64"] - sizes["f16s"] == pytest.approx(lat["f64"] - lat["f16s"] + nodes * pitch * 12,
                                                         abs=2048)


BAD3 = [("nz", 2), ("nx", 1), ("nu", -1.0), ("eta", 0.0), ("bottom", 1), ("top", 2),
        ("south", 2), ("storage", 7), ("force_capacity", -1), ("lattice", 7),
        ("moving", 2)]  # shapes turned with their body: 2D only


@pytest.mark.parametrize("field,value", BAD3)
def test_invalid_3d_parameters_rejected_before_cuda(lib, field, value):
    from paper_1901_08766_gb300 import _native
    L = lib.load()
    spec = _sphere_spec3()
    p = _native.params3_from_spec(spec, "f32")
    setattr(p, field, value)
    if field == "nu":
        p.tau_plus = 0.4
    shapes, ns = _native.shapes3_from_spec(spec)
    bodies, nb = _native.bodies3_from_spec(spec)
    h = C.c_void_p()
    st = L.lbm3_domain_create(C.byref(p), shapes, ns, bodies, nb, None, _native.ALLOC_FN(),
                              _native.FREE_FN(), None, C.byref(h))
    assert st == 1, L.lbm_last_error()
    assert h.value is None and len(L.lbm_last_error()) > 0


def test_3d_shape_body_ids_checked(lib):
    from paper_1901_08766_gb300 import _native
    L = lib.load()
    spec = _sphere_spec3()
    spec["shapes"][0]["body"] = 2  # only one body
    p = _native.params3_from_spec(spec, "f32")
    shapes, ns = _native.shapes3_from_spec(spec)
    bodies, nb = _native.bodies3_from_spec(spec)
    h = C.c_void_p()
    st = L.lbm3_domain_create(C.byref(p), shapes, ns, bodies, nb, None, _native.ALLOC_FN(),
                              _native.FREE_FN(), None, C.byref(h))
    assert st == 1 and b"body id" in L.lbm_last_error()


def test_3d_no_cpu_fallback(lib):
    import torch
    from paper_1901_08766_gb300 import _native
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = lib.load()
    spec = _sphere_spec3()
    p = _native.params3_from_spec(spec, "f32")
    shapes, ns = _native.shapes3_from_spec(spec)
    bodies, nb = _native.bodies3_from_spec(spec)
    h = C.c_void_p()
    st = L.lbm3_domain_create(C.byref(p), shapes, ns, bodies, nb, None, _native.ALLOC_FN(),
                              _native.FREE_FN(), None, C.byref(h))
    assert st == 3 and h.value is None


@pytest.mark.parametrize("args", [
    (0, 0, 2, 19),      # no slots
    (5000, 0, 2, 19),   # too many slots
    (4, 0, 9, 19),      # unknown storage
    (4, 0, 2, 17),      # unknown lattice
])
def test_3d_batch_arguments_rejected_before_cuda(lib, args):
    from paper_1901_08766_gb300 import _native
    L = lib.load()
    h = C.c_void_p()
    st = L.lbm3_batch_create(*args, None, _native.ALLOC_FN(), _native.FREE_FN(), None, C.byref(h))
    assert st == 1 and h.value is None
    # NULL handles are rejected, destroy(NULL) is a no-op
    n = C.c_int64()
    assert L.lbm3_batch_run(None, 1, C.byref(n)) == 1
    assert L.lbm3_batch_evict(None, 0) == 1
    assert L.lbm3_batch_destroy(None) == 0


def test_3d_batch_no_cpu_fallback(lib):
    import torch
    from paper_1901_08766_gb300 import _native
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = lib.load()
    h = C.c_void_p()
    st = L.lbm3_batch_create(4, 0, 2, 19, None, _native.ALLOC_FN(), _native.FREE_FN(), None, C.byref(h))
    assert st == 3 and h.value is None


def test_batch_null_handles_rejected(lib):
    # the 2D batch's setters and drains reject a NULL batch before touching CUDA
    L = lib.load()
    assert L.lbm_batch_set_grouped_admission(None, 1) == 1
    assert L.lbm_batch_set_tile(None, 8, 12, 4, 4) == 1
    n = C.c_int64()
    assert L.lbm_batch_run(None, 1, C.byref(n)) == 1
    assert L.lbm_batch_pack_halos(None) == 1
