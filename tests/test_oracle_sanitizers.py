"""The oracle's C code under AddressSanitizer and UndefinedBehaviorSanitizer (host only):
copies of the 2D and 3D oracle libraries are built with -fsanitize=address,undefined and
loaded, in a child process with the sanitizer runtimes preloaded, in place of the plain
ones; the child runs every oracle entry point the tests use on small cases (fixed,
translating, turning, pulsating and coupled bodies; edge sets; moments; both 3D lattices).
Any out-of-bounds access, use after free or undefined operation aborts the child with a
report, which fails the test."""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = textwrap.dedent("""
    import sys
    sys.path[:0] = [{root!r}, {tests!r}]
    import numpy as np
    import oracle
    from oracle import d3
    oracle._LIB = {lib2!r}
    d3._LIB = {lib3!r}
    import synth

    # 2D: every parity case (edge sets, ragged sizes, both magic parameters), TRT and SRT
    for name in synth.PARITY_CASES:
        sp = synth.parity_case(name)
        dom = oracle.Domain(sp, g=synth.random_populations(3, sp["nx"], sp["ny"], 0.05))
        dom.run(12)
        dom.moments()
        dom.run(3, srt=True)
        dom.step_once()
    sp = synth.parity_case("channel_97x61")
    # translating, turning, pulsating bodies; a coupled body
    for moving in (True, 2):
        b0 = dict(sp["bodies"][0], vx=0.01, omega=0.004)
        b1 = dict(sp["bodies"][1], deform={{"amplitude": 0.1, "rate": 0.05}})
        oracle.Domain(dict(sp, moving=moving, bodies=[b0, b1])).run(15)
    dyn = {{"mass": 800.0, "stiffness": (0.0, 2.0), "damping": (0.0, 0.1), "free": (0, 1)}}
    oracle.Domain(dict(sp, moving=True, bodies=[dict(sp["bodies"][0], dynamics=dyn), sp["bodies"][1]])).run(15)
    for step in (None, 7):
        oracle.rasterize(dict(sp, moving=2), step)
    oracle.rasterize(synth.naca0012(5.0, 600.0, chord=40.0, nx=120, ny=60, steps=1))
    oracle.rasterize(synth.couette(n=48, r_inner=8.0, r_outer=20.0))

    # 3D: both lattices, a sphere channel and periodic bodies, moving and coupled bodies
    for q in (19, 15):
        c = (12.3, 8.4, 6.2)
        s3 = synth.spec3("san3", 30, 16, 12, 0.05, [synth.sphere(1, c, 3.1), synth.cylinder_z(2, 22.0, 8.0, 2.0)],
                         [synth.body3(c, 6.2), synth.body3((22.0, 8.0, 0.0), 4.0)], 0, 0.03,
                         synth.channel_edges3(), u_in=(0.03, 0.0, 0.0), u0=(0.03, 0.0, 0.0), lattice=q)
        d = d3.Domain(s3, g=synth.random_populations3(4, 30, 16, 12, 0.05, q=q))
        d.run(6)
        d.moments()
        mv = dict(s3, moving=True, bodies=[dict(b, v=(0.01, 0.002, -0.001)) for b in s3["bodies"]])
        d3.Domain(mv).run(6)
        dyn3 = {{"mass": 300.0, "stiffness": (0.0, 1.0, 1.0), "damping": (0.0, 0.0, 0.0), "free": (0, 1, 1)}}
        cp = dict(s3, moving=True, bodies=[dict(s3["bodies"][0], v=(0.0, 0.005, 0.0), dynamics=dyn3)],
                  shapes=s3["shapes"][:1])
        d3.Domain(cp).run(6)
    print("sanitized oracle runs clean")
""")


def _runtime(name):
    p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


def test_oracle_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("sanitizer runtimes not installed")
    flags = ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
             "-fno-sanitize-recover=undefined", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", "-std=c11", "-fopenmp"]
    libs = {}
    for key, src in (("2", "lbm_oracle.c"), ("3", "lbm_oracle3d.c")):
        out = str(tmp_path / f"liboracle{key}_san.so")
        subprocess.check_call(["gcc", *flags, "-o", out, os.path.join(ROOT, "oracle", src), "-lm"])
        libs[key] = out
    script = tmp_path / "child.py"
    script.write_text(CHILD.format(root=ROOT, tests=HERE, lib2=libs["2"], lib3=libs["3"]))
    env = dict(os.environ, LD_PRELOAD=f"{asan}:{ubsan}", OMP_NUM_THREADS="2",
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, str(script)], capture_output=True, text=True, env=env, timeout=600)
    report = r.stdout[-3000:] + r.stderr[-6000:]
    assert r.returncode == 0, report
    assert "sanitized oracle runs clean" in r.stdout, report
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, report
    # the harness itself reports a planted heap overflow read through the same route
    bad = tmp_path / "bad.c"
    bad.write_text("#include <stdlib.h>\n"
                   "double planted(int n) { double *a = malloc(sizeof(double) * n); "
                   "for (int i = 0; i < n; ++i) a[i] = i; double s = a[n]; free(a); return s; }\n")
    so = str(tmp_path / "libbad.so")
    subprocess.check_call(["gcc", *flags, "-o", so, str(bad)])
    probe = tmp_path / "probe.py"
    probe.write_text(f"import ctypes\nL = ctypes.CDLL({so!r})\nL.planted.restype = ctypes.c_double\n"
                     "print(L.planted(5))\n")
    r = subprocess.run([sys.executable, str(probe)], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode != 0 and ("heap-buffer-overflow" in r.stderr or "runtime error" in r.stderr), r.stderr[-2000:]
