"""Write the stored oracle values used by the GPU physics tests. Calls only oracle/ and
synth/ (the FP64 CPU oracle on seeded inputs); run from the repository root:

    python tests/golden/make_golden.py precision

precision: the oracle-sized cylinder of the precision sweep (600x300, D = 30 at
(150, 150.5), Re = 200, U = 0.05, Lambda = 3/16, eta = 1e-4, free-slip channel, 80 000
steps); mean C_d, C_l rms and St (dominant spectral peak of C_l; zero crossings as a
secondary value) over the last half of the run (shedding is saturated from about 40k
steps), plus the force series decimated by 10 for reference.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def precision():
    spec = synth.precision_cylinder(large=False)
    dom = oracle.Domain(spec)
    t0 = time.time()
    forces = dom.run(spec["steps"])[:, 0]
    el = time.time() - t0
    D, U = spec["bodies"][0]["ref_length"], spec["U"]
    cd, cl = oracle.coefficients(forces, U, D)
    half = slice(len(cd) // 2, len(cd))
    out = {"spec": spec["name"], "steps": spec["steps"], "window": "last half",
           "cd_mean": float(cd[half].mean()), "cl_rms": oracle.rms(cl[half]),
           "cl_amp": 0.5 * float(cl[half].max() - cl[half].min()),
           "st": oracle.strouhal_fft(cl[half], D, U),
           "st_zero_crossing": oracle.strouhal(cl[half], D, U), "oracle_seconds": el,
           "cd_every10": cd[::10].tolist(), "cl_every10": cl[::10].tolist()}
    path = os.path.join(HERE, "precision_cylinder_600x300.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, {k: v for k, v in out.items() if not k.endswith("every10")})


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "precision"
    {"precision": precision}[what]()
