"""The served path on the GPU: each request's result is the same alone and in the mix."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _requests():
    specs = [synth.counter_rotating_pair(1.2, nx=300, ny=150, D=20.0),
             synth.naca0012(7.0, 600.0, chord=60.0, nx=400, ny=200),
             synth.counter_rotating_pair(0.3, nx=320, ny=160, D=20.0),
             synth.naca0012(2.0, 900.0, chord=50.0, nx=360, ny=180)]
    steps = [400, 250, 330, 180]
    return specs, steps


@pytest.mark.parametrize("storage", ["f16s", "f32"])
def test_served_results_equal_alone(lbm, storage):
    from paper_1901_08766_gb300.server import Server
    specs, steps = _requests()
    # budget for about two requests at a time: later ones queue and join mid-run
    budget = int(1.6 * max(lbm.domain_bytes(s, storage, force_capacity=72) for s in specs))
    srv = Server(storage=storage, hbm_budget=budget, chunk_steps=64, graph_steps=16)
    futs = [srv.submit(s, nsteps=n, arrival=srv.clock() + 0.002 * i)
            for i, (s, n) in enumerate(zip(specs, steps))]
    srv.run_until_idle(timeout=300)
    assert srv.max_queue >= 1  # some request had to wait for memory
    for f, s, n in zip(futs, specs, steps):
        r = f.result()
        assert r.status == "ok" and r.steps == n
        alone = lbm.Domain(s, storage=storage)
        fa = alone.run(n)
        alone.close()
        assert np.array_equal(r.forces, fa)
    st = srv.stats()
    assert st["completed"] == 4 and st["glups"] > 0
    srv.backend.close()
