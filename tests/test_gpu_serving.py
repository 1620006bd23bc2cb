"""Serving: concurrent requests of mixed spaces, degrees and meshes give the same
result as each request solved alone (deterministic kernels, independent handles)."""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_17406_gb300 import serve


def test_results_identical_alone_and_in_the_mix():
    reqs = serve.poisson_stream(8, rate=200.0, seed=5, degrees=(2, 3, 4), sizes=(3, 4))
    mix = serve.Server(hbm_budget_bytes=8 << 30, max_slots=4)
    done = mix.run(copy.deepcopy(reqs), realtime=True)
    st = serve.summary(done, mix.wall)
    assert st["completed"] == len(reqs)
    alone = serve.Server(hbm_budget_bytes=8 << 30, max_slots=1)
    for r_mix, r in zip(sorted(done, key=lambda r: r.rid), reqs):
        solo = alone.run([copy.deepcopy(r)], realtime=False)[0]
        assert r_mix.status == 0 and solo.status == 0
        assert r_mix.relres <= 1e-8 and solo.relres <= 1e-8
        assert r_mix.iters == solo.iters
        assert np.array_equal(r_mix.x, solo.x)
    assert st["latency_p99_s"] >= st["latency_p50_s"] > 0


def test_admission_respects_the_budget():
    reqs = serve.poisson_stream(4, rate=1000.0, seed=9, degrees=(3,), sizes=(4,))
    fps = []
    for r in reqs:
        h, fp = serve.Server()._prepare(r)
        fps.append(fp)
        h.close()
    # budget for exactly one request at a time
    srv = serve.Server(hbm_budget_bytes=int(max(fps) * 1.5), max_slots=4)
    peak = {"v": 0}
    orig = srv._run

    def watched(req, h, t0):
        with srv.lock:
            peak["v"] = max(peak["v"], srv.in_use)
        orig(req, h, t0)
    srv._run = watched
    done = srv.run(reqs, realtime=False)
    assert all(r.status == 0 for r in done)
    assert peak["v"] <= srv.budget
