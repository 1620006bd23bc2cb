"""Serving: concurrent requests of mixed spaces, degrees and meshes give the same
result as each request solved alone (deterministic kernels, independent handles),
match the oracle, overlap on the GPU, and stay within the HBM budget measured by
the device itself."""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import assemble as asm
from oracle.mesh import MeshDofs
from oracle.refelem import reference_element
from paper_2506_17406_gb300 import riesz as rz
from paper_2506_17406_gb300 import serve
from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_vector


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


def test_served_results_match_the_oracle():
    """Requests of every space, first and second kind (FP32 patch sweeps, FP64 residuals, the paper's
    decomposition per space), served concurrently, each solved to rtol 1e-11, against the oracle's sparse
    direct solve of the same mesh and right-hand side: 1e-8 relative L2 (the mixed path's accuracy target)."""
    reqs = serve.poisson_stream(6, rate=1000.0, seed=11, degrees=(2, 3, 4), sizes=(2, 3))
    # and the second-kind spaces, with the paper's decompositions
    reqs += serve.poisson_stream(4, rate=1000.0, seed=12, spaces=("N2curl", "BDM"), degrees=(2, 3), sizes=(2,))
    for i, r in enumerate(reqs):
        r.rtol = 1e-11
        r.rid = i
    done = serve.Server(hbm_budget_bytes=8 << 30, max_slots=6, recommended=True).run(reqs, realtime=True)
    for r in done:
        assert r.status == 0, r
        verts, cells = kuhn_mesh(r.n, r.amp, r.seed % 1000)
        ref = reference_element(r.space, r.p)
        md = MeshDofs(verts, cells, ref)
        A = asm.assemble(md, asm.element_matrices(ref, verts, cells))
        b = normal_vector(md.ndofs, r.seed % 7919)
        xe = asm.direct_solve(A, b)
        assert np.linalg.norm(r.x - xe) <= 1e-8 * np.linalg.norm(xe), (r.space, r.p, r.n)


def test_requests_overlap_on_the_gpu():
    """A burst of requests with several slots: the GPU spans (CUDA events on each request's own stream,
    from the start of its device setup to the end of its solve) of at least two requests intersect."""
    reqs = serve.poisson_stream(6, rate=5000.0, seed=3, degrees=(4, 5), sizes=(4,))
    done = serve.Server(hbm_budget_bytes=16 << 30, max_slots=4).run(reqs, realtime=True)
    assert all(r.status == 0 for r in done)
    spans = sorted(r.gpu_span for r in done)
    assert all(a < b for a, b in spans)
    overlaps = sum(1 for i in range(len(spans)) for j in range(i + 1, len(spans))
                   if spans[j][0] < spans[i][1] and spans[i][0] < spans[j][1])
    assert overlaps >= 1, spans


@pytest.mark.parametrize("space,p,kw", [("CG", 3, {}), ("N1curl", 3, dict(precond_precision=rz.PREC_FP32, nrhs_max=3)),
                                        ("RT", 3, dict(apply_precision=rz.PREC_FP32, dirichlet=1)),
                                        ("N1curl", 2, dict(decomposition=rz.DECOMP_HT)),
                                        ("RT", 4, dict(decomposition=rz.DECOMP_EDGE_STAR, coarse=0)),
                                        ("N1curl", 3, dict(alpha=1e3)),
                                        ("CG", 4, dict(apply_mode=rz.APPLY_MATRIX_FREE))])
def test_planned_bytes_are_the_device_footprint(space, p, kw):
    """riesz_plan_bytes (host-only) equals the bytes the device setup holds, buffer for buffer, and the
    admission estimate (planned bytes + one allocator page per allocation) bounds the drop of the
    device's free memory (cudaMemGetInfo) across the setup."""
    verts, cells = kuhn_mesh(4, 0.1, 2)
    # a first handle of the same shape loads the kernels it launches (lazy module loading and the
    # local-memory reservation of those kernels are the runtime's, not the handle's)
    rz.Riesz(space, p, verts, cells, **kw).close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    h = rz.Riesz(space, p, verts, cells, device=False, **kw)
    planned, nalloc = h.plan_bytes()
    est = serve.estimate_footprint(h)
    free0, _ = torch.cuda.mem_get_info()
    h.setup_device()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert h.stats()["device_bytes"] == planned
    assert free0 - free1 <= est, (free0 - free1, est)
    h.close()


def test_admission_respects_the_budget():
    """With a budget for one request at a time, the free device memory (cudaMemGetInfo), sampled while
    every request runs, never drops below the start value minus the budget."""
    reqs = serve.poisson_stream(4, rate=1000.0, seed=9, degrees=(3,), sizes=(4,))
    fps = []
    for r in reqs:
        h, fp = serve.Server()._prepare(r)
        fps.append(fp)
        h.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0, _ = torch.cuda.mem_get_info()
    srv = serve.Server(hbm_budget_bytes=int(max(fps) * 1.5), max_slots=4)
    low = {"v": free0}
    orig_setup = rz.Riesz.setup_device

    def setup_and_sample(self, stream=None):
        orig_setup(self, stream)
        torch.cuda.synchronize()
        with srv.lock:
            low["v"] = min(low["v"], torch.cuda.mem_get_info()[0])
    rz.Riesz.setup_device = setup_and_sample
    try:
        done = srv.run(reqs, realtime=False)
    finally:
        rz.Riesz.setup_device = orig_setup
    assert all(r.status == 0 for r in done)
    # the requests' own torch tensors (right-hand side, solution) are a few MB on top of the library's
    assert free0 - low["v"] <= srv.budget + (64 << 20), (free0 - low["v"], srv.budget)
