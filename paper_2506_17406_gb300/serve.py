"""Continuous-batching server for Riesz-map solves.

Requests (space, degree, mesh, right-hand side) arrive over time; each gets
its own host thread at arrival, which builds the request's host maps (in
parallel with other arrivals), waits until a slot is free and its device
footprint fits the HBM budget, then sets up and solves on its own CUDA stream
(the C calls release the GIL), so the kernels of concurrent requests overlap on
the GPU.  Completed requests free their memory and slots, which admits the
next ones.  Per request the server records queueing delay, latency and
iterations; overall it reports DOFs/s and p50/p99 latency.

The footprint of a request is known before any device allocation: the host
part (reference element, mesh maps, patch plans) is built first and its sizes
give the device bytes; requests whose element matrices would not fit use the
matrix-free operator.
"""
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import riesz as rz
from .inputs import kuhn_mesh, normal_vector


@dataclass
class Request:
    rid: int
    space: str
    p: int
    n: int                 # cubes per edge of the Kuhn mesh
    amp: float = 0.1       # vertex perturbation (fraction of h)
    seed: int = 0
    arrival: float = 0.0   # seconds after the start of the stream
    rtol: float = 1e-8
    # filled in by the server
    N: int = 0
    iters: int = 0
    relres: float = float("nan")
    status: int = -1
    t_admit: float = float("nan")
    t_done: float = float("nan")
    footprint: int = 0
    gpu_span: tuple = (float("nan"), float("nan"))  # ms after the server's start event: setup begins, solve ends
    x: np.ndarray = field(default=None, repr=False)

    @property
    def latency(self):
        return self.t_done - self.arrival

    @property
    def queue_delay(self):
        return self.t_admit - self.arrival


def poisson_stream(count, rate, seed, spaces=("CG", "N1curl", "RT"), degrees=(3, 4, 5, 6), sizes=(4, 5, 6, 8)):
    """Seeded Poisson arrivals with mean rate `rate` per second and a random mix of problems."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        out.append(Request(rid=i, space=str(rng.choice(spaces)), p=int(rng.choice(degrees)),
                           n=int(rng.choice(sizes)), seed=int(rng.integers(1 << 30)), arrival=t))
    return out


ALLOC_PAGE = 2 << 20  # device allocator granularity allowed for per allocation (an upper bound)


def estimate_footprint(h, opts=None):
    """Device bytes a created (host-only) handle will hold after setup_device: the library's own plan of
    its buffers (riesz_plan_bytes, the same sizes setup_device allocates) plus one allocator page per
    allocation.  `opts` is accepted for older callers; the handle's options decide the plan."""
    b, nalloc = h.plan_bytes()
    return int(b + nalloc * ALLOC_PAGE)


# the paper's recommended decomposition per space: vertex stars (H1), Hiptmair-Toselli (H(curl), Eq. (6.19)),
# edge stars (H(div), Eq. (6.24)); the same for the second-kind spaces (Hiptmair-Toselli with CG_{p+1}
# potentials for NedTwo_p)
RECOMMENDED = {"CG": rz.DECOMP_VERTEX_STAR, "N1curl": rz.DECOMP_HT, "RT": rz.DECOMP_EDGE_STAR,
               "N2curl": rz.DECOMP_HT, "BDM": rz.DECOMP_EDGE_STAR}


class Server:
    def __init__(self, hbm_budget_bytes=150 << 30, max_slots=4, precond_precision=rz.PREC_FP32, recommended=False,
                 apply_precision=rz.PREC_FP64):
        """recommended: solve each request with the paper's decomposition for its space (else vertex stars);
        apply_precision: precision of the search-direction products (FP32 element matrices need
        RIESZ_APPLY_ELEMENT, which every request that fits uses)."""
        self.budget = hbm_budget_bytes
        self.max_slots = max_slots
        self.prec = precond_precision
        self.recommended = recommended
        self.aprec = apply_precision
        self.lock = threading.Condition()
        self.in_use = 0
        self.active = 0

    def warm(self, spaces, degrees, threads=4):
        """Build the host reference elements of every (space, degree) pair before serving, as a
        server does at start-up: one host-only handle per pair on a single cube with this server's
        options, so the auxiliary spaces its decompositions use (the potentials' CG space, the
        lowest-order coarse space) are built as well.  The tables depend on neither the mesh nor the
        precisions and are cached process-wide, so a request then pays only its own mesh maps.
        Returns {(space, degree): host milliseconds of its handle}."""
        from concurrent.futures import ThreadPoolExecutor
        verts, cells = kuhn_mesh(1)

        def one(pair):
            space, p = pair
            opts = dict(precond_precision=self.prec, apply_precision=self.aprec, autotune=0)
            if self.recommended:
                opts["decomposition"] = RECOMMENDED[space]
            h = rz.Riesz(space, p, verts, cells, device=False, **opts)
            ms = float(h.stats()["setup_host_ms"])
            h.close()
            return ms

        pairs = [(space, p) for space in spaces for p in degrees]
        with ThreadPoolExecutor(max(1, threads)) as ex:
            return dict(zip(pairs, ex.map(one, pairs)))

    def _prepare(self, req):
        verts, cells = kuhn_mesh(req.n, req.amp, req.seed % 1000)
        # no setup-time autotuning: its timing runs would add latency and compete with the other requests
        opts = dict(precond_precision=self.prec, apply_precision=self.aprec, rtol=req.rtol, maxit=5000, autotune=0)
        if self.recommended:
            opts["decomposition"] = RECOMMENDED[req.space]
        h = rz.Riesz(req.space, req.p, verts, cells, device=False, **opts)
        fp = estimate_footprint(h, opts)
        if fp > self.budget // 2:  # element matrices too large: matrix-free operator
            h.close()
            opts["apply_mode"] = rz.APPLY_MATRIX_FREE
            if opts["apply_precision"] == rz.PREC_FP32:
                opts["apply_precision"] = rz.PREC_FP64  # FP32 products need the element matrices
            if self.recommended:
                opts["decomposition"] = RECOMMENDED[req.space]
            h = rz.Riesz(req.space, req.p, verts, cells, device=False, **opts)
            fp = estimate_footprint(h, opts)
        return h, fp

    def _run(self, req, h, t0):
        import torch
        try:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ev[0].record(stream)
                h.setup_device(stream)
                b = torch.tensor(normal_vector(h.N, req.seed % 7919), device="cuda")
                x = torch.zeros_like(b)
                it, rr, rc = h.solve(b, x, stream=stream, check=False)
                ev[1].record(stream)
                stream.synchronize()
                req.x = x.cpu().numpy()
                # the request's span on the GPU clock, relative to the server's start event
                req.gpu_span = (self.ev0.elapsed_time(ev[0]), self.ev0.elapsed_time(ev[1]))
            req.N, req.iters, req.relres, req.status = h.N, int(it[0]), float(rr[0]), int(rc)
        finally:
            req.t_done = time.perf_counter() - t0
            h.close()
            with self.lock:
                self.in_use -= req.footprint
                self.active -= 1
                self.lock.notify_all()

    def _serve_one(self, req, t0):
        """Host preparation, admission, device setup and solve of one request (own thread)."""
        h, fp = self._prepare(req)
        if fp > self.budget:
            h.close()
            req.status = 3  # RIESZ_ERR_OOM: larger than the whole budget
            req.t_admit = req.t_done = time.perf_counter() - t0
            return
        req.footprint = fp
        with self.lock:
            while self.active >= self.max_slots or self.in_use + fp > self.budget:
                self.lock.wait()
            self.in_use += fp
            self.active += 1
        req.t_admit = time.perf_counter() - t0
        self._run(req, h, t0)

    def run(self, requests, realtime=True):
        """Serve the requests; each gets its own thread at its arrival time, which prepares the
        host maps (in parallel with the others), waits for a slot and memory, then solves."""
        import torch
        self.ev0 = torch.cuda.Event(enable_timing=True)
        self.ev0.record()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        threads = []
        for req in sorted(requests, key=lambda r: r.arrival):
            if realtime:
                delay = req.arrival - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            th = threading.Thread(target=self._serve_one, args=(req, t0), daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        self.wall = time.perf_counter() - t0
        return requests


def summary(requests, wall):
    done = [r for r in requests if r.status == 0]
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    return {"requests": len(requests), "completed": len(done),
            "dofs_per_s": float(sum(r.N for r in done) / wall) if wall > 0 else 0.0,
            "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "queue_p50_s": float(np.percentile([r.queue_delay for r in done], 50)) if done else 0.0,
            "wall_s": wall}
