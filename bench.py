#!/usr/bin/env python
"""Benchmark of the Riesz-map PCG solver: DOFs/s solved to 1e-8 relative residual.

One step = one pass of the whole path over one synthetic problem, inputs
resident in HBM: device setup from the vertex coordinates (geometric factors,
element matrices, interior diagonal, patch assembly, batched FP64 Cholesky),
right-hand-side assembly, and PCG to ||b - A x|| <= 1e-8 ||b|| (true residual).
The host-side reference element and mesh maps are built once before timing.

Default workload (the largest single-GPU configuration): H(div) Riesz map,
Raviart-Thomas p = 8 on the unit cube split into 16^3 cubes x 6 tets (24576
tets, 8 017 920 DOFs), interior vertices perturbed by up to 0.1 h (seeded),
8 seeded N(0,1) right-hand sides solved in lockstep, FP64 outer PCG (residuals,
inner products, refinement) with FP32 products and FP32 patch sweeps inside,
rtol 1e-8.  --workload hcurl_ned1_p6_n8 gives the Ned1_6 8^3 line (FP64
operator, FP32 patch solves), --workload hgrad_cg3_n4 the CG_3 4^3 one.

Prints one JSON line (rank 0) with per-step latency (p50/p99 over the timed
steps) and, for the mixed-precision workloads, the same workload timed with the
plain FP64 solver (FP64 operator and FP64 patch solves) on the same GPU.
--impl reference times the CPU oracle instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: space, p, cubes per edge, perturbation, rhs seed, precond precision, nrhs
    "hcurl_ned1_p6_n8": dict(space="N1curl", p=6, n=8, amp=0.1, prec=1, nrhs=1,
                             label="H(curl) Ned1_6 on 8^3 x 6 tets, perturbed 0.1h, FP64 apply + FP32 precond"),
    "hcurl_ned1_p6_n4": dict(space="N1curl", p=6, n=4, amp=0.1, prec=1, nrhs=1,
                             label="H(curl) Ned1_6 on 4^3 x 6 tets, perturbed 0.1h, FP64 apply + FP32 precond "
                                   "(small case for kernel profiles)"),
    "hcurl_ned1_p6_n6": dict(space="N1curl", p=6, n=6, amp=0.1, prec=1, nrhs=1,
                             label="H(curl) Ned1_6 on 6^3 x 6 tets, perturbed 0.1h, FP64 apply + FP32 precond "
                                   "(medium case for kernel profiles)"),
    "hdiv_rt8_n4": dict(space="RT", p=8, n=4, amp=0.1, prec=1, nrhs=8, a32=1,
                        label="H(div) RT_8 on 4^3 x 6 tets, perturbed 0.1h, 8 RHS, FP32 inner products and patch "
                              "solves (small case for kernel profiles)"),
    "hdiv_rt8_n8": dict(space="RT", p=8, n=8, amp=0.1, prec=1, nrhs=8, a32=1,
                        label="H(div) RT_8 on 8^3 x 6 tets, perturbed 0.1h, 8 RHS, FP32 inner products and patch "
                              "solves (medium case for kernel profiles)"),
    "hgrad_cg3_n4": dict(space="CG", p=3, n=4, amp=0.0, prec=0, nrhs=1,
                         label="H(grad) CG_3 on 4^3 x 6 tets, FP64"),
    "hdiv_rt8_n16": dict(space="RT", p=8, n=16, amp=0.1, prec=1, nrhs=8, a32=2, plain_steps=3,
                         decomposition="edge_star", coarse=1,
                         variants=[("hybrid", dict(form="hybrid")),
                                   ("vertex_star_fp32_products", dict(decomposition="vertex_star", a32=1,
                                                                      steps=3))],
                         label="H(div) RT_8 on 16^3 x 6 tets, perturbed 0.1h, 8 RHS in lockstep, FP64 outer PCG "
                               "(residuals, inner products, replacement) with BF16x3 tensor-core contraction "
                               "(FP32 accumulation) for the inner products and FP32 patch solves; PAFW_1 edge "
                               "stars + interior Jacobi + W^2 by lowest-order PCG steps"),
}
DEFAULT = "hdiv_rt8_n16"
METRIC = "DOFs/s solved to 1e-8 rel. residual"
FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64, the profiling recipe's nominal figure (context only)
# CPU sample for the oracle: same space, degree, perturbation and RHS recipe on a small Kuhn mesh
# (cubes per edge, right-hand sides), sized for 10-30 s of CPU work per pass
CPU_SAMPLE = {"hdiv_rt8_n16": (2, 2), "hdiv_rt8_n4": (2, 2)}
CPU_SAMPLE_DEFAULT = (3, 1)
# mesh of the error check against the oracle's direct solve (same recipe, small mesh)
ERR_SAMPLE_N = 2


DECOMPOSITIONS = {"vertex_star": 0, "ht": 1, "edge_star": 2}  # riesz_opts.decomposition


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                    help="patch solves in FP64, or FP32 (mixed)")
    ap.add_argument("--apply-precision", default=None, choices=["fp64", "fp32", "bf16x3"],
                    help="precision of the operator products inside PCG (FP64 residuals either way): FP64 or "
                         "FP32 element matrices, or the BF16x3 tensor-core matrix-free contraction")
    ap.add_argument("--serve", action="store_true",
                    help="serving run: Poisson stream of mixed solves, reports DOFs/s and p50/p99 latency")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--batch", action="store_true",
                    help="batched run: seeded mixed systems solved in one graph launch per HBM wave")
    ap.add_argument("--systems", type=int, default=64)
    ap.add_argument("--hbm-budget-gb", type=float, default=200.0)
    ap.add_argument("--decomposition", default=None, choices=sorted(DECOMPOSITIONS),
                    help="subspace decomposition: vertex stars (Eq. 6.11), Hiptmair-Toselli edge stars + "
                         "gradient potential problems for H(curl) (Eq. 6.19), or PAFW_1 edge stars for "
                         "H(div) (Eq. 6.24)")
    ap.add_argument("--form", default=None, choices=["additive", "hybrid"],
                    help="combination of the subspace corrections: additive, or the paper's symmetric "
                         "multiplicative hybrid sweep (Section 7.1, Eqs. 7.2-7.3)")
    ap.add_argument("--coarse", type=int, default=None, choices=[0, 1, 2],
                    help="W^k coarse space: 0 off, 1 dense inverse up to 6144 DOFs and lowest-order PCG steps above, "
                         "2 lowest-order PCG steps")
    ap.add_argument("--replace-digits", type=int, default=None,
                    help="FP64 residual replacement every this many digits (inexact inner products)")
    ap.add_argument("--coarse-its", type=int, default=None,
                    help="PCG steps of the lowest-order coarse route (W^k above the dense limit)")
    ap.add_argument("--pcg-loop", default="graph", choices=["graph", "host"],
                    help="device-driven (CUDA graph) or host-driven PCG iterations; same kernels, same results")
    ap.add_argument("--p-sweep", action="store_true",
                    help="iteration counts against the degree p on a fixed mesh (p-robustness table)")
    ap.add_argument("--hodge", type=int, default=0, choices=[0, 1, 2, 3],
                    help="Hodge-Laplace problem of Section 7.2 (k = 1: CG_p x Ned1_p, k = 2: Ned1_p x RT_p, "
                         "k = 3: RT_p x DG_{p-1}) on a Kuhn Fichera corner, MINRES with the augmented-Lagrangian "
                         "preconditioner")
    ap.add_argument("--hodge-p", type=int, default=4)
    ap.add_argument("--hodge-n", type=int, default=8)
    ap.add_argument("--gamma", type=float, default=1e3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the run with the paper's finer decomposition (HT / edge stars)")
    ap.add_argument("--no-fp64-plain", action="store_true",
                    help="skip the comparison run of the plain FP64 solver on the same workload")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ---------------------------------------------------------------------------
def oracle_pass(space, p, n, amp, nrhs=1, seed=1):
    """One pass of the oracle (assembly, load, preconditioner setup, PCG per right-hand side); returns
    (N, seconds, iters).  One right-hand side: f with N(0,1) CG_p coefficients per component (b = (f, phi));
    several: N(0,1) vectors (the paper's random right-hand side), as the GPU workload draws them."""
    import numpy as np
    from oracle import assemble as asm
    from oracle.mesh import MeshDofs
    from oracle.refelem import reference_element
    from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_coeffs
    ref = reference_element(space, p)
    cg = reference_element("CG", p)
    verts, cells = kuhn_mesh(n, amp, seed)
    t0 = time.perf_counter()
    md = MeshDofs(verts, cells, ref)
    A = asm.assemble(md, asm.element_matrices(ref, verts, cells))
    if nrhs == 1:
        mcg = MeshDofs(verts, cells, cg)
        f = normal_coeffs((1 if space == "CG" else 3, mcg.ndofs), 2)
        B = asm.load_cg_field(ref, md, cg, mcg, f)[None, :]
    else:
        B = normal_coeffs((nrhs, md.ndofs), 2)
    P = asm.Preconditioner(A, md)
    its = []
    for k in range(nrhs):
        x, it, rr = asm.pcg(A, B[k], P.apply, rtol=1e-8)
        assert rr <= 1e-8 * 1.001, rr
        its.append(it)
    dt = time.perf_counter() - t0
    return md.ndofs, dt, max(its)


FORMS = {"additive": 0, "hybrid": 1}  # riesz_opts.form


def solver_opts(wl, args, decomposition=None, form=None):
    """Decomposition, form and coarse-space options of the workload (command-line overrides first)."""
    o = {"decomposition": DECOMPOSITIONS[decomposition or args.decomposition or wl.get("decomposition",
                                                                                       "vertex_star")],
         "form": FORMS[form or args.form or wl.get("form", "additive")]}
    coarse = args.coarse if args.coarse is not None else wl.get("coarse")
    if coarse is not None:
        o["coarse"] = coarse
    rd = args.replace_digits if args.replace_digits is not None else wl.get("replace_digits")
    if rd is not None:
        o["replace_digits"] = rd
    cits = args.coarse_its if args.coarse_its is not None else wl.get("coarse_its")
    if cits is not None:
        o["coarse_its"] = cits
    return o


def cpu_sample(args):
    return CPU_SAMPLE.get(args.workload, CPU_SAMPLE_DEFAULT)


def cpu_baseline(wl, args):
    n, nr = cpu_sample(args)
    N, dt, it = oracle_pass(wl["space"], wl["p"], n, wl["amp"], nrhs=nr)
    return {"value": N * nr / dt, "unit": "DOFs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%s p=%d on %d^3 x 6 tets (N=%d, same perturbation and RHS recipe), %d right-hand side(s), "
                      "one full oracle pass (numbering, quadrature assembly, load, patch Cholesky, PCG to 1e-8 per "
                      "right-hand side): %.1f s, %d iterations; BLAS threads at library default"
                      % (wl["space"], wl["p"], n, N, nr, dt, it)}


def err_vs_oracle(wl, args, make_solver):
    """The GPU path of the workload (same space, degree, precisions, right-hand-side recipe, number of
    right-hand sides and rtol) on the ERR_SAMPLE_N^3 mesh of the same recipe, against the oracle's FP64
    sparse direct solve: max over right-hand sides of ||x - x_oracle|| / ||x_oracle||."""
    import numpy as np
    import torch
    from oracle import assemble as asm
    from oracle.mesh import MeshDofs
    from oracle.refelem import reference_element
    from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_coeffs
    n = ERR_SAMPLE_N
    nrhs = wl.get("nrhs", 1)
    verts, cells = kuhn_mesh(n, wl["amp"], 1)
    s = make_solver(verts, cells)
    ref = reference_element(wl["space"], wl["p"])
    md = MeshDofs(verts, cells, ref)
    A = asm.assemble(md, asm.element_matrices(ref, verts, cells))
    if nrhs == 1:
        cg = reference_element("CG", wl["p"])
        mcg = MeshDofs(verts, cells, cg)
        f = normal_coeffs((1 if wl["space"] == "CG" else 3, mcg.ndofs), 2)
        B = asm.load_cg_field(ref, md, cg, mcg, f)[None, :]
    else:
        B = normal_coeffs((nrhs, md.ndofs), 2)
    b = torch.tensor(B, device="cuda")
    x = torch.zeros_like(b)
    it, rr, rc = s.solve(b, x, nrhs=nrhs, check=False)
    X = x.cpu().numpy()
    errs = []
    for k in range(nrhs):
        xe = asm.direct_solve(A, B[k])
        errs.append(float(np.linalg.norm(X[k] - xe) / np.linalg.norm(xe)))
    s.close()
    return {"max_rel_l2": max(errs), "rtol": 1e-8, "status": int(rc), "iterations": int(it[0]),
            "sample": "same recipe on %d^3 x 6 tets (N=%d, %d right-hand side(s)), oracle FP64 sparse direct solve"
                      % (n, md.ndofs, nrhs)}


# ---------------------------------------------------------------------------
def run_reference(args, wl, rank, world):
    if rank != 0:
        return
    n, nr = cpu_sample(args)
    for _ in range(args.warmup):
        oracle_pass(wl["space"], wl["p"], n, wl["amp"], nrhs=nr)
    tot, N = 0.0, 0
    for _ in range(args.steps):
        N, dt, _ = oracle_pass(wl["space"], wl["p"], n, wl["amp"], nrhs=nr)
        tot += dt
    value = N * nr * args.steps / tot
    cb = {"value": value, "unit": "DOFs/s", "cores": os.cpu_count(), "kind": "oracle",
          "sample": "%s p=%d on %d^3 x 6 tets (N=%d), %d right-hand side(s): full oracle pass per step"
                    % (wl["space"], wl["p"], n, N, nr)}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOFs/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": wl["label"], "cpu_sample_cubes_per_edge": n,
                                           "cpu_sample_rhs": nr},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "DOFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def measured_fp64_peak():
    """FP64 FMA rate of this GPU (riesz_probe_fp64, best of three bounded launches), TFLOP/s."""
    from paper_2506_17406_gb300 import riesz as rz
    return max(rz.probe_fp64(16384) for _ in range(3))


def fp64_peak_source(tf):
    return ("measured in this run: riesz_probe_fp64, a bounded FP64 FMA loop on this GPU (best of 3), "
            "%.3f TFLOP/s; nominal %.2f" % (tf, FP64_NOMINAL_TFLOPS))


def combine_ranks(ms, n_local, dist=None, device=None):
    """Replicas: every rank solves its own problem.  Returns (max time over ranks,
    total DOFs over ranks); a single process returns its own values."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms), float(n_local)
    import torch
    tm = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    tn = torch.tensor([float(n_local)], dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(tn, op=dist.ReduceOp.SUM)
    return float(tm.item()), float(tn.item())


SIDE_STREAM_KINDS = {"coarse", "coarse_apply"}
# kernel kinds launched inside the PCG loop (timing one per launch needs the host-driven loop)
LOOP_KIND_NAMES = {"apply", "apply32", "apply_tc", "gather", "patch_solve", "precond_gather", "dot", "scalar",
                   "update", "coarse_apply", "ht"}


def kernel_source_hash(name):
    """sha256 of one kernel's source text in kernels.cuh: from the line that declares `name(` to the
    brace that closes its body (None if not found)."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_2506_17406_gb300", "csrc", "kernels.cuh")).read()
    i = src.find(" " + name + "(")
    if i < 0:
        return None
    i = src.rfind("\n", 0, i) + 1
    j = src.index("{", i)
    depth, k = 0, j
    while k < len(src):
        depth += {"{": 1, "}": -1}.get(src[k], 0)
        k += 1
        if depth == 0:
            break
    return hashlib.sha256(src[i:k].encode()).hexdigest()


def measured_traffic(workload, kernel):
    """DRAM bytes per launch from the committed ncu summary, if that kernel's source has not changed
    since the counters were taken."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except Exception:
        return None
    e = t.get("workloads", {}).get(workload, {}).get(kernel)
    if not e or e.get("sha256") != kernel_source_hash(e.get("function", kernel)):
        return None
    return e.get("bytes")


def patch_flops_bytes(s):
    """Algorithmic FP64 Cholesky flops (sum n^3/3) and factor entries from the patch map."""
    import numpy as np
    off, _ = s.patch_map()
    n = np.diff(off).astype(np.float64)
    return float(np.sum(n ** 3 / 3.0)), float(np.sum(n * (n + 1) / 2.0)), float(np.sum(n))


def run_serving(args):
    """Poisson arrivals (mean 200 requests/s, seeded) of Riesz-map solves mixing CG, Ned1, RT, NedTwo and BDM
    with p in 3..10 and Kuhn meshes of 4..20 cubes per edge (384..48 000 tets), perturbed by 0.1h, admitted by a 150 GB
    HBM budget with up to 8 requests in flight, each solved with the paper's decomposition for its space
    (vertex stars, Hiptmair-Toselli, edge stars) and W^k.  The mixed server (FP32 patch sweeps, BF16x3
    tensor-core products) and the plain FP64 server serve the same stream one after the other."""
    import numpy as np
    import torch
    from paper_2506_17406_gb300 import riesz as rz
    from paper_2506_17406_gb300 import serve
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    degrees, sizes = tuple(range(3, 11)), tuple(range(4, 21))
    spaces = ("CG", "N1curl", "RT", "N2curl", "BDM")
    warm = serve.poisson_stream(6, rate=200.0, seed=100, degrees=(3, 4), sizes=(4,))
    serve.Server(max_slots=8, recommended=True).run(warm, realtime=False)
    # reference elements of every (space, degree) the stream can draw, built before timing as a server
    # does at start-up (process-wide cache): neither server's latencies include them
    t_warm = time.perf_counter()
    serve.Server(recommended=True).warm(spaces, degrees)
    t_warm = time.perf_counter() - t_warm
    out = {"metric": "serving: DOFs/s and p50/p99 latency of solves to 1e-8", "unit": "DOFs/s", "n_gpus": 1,
           "higher_is_better": True, "data": "synthetic",
           "config": {"workload": "Poisson stream, mean 200 req/s, CG/Ned1/RT/NedTwo/BDM, p 3..10, "
                                  "4..20 cubes per edge "
                                  "(384..48000 tets), perturbed 0.1h, 150 GB budget, 8 slots, recommended "
                                  "decompositions + W^k, reference elements built before the stream",
                      "requests": args.requests, "reference_build_s": round(t_warm, 1)}}
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    for name, kw in (("mixed", dict(precond_precision=rz.PREC_FP32, apply_precision=rz.PREC_BF16X3)),
                     ("fp64_plain", dict(precond_precision=rz.PREC_FP64, apply_precision=rz.PREC_FP64))):
        reqs = serve.poisson_stream(args.requests, rate=200.0, seed=7, spaces=spaces, degrees=degrees, sizes=sizes)
        srv = serve.Server(hbm_budget_bytes=150 << 30, max_slots=8, recommended=True, **kw)
        done = srv.run(reqs, realtime=True)
        st = serve.summary(done, srv.wall)
        ok = [r for r in done if r.status == 0]
        res = {"value": st["dofs_per_s"], "latency_p50_s": st["latency_p50_s"],
               "latency_p99_s": st["latency_p99_s"], "queue_p50_s": st["queue_p50_s"], "completed": st["completed"],
               "wall_s": st["wall_s"], "max_relres": max(r.relres for r in ok) if ok else None,
               "dofs_total": int(sum(r.N for r in ok)),
               "largest_request": max(((r.space, r.p, r.n, r.N) for r in ok), key=lambda t: t[3]) if ok else None}
        if name == "mixed":
            out.update(res)
        else:
            out["fp64_plain"] = res
    out["clocks"] = clocks.stop()
    out["speedup_vs_fp64_plain"] = out["value"] / out["fp64_plain"]["value"] if out["fp64_plain"]["value"] else None
    print(json.dumps(out), flush=True)


def batch_draws(count, seed=4, degrees=(2, 10), sizes=(4, 12)):
    """Seeded draws (space, p, cubes per edge) with p and n uniform in the given ranges."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    return [(str(rng.choice(["CG", "N1curl", "RT", "N2curl", "BDM"])), int(rng.integers(degrees[0], degrees[1] + 1)),
             int(rng.integers(sizes[0], sizes[1] + 1))) for _ in range(count)]


def run_batch(args):
    """Batched solves: seeded draws over spaces {CG, Ned1, RT, NedTwo, BDM}, p in 2..10, n^3 x 6 tets with n
    in 4..12, perturbed 0.1h, one seeded random right-hand side each, FP32 inner products and patch sweeps
    with FP64 residuals.  The systems are packed into waves that fit the HBM budget; a wave's device setups run
    together (riesz_update_geometry_batch: one stream per system) and its solves run as one graph launch
    (riesz_solve_batch).  The same systems are then set up and solved one after the other for comparison."""
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_2506_17406_gb300 import riesz as rz
    from paper_2506_17406_gb300 import serve
    from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_vector
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    draws = batch_draws(args.systems)
    opts = dict(precond_precision=rz.PREC_FP32, rtol=1e-8, maxit=5000)

    def prep(i):
        space, p, n = draws[i]
        verts, cells = kuhn_mesh(n, 0.1, 1000 + i)
        # the paper's decomposition per space, BF16x3 tensor-core products
        o = dict(opts, decomposition=serve.RECOMMENDED[space], apply_precision=rz.PREC_BF16X3)
        h = rz.Riesz(space, p, verts, cells, device=False, **o)
        return h, verts, serve.estimate_footprint(h)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        prepared = list(ex.map(prep, range(len(draws))))
    host_s = time.perf_counter() - t0
    budget = int(args.hbm_budget_gb * (1 << 30))
    waves, cur, used = [], [], 0
    for i, (_, _, fp) in enumerate(prepared):
        if cur and used + fp > budget:
            waves.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += fp
    if cur:
        waves.append(cur)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    setup_ms = solve_ms = seq_ms = seq_setup_ms = 0.0
    iters, relres, status, ndofs = [], [], [], []
    launches = 0
    for wave in waves:
        hs = [prepared[i][0] for i in wave]
        for h in hs:
            h.setup_device()
        verts_d = [torch.tensor(prepared[i][1], device="cuda") for i in wave]
        bs = [torch.tensor(normal_vector(h.N, 500 + i), device="cuda").reshape(1, -1) for h, i in zip(hs, wave)]
        xs = [torch.zeros_like(b) for b in bs]
        l0 = sum(h.stats()["launches"] for h in hs)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        rz.update_geometry_batch(hs, verts_d)  # every system's setup on its own stream, joined once
        e[1].record(stream)
        it, rr, st = rz.solve_batch(hs, bs, xs)
        e[2].record(stream)
        torch.cuda.synchronize()
        setup_ms += e[0].elapsed_time(e[1])
        solve_ms += e[1].elapsed_time(e[2])
        launches += sum(h.stats()["launches"] for h in hs) - l0
        iters += [int(k) for k in it]
        relres += [float(r) for r in rr]
        status += [int(k) for k in st]
        ndofs += [h.N for h in hs]
        # the same systems set up and solved one after the other
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        for h, v in zip(hs, verts_d):
            h.update_geometry(v)
        e1.record(stream)
        for h, b, x in zip(hs, bs, xs):
            h.solve(b, x, check=False)
        e2.record(stream)
        torch.cuda.synchronize()
        seq_setup_ms += e0.elapsed_time(e1)
        seq_ms += e1.elapsed_time(e2)
        for h in hs:
            h.close()
        del verts_d, bs, xs
        torch.cuda.empty_cache()
    clk = clocks.stop()
    ntot = float(sum(ndofs))
    by_space = {}
    for (space, p, n), it in zip(draws, iters):
        by_space.setdefault(space, {}).setdefault(p, []).append(it)
    out = {"metric": "batched: DOFs/s solved to 1e-8 (device setup + one-launch solve per wave)",
           "value": ntot / ((setup_ms + solve_ms) / 1e3), "unit": "DOFs/s", "n_gpus": 1, "higher_is_better": True,
           "data": "synthetic", "dtype": "f64+f32",
           "config": {"workload": "%d seeded draws: space in {CG, Ned1, RT, NedTwo, BDM}, p in 2..10, "
                                  "n^3 x 6 tets with n in "
                                  "4..12, perturbed 0.1h, random RHS, the paper's decomposition per space + W^k, "
                                  "BF16x3 tensor-core products and FP32 patch sweeps, FP64 residuals, rtol 1e-8"
                                  % len(draws),
                      "hbm_budget_gb": args.hbm_budget_gb, "waves": [len(w) for w in waves]},
           "dofs": int(ntot), "setup_ms": setup_ms, "solve_ms": solve_ms,
           "solve_dofs_per_s": ntot / (solve_ms / 1e3),
           "sequential_solve_ms": seq_ms, "batch_speedup_vs_sequential_solves": seq_ms / solve_ms,
           "sequential_setup_ms": seq_setup_ms, "batch_speedup_vs_sequential_setups": seq_setup_ms / setup_ms,
           "converged": sum(1 for k in status if k == 0), "max_relres": max(relres),
           "iterations_by_space_and_p": {sp: {str(p): sorted(v) for p, v in sorted(d.items())}
                                         for sp, d in by_space.items()},
           "host_prep_s": host_s, "gpu_launches": launches, "clocks": clk}
    print(json.dumps(out), flush=True)


def run_p_sweep(args):
    """PCG iterations to 1e-8 against the degree on fixed perturbed meshes (Section 7.1 setting: random
    right-hand side, zero initial guess), FP64 and mixed precision, for each space."""
    import numpy as np
    import torch
    from paper_2506_17406_gb300 import riesz as rz
    from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_vector
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    table = {}
    for n in (2, 4):
        verts, cells = kuhn_mesh(n, 0.1, 1)
        for space in ("CG", "N1curl", "RT", "N2curl", "BDM"):
            for p in range(1, 11):
                row = {}
                for name, kw in (("one_level", dict(coarse=0)), ("two_level", dict(coarse=1)),
                                 ("two_level_mixed", dict(coarse=1, precond_precision=rz.PREC_FP32)),
                                 ("hybrid", dict(coarse=1, form=rz.FORM_HYBRID)),
                                 ("hybrid_recommended", dict(coarse=1, form=rz.FORM_HYBRID,
                                                             decomposition={"CG": 0, "N1curl": 1, "RT": 2,
                                                                            "N2curl": 1, "BDM": 2}[space]))):
                    s = rz.Riesz(space, p, verts, cells, maxit=5000, **kw)
                    b = torch.tensor(normal_vector(s.N, 7), device="cuda")
                    x = torch.zeros_like(b)
                    it, rr, rc = s.solve(b, x, check=False)
                    row[name] = int(it[0]) if rc == 0 else None
                    row["dofs"] = s.N
                    s.close()
                table.setdefault("n=%d" % n, {}).setdefault(space, {})[str(p)] = row
    print(json.dumps({"metric": "PCG iterations to 1e-8 vs degree p", "data": "synthetic",
                      "config": {"meshes": "n^3 x 6 Kuhn tets, perturbed 0.1h", "rhs": "N(0,1) vector",
                                 "preconditioner": "interior Jacobi + vertex-star patches (one_level), "
                                                   "+ W^k coarse space (two_level), additive; two_level_mixed "
                                                   "with FP32 patch sweeps; hybrid: the paper's multiplicative "
                                                   "sweep with Lanczos weights (vertex stars), "
                                                   "hybrid_recommended: the same with the paper's decomposition "
                                                   "per space (Hiptmair-Toselli for Ned1, edge stars for RT)"},
                      "iterations": table}), flush=True)


def run_hodge(args):
    """Hodge-Laplace problem (Section 7.2): (sigma, u) in X^{k-1} x X^k on the Kuhn mesh of the Fichera
    corner (0,1)^3 minus (1/2,1)^3, interior vertices perturbed by 0.1h, constant source f = (1,1,1),
    preconditioned MINRES to 1e-8 with the weighted Riesz-map blocks of Eq. (7.6) replaced by the
    paper's per-space Schwarz preconditioners (FP64 patch sweeps, FP32 with --precision mixed)."""
    import numpy as np
    import torch
    from paper_2506_17406_gb300 import riesz as rz
    from paper_2506_17406_gb300.inputs import fichera_mesh
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    k, p, n, gamma = args.hodge, args.hodge_p, args.hodge_n, args.gamma
    verts, cells = fichera_mesh(n, 0.1, 1)
    prec = rz.PREC_FP32 if args.precision == "mixed" else rz.PREC_FP64
    form = args.form or "additive"
    h = rz.Hodge(k, p, verts, cells, gamma, decomposition=rz.DECOMP_HT, precond_precision=prec,
                 rtol=1e-8, maxit=5000, form=FORMS[form])
    stream = torch.cuda.current_stream()
    fcg_h = np.zeros((3 if k < 3 else 1, h.n_cg))
    fcg_h[:, :len(verts)] = 1.0  # f = (1,1,1) (f = 1 for k = 3): the vertex (Whitney) functions sum to one
    fcg = torch.tensor(fcg_h, device="cuda")
    verts_d = torch.tensor(verts, device="cuda")
    b = torch.zeros(h.N, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    iters, rels = [], []

    def step():
        h.update_geometry(verts_d)
        h.load(fcg, b)
        x.zero_()
        it, rr, _ = h.solve(b, x)
        iters.append(it)
        rels.append(rr)

    for _ in range(args.warmup):
        step()
    launches0 = h.stats()["launches"]
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for i in range(args.steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    launches = h.stats()["launches"] - launches0
    ms = sum(per)
    # the block operator alone (fused cell kernel + two interface gathers), CUDA events around 20 products
    xa = torch.randn(h.N, dtype=torch.float64, device="cuda")
    ya = torch.zeros_like(xa)
    for _ in range(3):
        h.apply(xa, ya)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        h.apply(xa, ya)
    e1.record(stream)
    torch.cuda.synchronize()
    apply_ms = e0.elapsed_time(e1) / 20
    sp = {1: ("CG", "N1curl"), 2: ("N1curl", "RT"), 3: ("RT", "DG")}[k]
    nref = {"CG": (p + 1) * (p + 2) * (p + 3) // 6, "N1curl": p * (p + 2) * (p + 3) // 2,
            "RT": p * (p + 1) * (p + 3) // 2, "DG": p * (p + 1) * (p + 2) // 6}
    n0, n1 = nref[sp[0]], nref[sp[1]]
    C = len(cells)
    flops = 2.0 * C * ((n1 * n1 if k < 3 else 0) + 2 * n0 * n1 + n0 * n0)
    tf = flops / (apply_ms * 1e-3) / 1e12
    pk = measured_fp64_peak()
    roof = {"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s",
            "frac": tf / pk, "traffic": None, "kernel": "k_hodge_apply (+2 k_gather_iface)",
            "peak_source": fp64_peak_source(pk),
            "algorithmic": "2 C (n_k^2 + 2 n_{k-1} n_k + n_{k-1}^2) = %.3e flop per block product (element "
                           "matrices of K_k, M_{k-1} and the coupling read once: %.3e B)"
                           % (flops, 8.0 * C * (n1 * n1 + n0 * n1 + n0 * n0))}
    # end to end: host vertices and source in, solution out
    verts_pin = torch.tensor(verts).pin_memory()
    fcg_pin = torch.tensor(fcg_h).pin_memory()
    x_pin = torch.zeros(h.N, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        verts_d.copy_(verts_pin, non_blocking=True)
        fcg.copy_(fcg_pin, non_blocking=True)
        step()
        x_pin.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
    te = time.perf_counter() - t0
    cb = None
    if not args.no_cpu_baseline:
        from oracle import hodge as ohodge
        vs, cs = fichera_mesh(2, 0.1, 1)
        t1 = time.perf_counter()
        hs = ohodge.HodgeSystem(k, p, vs, cs, gamma)
        bs = hs.rhs(np.ones(hs.n1))
        _, ito, _ = ohodge.minres(hs.A, bs, hs.schwarz_preconditioner(True, form=form), rtol=1e-8, maxit=5000)
        dt = time.perf_counter() - t1
        cb = {"value": (hs.n0 + hs.n1) / dt, "unit": "DOFs/s", "cores": os.cpu_count(), "kind": "oracle",
              "sample": "same k, p, gamma on the 2^3-cube Fichera mesh (N=%d): assembly, Schwarz blocks and "
                        "MINRES (%d iterations), %.1f s" % (hs.n0 + hs.n1, ito, dt)}
    out = {"metric": "Hodge-Laplace DOFs/s solved (MINRES to 1e-8, preconditioned residual)",
           "value": h.N * args.steps / (ms / 1e3), "unit": "DOFs/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64+f32" if prec == rz.PREC_FP32 else "f64", "data": "synthetic",
           "config": {"workload": "Hodge-Laplace k=%d (%s x %s), p=%d, Kuhn Fichera corner %d^3 cubes minus "
                                  "the (1/2,1)^3 octant (%d tets), perturbed 0.1h, f=%s, gamma=%g"
                                  % (k, sp[0], sp[1], p, n, C, "(1,1,1)" if k < 3 else "1", gamma),
                      "n0": h.n0, "n1": h.n1, "dofs": h.N,
                      "preconditioner": "block diagonal weighted Riesz maps (Eq. 7.6), each one application "
                                        "of its Schwarz preconditioner (CG: vertex stars, Ned1: Hiptmair-Toselli, "
                                        "DG: exact diagonal, "
                                        "RT: edge stars; W^k with FP64 coarse inverse)",
                      "sweeps": "fp32" if prec == rz.PREC_FP32 else "fp64", "form": form,
                      "step": "device setup of all blocks + load + MINRES", "l2": "element matrices and patch "
                                                                               "factors larger than L2"},
           "iterations": float(np.median(iters[-args.steps:])), "max_relres": max(rels[-args.steps:]),
           "latency_p50_ms": float(np.percentile(per, 50)), "latency_p99_ms": float(np.percentile(per, 99)),
           "block_apply_ms": apply_ms, "roofline": roof, "cpu_baseline": cb,
           "e2e": {"value": h.N * args.steps / te, "unit": "DOFs/s", "h2d_bytes_per_step": verts.size * 8 +
                   fcg_h.size * 8, "d2h_bytes_per_step": h.N * 8},
           "gpu_launches": launches, "clocks": clk}
    print(json.dumps(out), flush=True)
    h.close()


def main():
    args = parse()
    if args.p_sweep:
        return run_p_sweep(args)
    if args.hodge:
        return run_hodge(args)
    if args.serve:
        return run_serving(args)
    if args.batch:
        return run_batch(args)
    wl = dict(WORKLOADS[args.workload])
    if args.precision == "fp64":
        wl["prec"] = 0
    elif args.precision == "mixed":
        wl["prec"] = 1
    if args.apply_precision == "fp64":
        wl["a32"] = 0
    elif args.apply_precision == "fp32":
        wl["a32"] = 1
    elif args.apply_precision == "bf16x3":
        wl["a32"] = 2
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, wl, rank, world)

    import numpy as np
    import torch
    from paper_2506_17406_gb300 import riesz as rz
    from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_coeffs

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    verts, cells = kuhn_mesh(wl["n"], wl["amp"], seed=1 + rank)
    nrhs = wl.get("nrhs", 1)
    stream = torch.cuda.current_stream()
    verts_d = torch.tensor(verts, device="cuda")
    ncomp = 1 if wl["space"] == "CG" else 3

    def make(prec, a32, decomposition=None, form=None):
        """A solver handle for the workload and its step closure (device setup + load + solve)."""
        s = rz.Riesz(wl["space"], wl["p"], verts, cells, precond_precision=prec, nrhs_max=nrhs,
                     apply_precision=a32, loop=rz.LOOP_HOST if args.pcg_loop == "host" else rz.LOOP_GRAPH,
                     **solver_opts(wl, args, decomposition, form))
        if nrhs == 1:  # f with N(0,1) CG_p coefficients per Cartesian component, b = (f, phi)
            fcg_h = normal_coeffs((ncomp, s.n_cg), 2 + rank)
        else:  # the paper's random right-hand side vectors (Section 7.1), one per RHS
            fcg_h = normal_coeffs((nrhs, s.N), 2 + rank)
        fcg = torch.tensor(fcg_h, device="cuda")
        b = torch.zeros((nrhs, s.N), dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        iters, relres = [], []

        def step():
            s.update_geometry(verts_d)
            if nrhs == 1:
                s.load(fcg, b)
            else:
                b.copy_(fcg)
            x.zero_()
            it, rr, _ = s.solve(b, x, nrhs=nrhs)
            iters.append(int(it[0]))
            relres.append(float(np.max(rr)))

        return s, step, iters, relres, fcg, fcg_h, b, x

    def timed(step, steps):
        """Per-step device times (CUDA events on the launching stream between consecutive steps)."""
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for i in range(steps):
            step()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        return [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]

    s, step, iters, relres_l, fcg, fcg_h, b, x = make(wl["prec"], wl.get("a32", 0))
    for _ in range(args.warmup):
        step()
    # full per-kernel breakdown from one untimed step with every kernel bracketed
    # by CUDA events (the PCG loop is host-driven while loop kernels are timed)
    s.profile(True)
    step()
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    # the coarse setup and the coarse correction run on a side stream beside k_cholesky and the patch
    # sweeps: their event spans overlap other kernels, so they are not candidates for the dominant kernel
    dom = max((k for k in prof if k not in SIDE_STREAM_KINDS), key=lambda k: prof[k][0])
    # timed region: only the dominant kernel is timed per launch; if it runs inside
    # the PCG loop, the loop is host-driven there (graph passes cannot be timed per launch)
    loop_driver = "host" if (dom in LOOP_KIND_NAMES or args.pcg_loop == "host") else "graph"
    torch.cuda.synchronize()
    launches0 = s.stats()["launches"]
    s.profile(True, kinds=[dom])
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    per_step = timed(step, args.steps)
    ms = sum(per_step)
    clk = clocks.stop()
    relres = max(relres_l[-args.steps:])
    live = s.profile_read()
    s.profile(False)
    launches = s.stats()["launches"] - launches0
    ms, ntot = combine_ranks(ms, s.N, dist, device="cuda")
    value = ntot * nrhs * args.steps / (ms / 1e3)

    # setup / solve split from the profiler (kernel time only)
    setup_kinds = ["geom", "elem", "diag", "assemble", "cholesky", "to_f32", "coarse"]
    k_ms = {k: v[0] for k, v in prof.items()}
    # dominant kernel and its roofline (average launch time measured live in the timed region)
    src = live if live[dom][1] > 0 else prof
    dom_ms = src[dom][0] / max(1, src[dom][1])
    st = s.stats()
    chol_flops = st["chol_flops"]
    dense_flops, fentries, psum = patch_flops_bytes(s)
    n = s.nref
    C = s.ncells
    fbytes = 4 if wl["prec"] == 1 else 8
    peak_hbm = 6701.5
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak_hbm = float(peaks.get("hbm_gbs", peak_hbm))
    except Exception:
        pass
    fp64_pk = measured_fp64_peak()
    if dom == "cholesky":
        achieved = chol_flops / (dom_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_pk, "unit": "TFLOP/s",
                "frac": achieved / fp64_pk, "traffic": measured_traffic(args.workload, "k_cholesky"),
                "kernel": "k_cholesky",
                "peak_source": fp64_peak_source(fp64_pk),
                "algorithmic": "tile-sparse Cholesky of all patches = %.3e flop per launch (dense "
                               "sum n_V^3/3 would be %.3e)" % (chol_flops, dense_flops)}
    elif dom == "patch_solve":
        byt = st["precond_bytes"] + psum * 16.0 * (nrhs - 1)  # every RHS gathers r and writes its patch copy
        achieved = byt / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
                "frac": achieved / peak_hbm, "traffic": measured_traffic(args.workload, "k_patch_solve"),
                "kernel": "k_patch_sweep" if nrhs == 1 else "k_patch_solve_multi",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                "algorithmic": "2 sweeps over the stored factor tiles and diagonal inverses + patch "
                               "vectors of every RHS = %.3e B per launch" % byt}
    elif dom == "apply_tc":
        # BF16x3 contraction: algorithmic 2 Q n^2 C nrhs flop per launch (the operator); the tensor pipe
        # executes three BF16 products per term over the padded tile (rows 128 per tile, N = n padded to
        # 16, K = Q x n padded to 32)
        Q = {"CG": 7, "N1curl": 12, "RT": 7}[wl["space"]]
        algo = 2.0 * Q * n * n * C * nrhs
        rt = 8 if nrhs >= 8 else (4 if nrhs >= 4 else (2 if nrhs >= 2 else 1))
        tiles = -(-C // (128 // rt)) * -(-nrhs // rt)
        np_, kpad = -(-n // 16) * 16, -(-n // 32) * 32 * Q
        executed = 3 * 2.0 * 128 * np_ * kpad * tiles
        peak_bf16 = 1704.7
        try:
            peak_bf16 = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops_sustained",
                                                                                             peak_bf16))
        except Exception:
            pass
        tf = executed / (dom_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": tf, "peak": peak_bf16, "unit": "TFLOP/s", "frac": tf / peak_bf16,
                "traffic": measured_traffic(args.workload, "k_apply_tc"), "kernel": "k_apply_tc",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16 GEMM, seconds-long loop)",
                "algorithmic_tflops": algo / (dom_ms / 1e3) / 1e12,
                "algorithmic": "operator 2 Q n^2 C nrhs = %.3e flop per launch; executed BF16 MMA work (3 split "
                               "products, padded tiles) %.3e flop" % (algo, executed)}
    else:
        esize = 4.0 if dom == "apply32" else 8.0
        byt = C * n * n * esize + nrhs * (C * n * 12.0 + s.N * 16.0)
        flops = 2.0 * C * n * n * nrhs
        achieved = byt / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
                "frac": achieved / peak_hbm, "traffic": measured_traffic(args.workload, "k_" + dom),
                "kernel": dom,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                "algorithmic": "element matrices + gathered vectors = %.3e B per launch" % byt}
        if dom == "apply" and flops / (fp64_pk * 1e12) > byt / (peak_hbm * 1e9):
            # FP64 element products: one DFMA per 8-byte matrix entry and right-hand side, so the FP64
            # pipe, not HBM, bounds the launch (2 C n^2 nrhs flop)
            tf = flops / (dom_ms / 1e3) / 1e12
            roof.update({"bound": "alu", "achieved": tf, "peak": fp64_pk, "unit": "TFLOP/s",
                         "frac": tf / fp64_pk, "hbm_gbs": achieved, "hbm_frac": achieved / peak_hbm,
                         "peak_source": fp64_peak_source(fp64_pk),
                         "algorithmic": "2 C n^2 nrhs = %.3e flop per launch (element matrices + gathered "
                                        "vectors = %.3e B)" % (flops, byt)})

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        verts_pin = torch.tensor(verts).pin_memory()
        fcg_pin = torch.tensor(fcg_h).pin_memory()
        x_pin = torch.zeros((nrhs, s.N), dtype=torch.float64).pin_memory()
        h2d = verts_pin.numel() * 8 + fcg_pin.numel() * 8
        d2h = s.N * nrhs * 8
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            verts_d.copy_(verts_pin, non_blocking=True)
            fcg.copy_(fcg_pin, non_blocking=True)
            s.update_geometry(verts_d)
            if nrhs == 1:
                s.load(fcg, b)
            else:
                b.copy_(fcg)
            x.zero_()
            s.solve(b, x, nrhs=nrhs)
            x_pin.copy_(x, non_blocking=True)
            torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": float(s.N) * nrhs * args.steps / te, "unit": "DOFs/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # the same workload with the plain FP64 solver (FP64 operator and FP64 patch solves)
    x_mixed = x.clone()  # the last step's solution, for the comparison with the plain FP64 solver
    plain = None
    if (wl["prec"] != 0 or wl.get("a32", 0)) and not args.no_fp64_plain:
        s64, step64, it64, rr64, _, _, _, x64 = make(0, 0)
        # the plain solver is several times slower: fewer steps keep the run within minutes
        psteps = min(args.steps, wl.get("plain_steps", args.steps))
        for _ in range(min(args.warmup, 1 if psteps < args.steps else args.warmup)):
            step64()
        per64 = timed(step64, psteps)
        ms64, _ = combine_ranks(sum(per64), s64.N, dist, device="cuda")
        dx = [float(torch.linalg.norm(x_mixed[k] - x64[k]) / torch.linalg.norm(x64[k])) for k in range(nrhs)]
        plain = {"value": ntot * nrhs * psteps / (ms64 / 1e3), "unit": "DOFs/s",
                 "steps": psteps, "ms_per_step": ms64 / psteps,
                 "latency_p50_ms": float(np.percentile(per64, 50)),
                 "latency_p99_ms": float(np.percentile(per64, 99)),
                 "iterations": statistics.median(it64[-psteps:]), "max_relres": max(rr64[-psteps:]),
                 "max_rel_l2_diff_of_solutions": max(dx),
                 "config": "same mesh, right-hand side and rtol; FP64 operator and FP64 patch solves"}
        s64.close()

    # the same workload with the paper's finer decomposition for the space (Hiptmair-Toselli for H(curl),
    # PAFW_1 edge stars for H(div)): same mesh, right-hand side, precisions and rtol
    # other configurations of the same workload: the paper's finer decomposition for the space when the main
    # line uses vertex stars (Hiptmair-Toselli for H(curl), PAFW_1 edge stars for H(div)), the hybrid form, and
    # whatever the workload lists (e.g. the previous default); same mesh, right-hand sides, precisions and rtol
    variants = {}
    main_decomp = args.decomposition or wl.get("decomposition", "vertex_star")
    vlist = []
    alt = {"N1curl": "ht", "RT": "edge_star"}.get(wl["space"])
    if alt and alt != main_decomp:
        vlist.append((alt, dict(decomposition=alt)))
    vlist += wl.get("variants", [])
    for vname, vkw in ([] if args.no_variants else vlist):
        sv, stepv, itv, rrv, *_ = make(vkw.get("prec", wl["prec"]), vkw.get("a32", wl.get("a32", 0)),
                                       vkw.get("decomposition"), vkw.get("form"))
        for _ in range(args.warmup):
            stepv()
        sv.profile(True)
        stepv()
        torch.cuda.synchronize()
        profv = sv.profile_read()
        sv.profile(False)
        vsteps = min(args.steps, vkw.get("steps", args.steps))
        perv = timed(stepv, vsteps)
        msv, _ = combine_ranks(sum(perv), sv.N, dist, device="cuda")
        kv = {k: v[0] for k, v in profv.items()}
        variants[vname] = {"value": ntot * nrhs * vsteps / (msv / 1e3), "unit": "DOFs/s",
                           "steps": vsteps, "ms_per_step": msv / vsteps,
                           "latency_p50_ms": float(np.percentile(perv, 50)),
                           "latency_p99_ms": float(np.percentile(perv, 99)),
                           "iterations": statistics.median(itv[-vsteps:]), "max_relres": max(rrv[-vsteps:]),
                           "largest_patch": int(np.diff(sv.patch_map()[0]).max()),
                           "kernel_ms_per_step": {k: round(v, 4) for k, v in kv.items() if v > 0},
                           "pcg_loop": args.pcg_loop,
                           "config": "same mesh, right-hand sides and rtol; " + ", ".join(
                               "%s %s" % kv_ for kv_ in sorted(vkw.items()))}
        sv.close()

    cb = err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(wl, args)

        def small_solver(v, c):
            return rz.Riesz(wl["space"], wl["p"], v, c, precond_precision=wl["prec"], nrhs_max=nrhs,
                            apply_precision=wl.get("a32", 0), **solver_opts(wl, args))
        err = err_vs_oracle(wl, args, small_solver)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "DOFs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32+bf16" if wl.get("a32", 0) == 2 else ("f64" if wl["prec"] == 0 and not wl.get("a32", 0)
                                                                   else "f64+f32"),
            "data": "synthetic",
            "config": {"workload": wl["label"], "space": wl["space"], "p": wl["p"], "cells": C, "dofs": s.N,
                       "nrhs": nrhs, "apply_precision": {0: "fp64", 1: "fp32", 2: "bf16x3 tensor cores"}[
                           wl.get("a32", 0)],
                       "precond_precision": "fp32" if wl["prec"] == 1 else "fp64",
                       "rtol": 1e-8, "step": "device setup + load + PCG solve",
                       "pcg_loop": loop_driver, "decomposition": main_decomp,
                       "form": args.form or wl.get("form", "additive"),
                       "coarse_solve": {0: "none", 1: "dense inverse", 2: "lowest-order PCG"}[
                           s.tuning()["coarse_mode"]] if "coarse_mode" in s.tuning() else None,
                       "autotuned": s.tuning(),
                       "l2": "inputs larger than L2 (element matrices and patch factors)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "iterations": statistics.median(iters[-args.steps:]), "max_relres": relres,
            "latency_p50_ms": float(np.percentile(per_step, 50)),
            "latency_p99_ms": float(np.percentile(per_step, 99)),
            "err_vs_oracle": err,
            "fp64_plain": plain,
            "speedup_vs_fp64_plain": (value / plain["value"]) if plain else None,
            "decomposition_variants": variants,
            "setup_kernel_ms": sum(k_ms[k] for k in setup_kinds if k not in SIDE_STREAM_KINDS),
            "solve_kernel_ms": sum(v for k, v in k_ms.items() if k not in setup_kinds and k not in SIDE_STREAM_KINDS),
            "kernel_ms_per_step": {k: round(v, 4) for k, v in k_ms.items() if v > 0},
            "kernel_ms_per_step_source": "one untimed step before the timed region with every kernel bracketed "
                                         "by CUDA events (host-driven PCG loop); coarse and coarse_apply run on "
                                         "a side stream beside cholesky and patch_solve, so their spans overlap",
            "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
