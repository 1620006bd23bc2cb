"""Device-driven PCG loop (CUDA graph with a WHILE node) and batched solves.

The graph-driven loop runs the same kernels in the same order as the
host-driven loop, so iterates, iteration counts and residuals must be bitwise
equal; riesz_solve_batch must give every system the result it gets alone.
"""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle.mesh import MeshDofs
from oracle.refelem import reference_element
from paper_2506_17406_gb300 import riesz as rz
from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


# space, p, n, perturbation, options, right-hand sides
LOOP_CASES = [
    ("CG", 3, 4, 0.0, dict(), 1),
    ("N1curl", 3, 3, 0.1, dict(precond_precision=rz.PREC_FP32), 1),
    ("RT", 3, 3, 0.1, dict(precond_precision=rz.PREC_FP32, apply_precision=rz.PREC_FP32), 3),
    ("N1curl", 2, 3, 0.1, dict(apply_mode=rz.APPLY_MATRIX_FREE), 2),
    # the lowest-order coarse route (its PCG steps inside every preconditioner application)
    ("RT", 2, 3, 0.1, dict(decomposition=rz.DECOMP_EDGE_STAR, coarse=2, precond_precision=rz.PREC_FP32), 2),
]


def solve_with(loop, space, p, n, amp, opts, nrhs, rtol=1e-10, maxit=1000, b=None):
    verts, cells = kuhn_mesh(n, amp, 3)
    s = rz.Riesz(space, p, verts, cells, nrhs_max=nrhs, rtol=rtol, maxit=maxit, loop=loop, **opts)
    if b is None:
        b = np.stack([normal_vector(s.N, 20 + k) for k in range(nrhs)])
    x = torch.zeros((nrhs, s.N), dtype=torch.float64, device="cuda")
    l0 = s.stats()["launches"]
    it, rr, rc = s.solve(dev(b), x, nrhs=nrhs, check=False)
    launches = s.stats()["launches"] - l0
    out = host(x)
    s.close()
    return out, it, rr, rc, launches


@pytest.mark.parametrize("space,p,n,amp,opts,nrhs", LOOP_CASES)
def test_graph_loop_equals_host_loop(space, p, n, amp, opts, nrhs):
    xg, itg, rrg, rcg, lg = solve_with(rz.LOOP_GRAPH, space, p, n, amp, opts, nrhs)
    xh, ith, rrh, rch, lh = solve_with(rz.LOOP_HOST, space, p, n, amp, opts, nrhs)
    assert rcg == 0 and rch == 0
    assert np.array_equal(itg, ith)
    assert np.array_equal(rrg, rrh)
    assert np.array_equal(xg, xh)
    assert np.all(rrg <= 1e-10)


def test_graph_loop_launch_count():
    """The launch counter follows the passes of the graph loop: one control kernel
    per iteration more than the host loop, which also runs one speculative
    preconditioner step (patch sweeps + gather) after the last iteration."""
    _, itg, _, _, lg = solve_with(rz.LOOP_GRAPH, "CG", 3, 4, 0.0, dict(coarse=0), 1)
    _, ith, _, _, lh = solve_with(rz.LOOP_HOST, "CG", 3, 4, 0.0, dict(coarse=0), 1)
    assert itg[0] == ith[0] > 0
    assert lg == lh + int(itg[0]) - 2


@pytest.mark.parametrize("loop", [rz.LOOP_GRAPH, rz.LOOP_HOST])
def test_iteration_limit(loop):
    x5, it5, rr5, rc5, _ = solve_with(loop, "N1curl", 3, 3, 0.1, {}, 1, maxit=5)
    assert rc5 == 4 and it5[0] == 5 and rr5[0] > 1e-10
    x0, it0, rr0, rc0, _ = solve_with(loop, "N1curl", 3, 3, 0.1, {}, 1, maxit=0)
    assert rc0 == 4 and it0[0] == 0 and np.all(x0 == 0.0)
    assert abs(rr0[0] - 1.0) < 1e-14  # x = 0: the relative residual is 1


def test_iteration_limit_same_in_both_loops():
    xg, itg, rrg, rcg, _ = solve_with(rz.LOOP_GRAPH, "RT", 3, 3, 0.1,
                                      dict(precond_precision=rz.PREC_FP32, apply_precision=rz.PREC_FP32), 2,
                                      maxit=7)
    xh, ith, rrh, rch, _ = solve_with(rz.LOOP_HOST, "RT", 3, 3, 0.1,
                                      dict(precond_precision=rz.PREC_FP32, apply_precision=rz.PREC_FP32), 2,
                                      maxit=7)
    assert rcg == rch == 4
    assert np.array_equal(itg, ith) and np.array_equal(rrg, rrh) and np.array_equal(xg, xh)


def test_graph_loop_nonfinite_rhs():
    verts, cells = kuhn_mesh(2, 0.0, 1)
    s = rz.Riesz("CG", 2, verts, cells)
    b = normal_vector(s.N, 4)
    b[3] = np.nan
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    _, _, rc = s.solve(dev(b), x, check=False)
    assert rc == 5


def test_profiler_on_loop_kernels_uses_host_loop():
    """While the profiler times loop kernels the host loop runs; same result."""
    verts, cells = kuhn_mesh(3, 0.1, 3)
    s = rz.Riesz("N1curl", 3, verts, cells, rtol=1e-10)
    b = dev(normal_vector(s.N, 20))
    x1 = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    it1, _, _ = s.solve(b, x1)
    s.profile(True, kinds=["apply"])
    x2 = torch.zeros_like(x1)
    it2, _, _ = s.solve(b, x2)
    prof = s.profile_read()
    s.profile(False)
    assert prof["apply"][1] >= it2[0]  # every iteration's product was timed
    assert it1[0] == it2[0]
    assert torch.equal(x1, x2)


# ---------------------------------------------------------------------------
BATCH = [  # space, p, n, perturbation, options, right-hand sides
    ("CG", 2, 3, 0.1, dict(), 1),
    ("N1curl", 3, 2, 0.1, dict(precond_precision=rz.PREC_FP32), 1),
    ("RT", 2, 3, 0.1, dict(), 2),
    ("CG", 4, 2, 0.0, dict(precond_precision=rz.PREC_FP32), 1),
    ("RT", 3, 2, 0.1, dict(precond_precision=rz.PREC_FP32, apply_precision=rz.PREC_FP32), 3),
    ("N1curl", 1, 4, 0.1, dict(apply_mode=rz.APPLY_MATRIX_FREE), 1),
]


def make_batch(cases, rtol=1e-10, maxits=None):
    solvers, bs, xs, nr = [], [], [], []
    for i, (space, p, n, amp, opts, nrhs) in enumerate(cases):
        verts, cells = kuhn_mesh(n, amp, 10 + i)
        maxit = 1000 if maxits is None else maxits[i]
        s = rz.Riesz(space, p, verts, cells, nrhs_max=nrhs, rtol=rtol, maxit=maxit, **opts)
        solvers.append(s)
        bs.append(dev(np.stack([normal_vector(s.N, 100 * i + k) for k in range(nrhs)])))
        xs.append(torch.zeros((nrhs, s.N), dtype=torch.float64, device="cuda"))
        nr.append(nrhs)
    return solvers, bs, xs, nr


def test_batch_equals_individual_solves():
    solvers, bs, xs, nr = make_batch(BATCH)
    iters, relres, status = rz.solve_batch(solvers, bs, xs, nrhs=nr)
    assert np.all(status == 0)
    off = 0
    for s, b, x, k in zip(solvers, bs, xs, nr):
        xi = torch.zeros_like(x)
        it, rr, _ = s.solve(b, xi, nrhs=k)
        assert np.array_equal(iters[off:off + k], it)
        assert np.array_equal(relres[off:off + k], rr)
        assert torch.equal(x, xi)
        off += k
    assert np.all(relres <= 1e-10)


def test_repeated_solves_are_bitwise_equal():
    """A solve depends only on its inputs: two solves in a row give bitwise the same iterates, also with the
    lowest-order coarse route, whose PCG steps start every application from the residual alone."""
    for opts in (dict(decomposition=rz.DECOMP_EDGE_STAR, coarse=2, precond_precision=rz.PREC_FP32),
                 dict(coarse=2), dict(decomposition=rz.DECOMP_EDGE_STAR, form=rz.FORM_HYBRID)):
        verts, cells = kuhn_mesh(3, 0.1, 18)
        s = rz.Riesz("RT", 2, verts, cells, rtol=1e-10, **opts)
        b = dev(normal_vector(s.N, 800).reshape(1, -1))
        out = []
        for _ in range(2):
            x = torch.zeros_like(b)
            it, rr, rc = s.solve(b, x)
            assert rc == 0
            out.append((host(x), int(it[0]), float(rr[0])))
        assert np.array_equal(out[0][0], out[1][0]) and out[0][1:] == out[1][1:], opts


def test_batched_setup_equals_individual_setups():
    """riesz_update_geometry_batch (every system's device setup on its own stream, joined once) gives every
    system bitwise the factors of its own riesz_update_geometry: the solves after either setup are equal
    bit for bit (mixed spaces, Hiptmair-Toselli, edge stars, hybrid form, the lowest-order coarse route)."""
    cases = BATCH + [("N1curl", 3, 3, 0.1, dict(decomposition=rz.DECOMP_HT, precond_precision=rz.PREC_FP32), 1),
                     ("RT", 3, 3, 0.1, dict(decomposition=rz.DECOMP_EDGE_STAR, form=rz.FORM_HYBRID), 2),
                     ("RT", 2, 3, 0.1, dict(decomposition=rz.DECOMP_EDGE_STAR, coarse=2), 1)]
    solvers, bs, xs, nr = make_batch(cases)
    moved = [dev(kuhn_mesh(n, amp, 50 + i)[0]) for i, (_, _, n, amp, _, _) in enumerate(cases)]
    out = []
    for batched in (True, False):
        if batched:
            rz.update_geometry_batch(solvers, moved)
        else:
            for s, v in zip(solvers, moved):
                s.update_geometry(v)
        res = []
        for s, b, k in zip(solvers, bs, nr):
            x = torch.zeros((k, s.N), dtype=torch.float64, device="cuda")
            it, rr, rc = s.solve(b, x, nrhs=k)
            assert rc == 0
            res.append((host(x), it.copy(), rr.copy()))
        out.append(res)
    for (x1, i1, r1), (x2, i2, r2) in zip(*out):
        assert np.array_equal(x1, x2) and np.array_equal(i1, i2) and np.array_equal(r1, r2)


def test_batch_matches_oracle():
    cases = BATCH[:3]
    solvers, bs, xs, nr = make_batch(cases, rtol=1e-13)
    _, relres, status = rz.solve_batch(solvers, bs, xs, nrhs=nr)
    assert np.all(status == 0)
    for i, ((space, p, n, amp, _, k), b, x) in enumerate(zip(cases, bs, xs)):
        verts, cells = kuhn_mesh(n, amp, 10 + i)
        ref = reference_element(space, p)
        md = MeshDofs(verts, cells, ref)
        A = asm.assemble(md, asm.element_matrices(ref, verts, cells))
        B, X = host(b), host(x)
        for r in range(k):
            xe = asm.direct_solve(A, B[r])
            assert np.linalg.norm(X[r] - xe) <= 1e-10 * np.linalg.norm(xe)


def test_batch_reports_status_per_system():
    cases = BATCH[:3]
    solvers, bs, xs, nr = make_batch(cases, maxits=[1000, 3, 1000])
    iters, relres, status = rz.solve_batch(solvers, bs, xs, nrhs=nr)
    assert list(status) == [0, 4, 0]
    assert iters[1] == 3 and relres[1] > 1e-10
    assert relres[0] <= 1e-10 and np.all(relres[2:4] <= 1e-10)


def test_batch_rejects_repeated_handle_and_empty():
    solvers, bs, xs, nr = make_batch(BATCH[:1])
    with pytest.raises(rz.RieszError):
        rz.solve_batch([solvers[0], solvers[0]], [bs[0], bs[0]], [xs[0], xs[0]])
    iters, relres, status = rz.solve_batch([], [], [])
    assert len(iters) == 0 and len(status) == 0


def test_batch_of_mixed_draws_matches_oracle():
    """The batched configuration's recipe at oracle-sized meshes: seeded draws of
    space, degree and mesh, perturbed, random right-hand sides, FP32 products and
    patch sweeps with FP64 residuals, all systems in one graph launch; every
    solution against the oracle's sparse direct solve."""
    rng = np.random.Generator(np.random.PCG64(4))
    draws = [(str(rng.choice(["CG", "N1curl", "RT"])), int(rng.integers(2, 5)), int(rng.integers(2, 4)))
             for _ in range(16)]
    opts = dict(precond_precision=rz.PREC_FP32, apply_precision=rz.PREC_FP32, rtol=1e-10, maxit=5000)
    solvers, bs, xs, meshes = [], [], [], []
    for i, (space, p, n) in enumerate(draws):
        verts, cells = kuhn_mesh(n, 0.1, 1000 + i)
        s = rz.Riesz(space, p, verts, cells, **opts)
        solvers.append(s)
        meshes.append((verts, cells))
        bs.append(dev(normal_vector(s.N, 500 + i)).reshape(1, -1))
        xs.append(torch.zeros((1, s.N), dtype=torch.float64, device="cuda"))
    iters, relres, status = rz.solve_batch(solvers, bs, xs)
    assert np.all(status == 0) and np.all(relres <= 1e-10)
    for (space, p, n), (verts, cells), b, x in zip(draws, meshes, bs, xs):
        ref = reference_element(space, p)
        md = MeshDofs(verts, cells, ref)
        A = asm.assemble(md, asm.element_matrices(ref, verts, cells))
        bh = host(b)[0]
        xe = asm.direct_solve(A, bh)
        assert np.linalg.norm(A @ host(x)[0] - bh) <= 1.05e-10 * np.linalg.norm(bh)
        assert np.linalg.norm(host(x)[0] - xe) <= 1e-7 * np.linalg.norm(xe)
