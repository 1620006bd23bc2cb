"""The finer space decompositions against the oracle: Hiptmair-Toselli for H(curl) (Eq. (6.19)) and
PAFW_1 edge stars for H(div) (Eq. (6.24))."""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle.mesh import MeshDofs
from oracle.refelem import reference_element
from paper_2506_17406_gb300 import riesz as rz
from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_coeffs, normal_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def setup(p, n, amp=0.1, seed=3, alpha=1.0, beta=1.0):
    verts, cells = kuhn_mesh(n, amp, seed)
    rn, rc = reference_element("N1curl", p), reference_element("CG", p)
    mn, mc = MeshDofs(verts, cells, rn), MeshDofs(verts, cells, rc)
    A = asm.assemble(mn, asm.element_matrices(rn, verts, cells, alpha=alpha, beta=beta))
    return verts, cells, mn, mc, A


@pytest.mark.parametrize("p,n,alpha,beta", [(2, 3, 1.0, 1.0), (3, 3, 1.0, 1.0), (4, 2, 1.0, 1.0),
                                             (3, 3, 2.0, 0.5), (3, 3, 1e3, 1.0)])
def test_ht_precond_matches_oracle(p, n, alpha, beta):
    """The potential problems carry beta (G^T A G = beta times the CG stiffness), the edge stars
    and W^1 both coefficients."""
    verts, cells, mn, mc, A = setup(p, n, alpha=alpha, beta=beta)
    s = rz.Riesz("N1curl", p, verts, cells, decomposition=rz.DECOMP_HT, alpha=alpha, beta=beta)
    P = asm.HTPreconditioner(A, mn, mc)
    r = normal_vector(s.N, 5)
    z = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    s.precond(dev(r), z)
    ze = P.apply(r)
    tol = 1e-10 * max(1.0, alpha)
    assert np.abs(host(z) - ze).max() <= tol * np.abs(ze).max()


@pytest.mark.parametrize("prec", [rz.PREC_FP64, rz.PREC_FP32])
@pytest.mark.parametrize("p,n", [(3, 3), (2, 4)])
def test_ht_solve_matches_direct_solve(p, n, prec):
    verts, cells, mn, mc, A = setup(p, n)
    s = rz.Riesz("N1curl", p, verts, cells, decomposition=rz.DECOMP_HT, precond_precision=prec, rtol=1e-10,
                 maxit=3000)
    b = normal_vector(s.N, 8)
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    it, rr, rc = s.solve(dev(b), x)
    assert rc == 0
    xh = host(x)
    assert np.linalg.norm(b - A @ xh) <= 1.001e-10 * np.linalg.norm(b)
    xe = asm.direct_solve(A, b)
    assert np.linalg.norm(xh - xe) <= 1e-7 * np.linalg.norm(xe)
    _, it_o, _ = asm.pcg(A, b, asm.HTPreconditioner(A, mn, mc).apply, rtol=1e-10)
    assert int(it[0]) <= it_o + 3


def test_ht_graph_loop_equals_host_loop_and_lockstep():
    verts, cells, mn, mc, A = setup(3, 3)
    out = []
    for loop in (rz.LOOP_GRAPH, rz.LOOP_HOST):
        s = rz.Riesz("N1curl", 3, verts, cells, decomposition=rz.DECOMP_HT, loop=loop, nrhs_max=3,
                     precond_precision=rz.PREC_FP32, rtol=1e-10)
        B = normal_coeffs((3, s.N), 4)
        X = torch.zeros((3, s.N), dtype=torch.float64, device="cuda")
        it, rr, rc = s.solve(dev(B), X, nrhs=3)
        assert rc == 0 and np.all(rr <= 1e-10)
        out.append((host(X), it))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def setup_rt(p, n, amp=0.1, seed=3, alpha=1.0, beta=1.0):
    verts, cells = kuhn_mesh(n, amp, seed)
    ref = reference_element("RT", p)
    md = MeshDofs(verts, cells, ref)
    A = asm.assemble(md, asm.element_matrices(ref, verts, cells, alpha=alpha, beta=beta))
    return verts, cells, md, A


@pytest.mark.parametrize("p,n,alpha", [(1, 3, 1.0), (3, 3, 1.0), (5, 2, 1.0), (3, 3, 1e3)])
@pytest.mark.parametrize("prec,tol", [(rz.PREC_FP64, 1e-10), (rz.PREC_FP32, 1e-4)])
def test_edge_star_precond_matches_oracle(p, n, alpha, prec, tol):
    verts, cells, md, A = setup_rt(p, n, alpha=alpha)
    s = rz.Riesz("RT", p, verts, cells, decomposition=rz.DECOMP_EDGE_STAR, precond_precision=prec, alpha=alpha)
    P = asm.TwoLevelPreconditioner(A, md, asm.edge_star_dofs(md))
    r = normal_vector(s.N, 5)
    z = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    s.precond(dev(r), z)
    ze = P.apply(r)
    tol = tol * max(1.0, alpha if prec == rz.PREC_FP64 else 1.0)
    assert np.abs(host(z) - ze).max() <= tol * np.abs(ze).max()


@pytest.mark.parametrize("p,n,nr", [(5, 2, 3), (8, 2, 8)])
def test_edge_star_precond_several_rhs_matches_oracle(p, n, nr):
    """FP32 edge-star sweeps for several right-hand sides (one warp per patch of up to 8 tiles: RT_8 edge
    stars hold up to 216 DOFs), each column against the oracle's preconditioner."""
    verts, cells, md, A = setup_rt(p, n)
    s = rz.Riesz("RT", p, verts, cells, decomposition=rz.DECOMP_EDGE_STAR, precond_precision=rz.PREC_FP32,
                 nrhs_max=nr)
    P = asm.TwoLevelPreconditioner(A, md, asm.edge_star_dofs(md))
    R = normal_coeffs((nr, s.N), 7)
    Z = torch.zeros((nr, s.N), dtype=torch.float64, device="cuda")
    s.precond(dev(R), Z, nrhs=nr)
    Zh = host(Z)
    tol = 1e-4
    for k in range(nr):
        ze = P.apply(R[k])
        assert np.abs(Zh[k] - ze).max() <= tol * np.abs(ze).max(), k


def test_sweep_shape_autotuner():
    """The multi-RHS FP32 sweep shape for edge stars is picked by timing the candidates on the handle's own
    factors (one CTA per patch, or one warp per patch with 4 or 8 warps per block); without tuning the
    8-warp shape runs.  Both handles' preconditioners match the oracle's."""
    verts, cells, md, A = setup_rt(5, 2)
    P = asm.TwoLevelPreconditioner(A, md, asm.edge_star_dofs(md))
    R = normal_coeffs((8, md.ndofs), 3)
    for autotune in (1, 0):
        s = rz.Riesz("RT", 5, verts, cells, decomposition=rz.DECOMP_EDGE_STAR, precond_precision=rz.PREC_FP32,
                     nrhs_max=8, autotune=autotune)
        t = s.tuning()
        if autotune:
            assert t["sweep_shape"] in (0, 4, 8) and t["sweep_candidates_timed"] in (0, 3)
        else:
            assert t["sweep_shape"] == 8 and t["sweep_candidates_timed"] == 0
        Z = torch.zeros((8, s.N), dtype=torch.float64, device="cuda")
        s.precond(dev(R), Z, nrhs=8)
        Zh = host(Z)
        tol = 1e-4
        for k in range(8):
            ze = P.apply(R[k])
            assert np.abs(Zh[k] - ze).max() <= tol * np.abs(ze).max(), (autotune, k)
    s1 = rz.Riesz("RT", 5, verts, cells, precond_precision=rz.PREC_FP32, nrhs_max=8)  # vertex stars: n/a
    assert s1.tuning()["sweep_shape"] == -1


def test_edge_star_dirichlet_precond_matches_oracle():
    verts, cells, md, A = setup_rt(3, 3)
    s = rz.Riesz("RT", 3, verts, cells, decomposition=rz.DECOMP_EDGE_STAR, dirichlet=1)
    D = asm.dirichlet_dofs(md)
    P = asm.DirichletPreconditioner(A, md, D, patches=asm.edge_star_dofs(md))
    r = normal_vector(s.N, 6)
    z = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    s.precond(dev(r), z)
    ze = P.apply(r)
    tol = 1e-10
    assert np.abs(host(z) - ze).max() <= tol * np.abs(ze).max()


@pytest.mark.parametrize("nrhs", [1, 3])
def test_edge_star_solve_matches_direct_solve(nrhs):
    verts, cells, md, A = setup_rt(3, 3)
    s = rz.Riesz("RT", 3, verts, cells, decomposition=rz.DECOMP_EDGE_STAR, precond_precision=rz.PREC_FP32,
                 nrhs_max=nrhs, rtol=1e-10)
    B = normal_coeffs((nrhs, s.N), 8)
    X = torch.zeros((nrhs, s.N), dtype=torch.float64, device="cuda")
    it, rr, rc = s.solve(dev(B), X, nrhs=nrhs)
    assert rc == 0
    Xh = host(X)
    _, it_o, _ = asm.pcg(A, B[0], asm.TwoLevelPreconditioner(A, md, asm.edge_star_dofs(md)).apply, rtol=1e-10)
    for k in range(nrhs):
        assert np.linalg.norm(B[k] - A @ Xh[k]) <= 1.001e-10 * np.linalg.norm(B[k])
        xe = asm.direct_solve(A, B[k])
        assert np.linalg.norm(Xh[k] - xe) <= 1e-7 * np.linalg.norm(xe)
    assert int(it[0]) <= it_o + 3
