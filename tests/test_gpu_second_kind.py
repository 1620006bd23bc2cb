"""GPU parity for the second-kind solution spaces NedTwo_p and BDM_p (Eq. (2.6)) through the C ABI against
the oracle: operator products (element matrices, matrix-free, BF16x3 tensor cores), the preconditioners
(vertex stars, Hiptmair-Toselli with CG_{p+1} potentials, PAFW_1 edge stars, W^k by the Whitney DOFs) and
solves against the oracle's direct solve."""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle.mesh import MeshDofs
from oracle.refelem import reference_element
from paper_2506_17406_gb300 import riesz as rz
from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_coeffs, normal_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_SYS = {}


def system(space, p, n, seed=3, alpha=1.0, beta=1.0):
    key = (space, p, n, seed, alpha, beta)
    if key not in _SYS:
        verts, cells = kuhn_mesh(n, 0.1, seed)
        ref = reference_element(space, p)
        md = MeshDofs(verts, cells, ref)
        A = asm.assemble(md, asm.element_matrices(ref, verts, cells, alpha=alpha, beta=beta)).tocsr()
        _SYS[key] = (verts, cells, md, A)
    return _SYS[key]


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = [("N2curl", 1, 3), ("N2curl", 2, 3), ("N2curl", 4, 2), ("BDM", 1, 3), ("BDM", 2, 3), ("BDM", 4, 2)]


@pytest.mark.parametrize("mode", [rz.APPLY_ELEMENT, rz.APPLY_MATRIX_FREE])
@pytest.mark.parametrize("space,p,n", CASES)
def test_apply_matches_oracle(space, p, n, mode):
    verts, cells, md, A = system(space, p, n)
    s = rz.Riesz(space, p, verts, cells, apply_mode=mode, nrhs_max=2)
    assert s.N == md.ndofs and np.array_equal(s.dof_map(), md.cell_dofs)
    X = normal_coeffs((2, s.N), 11)
    y = torch.zeros((2, s.N), dtype=torch.float64, device="cuda")
    s.apply(dev(X), y, nrhs=2)
    Y = host(y)
    for r in range(2):
        ye = A @ X[r]
        assert np.abs(Y[r] - ye).max() <= 1e-11 * np.abs(ye).max()


@pytest.mark.parametrize("space,p", [("N2curl", 9), ("BDM", 10)])
def test_high_degree_apply_matches_oracle(space, p):
    """n_ref = 660 / 858 on one cube (6 cells): the element matrices and the two-CTA tensor-core split."""
    verts, cells, md, A = system(space, p, 1)
    for prec, tol in ((rz.PREC_FP64, 1e-8), (rz.PREC_BF16X3, 2e-4)):
        s = rz.Riesz(space, p, verts, cells, apply_precision=prec, nrhs_max=2)
        X = normal_coeffs((2, s.N), 12)
        y = torch.zeros((2, s.N), dtype=torch.float64, device="cuda")
        s.apply_prec(dev(X), y, prec, nrhs=2)
        Y = host(y)
        for r in range(2):
            ye = A @ X[r]
            assert np.abs(Y[r] - ye).max() <= tol * np.abs(ye).max(), (prec, r)


@pytest.mark.parametrize("prec,tol", [(rz.PREC_FP64, 1e-10), (rz.PREC_FP32, 1e-4)])
@pytest.mark.parametrize("space,p,n", CASES)
def test_vertex_star_precond_matches_oracle(space, p, n, prec, tol):
    verts, cells, md, A = system(space, p, n)
    s = rz.Riesz(space, p, verts, cells, precond_precision=prec)
    P = asm.TwoLevelPreconditioner(A, md)
    r = normal_vector(s.N, 5)
    z = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    s.precond(dev(r), z)
    ze = P.apply(r)
    assert np.abs(host(z) - ze).max() <= tol * np.abs(ze).max()


@pytest.mark.parametrize("prec,tol", [(rz.PREC_FP64, 1e-10), (rz.PREC_FP32, 1e-4)])
@pytest.mark.parametrize("p,n", [(1, 3), (2, 3), (3, 2)])
def test_ht_precond_matches_oracle(p, n, prec, tol):
    """NedTwo_p with Hiptmair-Toselli: the gradient potentials are CG_{p+1} (the space's X^0)."""
    verts, cells, md, A = system("N2curl", p, n)
    mc = MeshDofs(verts, cells, reference_element("CG", p + 1))
    s = rz.Riesz("N2curl", p, verts, cells, decomposition=rz.DECOMP_HT, precond_precision=prec, nrhs_max=8)
    P = asm.HTPreconditioner(A, md, mc)
    R = normal_coeffs((8, s.N), 5)
    Z = torch.zeros((8, s.N), dtype=torch.float64, device="cuda")
    s.precond(dev(R), Z, nrhs=8)
    Zh = host(Z)
    A0 = A[P.W][:, P.W].toarray()
    for k in range(8):
        ze = P.apply(R[k])
        assert np.abs(Zh[k] - ze).max() <= tol * np.abs(ze).max(), k


@pytest.mark.parametrize("prec,tol", [(rz.PREC_FP64, 1e-10), (rz.PREC_FP32, 1e-4)])
@pytest.mark.parametrize("p,n,nr", [(1, 3, 1), (3, 2, 8), (5, 2, 5)])
def test_edge_star_precond_matches_oracle(p, n, nr, prec, tol):
    verts, cells, md, A = system("BDM", p, n)
    s = rz.Riesz("BDM", p, verts, cells, decomposition=rz.DECOMP_EDGE_STAR, precond_precision=prec, nrhs_max=nr)
    P = asm.TwoLevelPreconditioner(A, md, asm.edge_star_dofs(md))
    R = normal_coeffs((nr, s.N), 6)
    Z = torch.zeros((nr, s.N), dtype=torch.float64, device="cuda")
    s.precond(dev(R), Z, nrhs=nr)
    Zh = host(Z)
    for k in range(nr):
        ze = P.apply(R[k])
        assert np.abs(Zh[k] - ze).max() <= tol * np.abs(ze).max(), k


@pytest.mark.parametrize("space,p,n,decomp", [("N2curl", 2, 3, rz.DECOMP_VERTEX_STAR), ("N2curl", 3, 2, rz.DECOMP_HT),
                                              ("BDM", 2, 3, rz.DECOMP_VERTEX_STAR), ("BDM", 3, 2, rz.DECOMP_EDGE_STAR)])
def test_solve_matches_direct_solve(space, p, n, decomp):
    """FP64 path: 1e-10 relative L2 against the oracle's sparse direct solve."""
    verts, cells, md, A = system(space, p, n)
    s = rz.Riesz(space, p, verts, cells, decomposition=decomp, rtol=1e-13, maxit=5000)
    b = normal_vector(s.N, 8)
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    iters, relres, rc = s.solve(dev(b), x)
    assert rc == 0 and relres[0] <= 1e-13
    xe = asm.direct_solve(A, b)
    assert np.linalg.norm(host(x) - xe) <= 1e-10 * np.linalg.norm(xe)


@pytest.mark.parametrize("space,p,n,decomp", [("N2curl", 3, 2, rz.DECOMP_HT), ("BDM", 3, 2, rz.DECOMP_EDGE_STAR),
                                              ("BDM", 6, 1, rz.DECOMP_EDGE_STAR)])
def test_mixed_precision_solve_error_against_oracle(space, p, n, decomp):
    """BF16x3 products, FP32 patch sweeps, FP64 residual replacement, 8 right-hand sides in lockstep: every
    relative residual measured with the oracle's matrix is within 2e-11 (the solver stops at 1e-11 measured
    with its own FP64 operator, which agrees with the oracle's to about 1e-11 relative at p = 6), and the
    error against the oracle's direct solve is below 1e-8 relative L2."""
    verts, cells, md, A = system(space, p, n)
    s = rz.Riesz(space, p, verts, cells, decomposition=decomp, precond_precision=rz.PREC_FP32,
                 apply_precision=rz.PREC_BF16X3, nrhs_max=8, rtol=1e-11, maxit=3000)
    B = normal_coeffs((8, s.N), 9)
    X = torch.zeros((8, s.N), dtype=torch.float64, device="cuda")
    it, rr, rc = s.solve(dev(B), X, nrhs=8)
    assert rc == 0
    Xh = host(X)
    for k in range(8):
        assert np.linalg.norm(B[k] - A @ Xh[k]) <= 2e-11 * np.linalg.norm(B[k])
        xe = asm.direct_solve(A, B[k])
        assert np.linalg.norm(Xh[k] - xe) <= 1e-8 * np.linalg.norm(xe), k


def test_lowest_order_coarse_route_matches_dense_coarse():
    """W^k above the dense limit goes through the Ned1_1 / RT_1 handle (the Whitney forms, Lemma 4.1): with
    coarse = 2 (forced lowest-order PCG steps) the solve still reaches the oracle's solution."""
    for space, decomp in (("N2curl", rz.DECOMP_VERTEX_STAR), ("BDM", rz.DECOMP_EDGE_STAR)):
        verts, cells, md, A = system(space, 2, 3)
        s = rz.Riesz(space, 2, verts, cells, decomposition=decomp, coarse=2, rtol=1e-12, maxit=3000)
        assert s.tuning()["coarse_mode"] == 2
        b = normal_vector(s.N, 4)
        x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
        it, rr, rc = s.solve(dev(b), x)
        assert rc == 0
        xe = asm.direct_solve(A, b)
        assert np.linalg.norm(host(x) - xe) <= 1e-9 * np.linalg.norm(xe)


@pytest.mark.parametrize("space,p,n,decomp", [("N2curl", 2, 3, rz.DECOMP_HT), ("BDM", 2, 3, rz.DECOMP_EDGE_STAR),
                                              ("N2curl", 3, 2, rz.DECOMP_VERTEX_STAR)])
def test_hybrid_precond_matches_oracle(space, p, n, decomp):
    """The paper's hybrid sweep on the second-kind spaces, with the oracle's weights set on the handle and
    W^k converged on the lowest-order problem (200 PCG steps): 1e-9 against the oracle's sweep."""
    verts, cells, md, A = system(space, p, n)
    iface, patches = None, None
    if decomp == rz.DECOMP_HT:
        mc = MeshDofs(verts, cells, reference_element("CG", p + 1))
        iface = asm.HTPreconditioner(A, md, mc, weight=0.0)
    elif decomp == rz.DECOMP_EDGE_STAR:
        patches = asm.edge_star_dofs(md)
    H = asm.HybridPreconditioner(A, md, patches, coarse=True, interface=iface)
    s = rz.Riesz(space, p, verts, cells, form=rz.FORM_HYBRID, coarse=2, coarse_its=200, decomposition=decomp,
                 nrhs_max=2)
    s.hybrid_weights([H.rho.get(1, 1.0), H.rho[2], H.rho.get(3, 1.0)])
    R = normal_coeffs((2, s.N), 5)
    Z = torch.zeros((2, s.N), dtype=torch.float64, device="cuda")
    s.precond(dev(R), Z, nrhs=2)
    Zh = host(Z)
    for k in range(2):
        ze = H.apply(R[k])
        assert np.abs(Zh[k] - ze).max() <= 1e-9 * np.abs(ze).max(), k


@pytest.mark.parametrize("space,p,n", [("N2curl", 2, 3), ("BDM", 2, 3)])
def test_dirichlet_solve_matches_oracle(space, p, n):
    """Homogeneous Dirichlet conditions on the whole boundary (Eq. (2.8)): the fixed set equals the oracle's
    bit for bit and the solve of the free DOFs matches the oracle's direct solve to 1e-10."""
    verts, cells, md, A = system(space, p, n)
    s = rz.Riesz(space, p, verts, cells, dirichlet=1, rtol=1e-13, maxit=3000)
    D = asm.dirichlet_dofs(md)
    mask = s.dirichlet_map().astype(bool)
    assert np.array_equal(np.nonzero(mask)[0], D)
    b = normal_vector(s.N, 6)
    b[D] = 0.0
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    it, rr, rc = s.solve(dev(b), x)
    assert rc == 0
    xe = asm.direct_solve(asm.constrained(A, D), b)
    assert np.linalg.norm(host(x) - xe) <= 1e-10 * np.linalg.norm(xe)
