"""Homogeneous Dirichlet conditions on the whole boundary (X_{p,D} of Eq. (2.8)) against the oracle."""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle.mesh import MeshDofs
from oracle.polys import quadrature
from oracle.refelem import reference_element
from paper_2506_17406_gb300 import riesz as rz
from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_coeffs, normal_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("CG", 3, 3, 0.1), ("N1curl", 3, 3, 0.1), ("RT", 3, 3, 0.1), ("N1curl", 2, 4, 0.1)]


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def setup(space, p, n, amp):
    verts, cells = kuhn_mesh(n, amp, 3)
    ref = reference_element(space, p)
    md = MeshDofs(verts, cells, ref)
    A = asm.assemble(md, asm.element_matrices(ref, verts, cells))
    D = asm.dirichlet_dofs(md)
    return verts, cells, ref, md, A, D


@pytest.mark.parametrize("space,p,n,amp", CASES)
def test_dirichlet_apply_precond_solve(space, p, n, amp):
    verts, cells, ref, md, A, D = setup(space, p, n, amp)
    Ac = asm.constrained(A, D)
    for coarse in (0, 1):
        s = rz.Riesz(space, p, verts, cells, dirichlet=1, coarse=coarse, rtol=1e-13, maxit=3000)
        x = normal_vector(s.N, 5)
        y = torch.zeros(s.N, dtype=torch.float64, device="cuda")
        s.apply(dev(x), y)
        ye = Ac @ x
        assert np.abs(host(y) - ye).max() <= 1e-11 * np.abs(ye).max()
        z = torch.zeros_like(y)
        s.precond(dev(x), z)
        P = asm.DirichletPreconditioner(A, md, D, two_level=bool(coarse))
        ze = P.apply(x)
        tol = 1e-10
        assert np.abs(host(z) - ze).max() <= tol * np.abs(ze).max()
        b = normal_vector(s.N, 6)
        b[D] = 0.0
        xs = torch.zeros_like(y)
        it, rr, rc = s.solve(dev(b), xs)
        assert rc == 0
        xh = host(xs)
        assert np.all(xh[D] == 0.0)
        xe = asm.direct_solve(Ac, b)
        assert np.linalg.norm(xh - xe) <= 1e-10 * np.linalg.norm(xe)


def test_dirichlet_load_zeroes_fixed_rows():
    verts, cells, ref, md, A, D = setup("N1curl", 3, 3, 0.1)
    s = rz.Riesz("N1curl", 3, verts, cells, dirichlet=1)
    s0 = rz.Riesz("N1curl", 3, verts, cells)
    f = normal_coeffs((3, s.n_cg), 2)
    b = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    b0 = torch.zeros_like(b)
    s.load(dev(f), b)
    s0.load(dev(f), b0)
    bh, b0h = host(b), host(b0)
    assert np.all(bh[D] == 0.0)
    free = np.setdiff1d(np.arange(s.N), D)
    assert np.array_equal(bh[free], b0h[free])


def test_dirichlet_manufactured_bubble_cg6():
    """u = xyz(1-x)(1-y)(1-z) lies in CG_6 with zero trace: the library's constrained solve reproduces it."""
    verts, cells = kuhn_mesh(1, 0.0, 1)
    ref = reference_element("CG", 6)
    md = MeshDofs(verts, cells, ref)
    D = asm.dirichlet_dofs(md)

    def u(x):
        return (x[:, 0] * (1 - x[:, 0]) * x[:, 1] * (1 - x[:, 1]) * x[:, 2] * (1 - x[:, 2]))[:, None]

    def gu(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        bx, by, bz = X * (1 - X), Y * (1 - Y), Z * (1 - Z)
        return np.stack([(1 - 2 * X) * by * bz, bx * (1 - 2 * Y) * bz, bx * by * (1 - 2 * Z)], 1)

    b = asm.load_function(ref, md, u, gu)
    b[D] = 0.0
    s = rz.Riesz("CG", 6, verts, cells, dirichlet=1, rtol=1e-13, maxit=2000)
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    _, rr, rc = s.solve(dev(b), x)
    assert rc == 0
    X, _ = quadrature(3, 3)
    xq, val = asm.evaluate(ref, md, host(x), X)
    ue = u(xq.reshape(-1, 3)).reshape(val.shape)
    assert np.abs(val - ue).max() <= 1e-9 * np.abs(ue).max()


@pytest.mark.parametrize("space,p", [("CG", 3), ("N1curl", 3), ("RT", 3)])
def test_partial_dirichlet_apply_precond_solve(space, p):
    """Gamma_D = the faces x = 0 and y = 0 (a proper part of the boundary, Eq. (2.8)), the rest Neumann:
    apply, preconditioner (one- and two-level) and solve against the oracle's constrained system."""
    verts, cells = kuhn_mesh(3, 0.1, 3)
    mask = (np.isclose(verts[:, 0], 0.0) | np.isclose(verts[:, 1], 0.0)).astype(np.uint8)
    ref = reference_element(space, p)
    md = MeshDofs(verts, cells, ref)
    A = asm.assemble(md, asm.element_matrices(ref, verts, cells))
    D = asm.dirichlet_dofs(md, vertex_mask=mask)
    Ac = asm.constrained(A, D)
    for coarse in (0, 1):
        s = rz.Riesz(space, p, verts, cells, dirichlet=1, dirichlet_vertices=mask, coarse=coarse, rtol=1e-13,
                     maxit=3000)
        assert np.array_equal(np.nonzero(s.dirichlet_map())[0], D)
        x = normal_vector(s.N, 5)
        y = torch.zeros(s.N, dtype=torch.float64, device="cuda")
        s.apply(dev(x), y)
        ye = Ac @ x
        assert np.abs(host(y) - ye).max() <= 1e-11 * np.abs(ye).max()
        z = torch.zeros_like(y)
        s.precond(dev(x), z)
        P = asm.DirichletPreconditioner(A, md, D, two_level=bool(coarse))
        ze = P.apply(x)
        tol = 1e-10
        assert np.abs(host(z) - ze).max() <= tol * np.abs(ze).max()
        b = normal_vector(s.N, 6)
        b[D] = 0.0
        xs = torch.zeros_like(y)
        it, rr, rc = s.solve(dev(b), xs)
        assert rc == 0
        xh = host(xs)
        assert np.all(xh[D] == 0.0)
        xe = asm.direct_solve(Ac, b)
        assert np.linalg.norm(xh - xe) <= 1e-10 * np.linalg.norm(xe)
