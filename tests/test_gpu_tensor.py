"""The BF16x3 tensor-core contraction (tcgen05, apply_precision = RIESZ_PREC_BF16X3): the matrix-free
operator of Section 6.4 on the tensor cores against the oracle's quadrature-assembled matrix, and the
mixed-precision solve built on it against the oracle's direct solve."""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle.mesh import MeshDofs
from oracle.refelem import reference_element
from paper_2506_17406_gb300 import riesz as rz
from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_coeffs, normal_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def system(space, p, n, seed=3):
    verts, cells = kuhn_mesh(n, 0.1, seed)
    ref = reference_element(space, p)
    md = MeshDofs(verts, cells, ref)
    A = asm.assemble(md, asm.element_matrices(ref, verts, cells)).tocsr()
    return verts, cells, md, A


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


# (space, p, cubes per edge, right-hand sides): n_ref from 4 to 715 (one and two N pieces of the MMA, and
# above 512 outputs the columns split over two CTAs), tiles of 128 cells (1 RHS) down to 16 cells x 8 RHS,
# ragged last tiles
CASES = [("CG", 1, 3, 1), ("CG", 3, 4, 2), ("N1curl", 3, 3, 3), ("RT", 3, 3, 8), ("N1curl", 6, 2, 8),
         ("RT", 8, 2, 8), ("RT", 8, 1, 1), ("CG", 8, 2, 4), ("N1curl", 8, 1, 5), ("N1curl", 9, 1, 3),
         ("RT", 10, 1, 2)]


@pytest.mark.parametrize("space,p,n,nr", CASES)
def test_tensor_apply_matches_oracle(space, p, n, nr):
    """y = A x on the tensor cores against the oracle's A x.  Every operand is split into two BF16
    parts (relative representation error 2^-17 each) and the three leading products are accumulated in
    FP32, so each product term carries a relative error of about 3 * 2^-16; summed over the Q n_ref
    terms of a row with the cancellation of the stiffness terms this stays below 2e-4 of the largest
    output entry.  The FP64 apply of the same handle agrees with the oracle to 1e-11."""
    verts, cells, md, A = system(space, p, n)
    s = rz.Riesz(space, p, verts, cells, apply_precision=rz.PREC_BF16X3, nrhs_max=nr)
    X = normal_coeffs((nr, s.N), 11)
    y = torch.zeros((nr, s.N), dtype=torch.float64, device="cuda")
    s.apply_prec(dev(X), y, rz.PREC_BF16X3, nrhs=nr)
    Y = y.cpu().numpy()
    y64 = torch.zeros_like(y)
    s.apply(dev(X), y64, nrhs=nr)
    Y64 = y64.cpu().numpy()
    tol64 = 1e-11 if p <= 5 else (1e-10 if p <= 8 else 1e-8)  # basis agreement by degree
    for r in range(nr):
        ye = A @ X[r]
        assert np.abs(Y64[r] - ye).max() <= tol64 * np.abs(ye).max()
        err = np.abs(Y[r] - ye).max() / np.abs(ye).max()
        assert err <= 2e-4, (r, err)
        assert np.linalg.norm(Y[r] - ye) <= 5e-5 * np.linalg.norm(ye)


def test_tensor_apply_dirichlet_and_repeatable():
    """With a Dirichlet mask the fixed entries of x are read as zero and the fixed rows carry the identity,
    as in the FP64 apply; two applications give bitwise the same result (fixed accumulation order)."""
    verts, cells, md, A = system("N1curl", 3, 3)
    s = rz.Riesz("N1curl", 3, verts, cells, apply_precision=rz.PREC_BF16X3, dirichlet=1)
    x = dev(normal_vector(s.N, 2))
    y1 = torch.zeros_like(x)
    y2 = torch.zeros_like(x)
    y64 = torch.zeros_like(x)
    s.apply_prec(x, y1, rz.PREC_BF16X3)
    s.apply_prec(x, y2, rz.PREC_BF16X3)
    s.apply(x, y64)
    assert torch.equal(y1, y2)
    fixed = torch.tensor(s.dirichlet_map().astype(bool), device="cuda")
    assert torch.equal(y1[fixed], x[fixed])
    assert float((y1 - y64).abs().max()) <= 2e-4 * float(y64.abs().max())


@pytest.mark.parametrize("form", [rz.FORM_ADDITIVE, rz.FORM_HYBRID])
@pytest.mark.parametrize("space,p,n,nr", [("CG", 3, 4, 1), ("N1curl", 3, 3, 2), ("RT", 4, 3, 8)])
def test_tensor_products_solve_matches_oracle(space, p, n, nr, form):
    """PCG with the search-direction products (and, in the hybrid form, the sweep's residual updates) on the
    tensor cores, FP32 patch sweeps, FP64 residuals and residual replacement: stopped at rtol 1e-11 the
    solution is within 1e-8 relative L2 of the oracle's direct solve, and the iteration count stays close
    to the FP64-product solve's."""
    verts, cells, md, A = system(space, p, n)
    B = normal_coeffs((nr, md.ndofs), 19)
    s = rz.Riesz(space, p, verts, cells, apply_precision=rz.PREC_BF16X3, precond_precision=rz.PREC_FP32,
                 form=form, rtol=1e-11, maxit=3000, nrhs_max=nr)
    x = torch.zeros((nr, s.N), dtype=torch.float64, device="cuda")
    it, rr, rc = s.solve(dev(B), x, nrhs=nr)
    assert rc == 0
    X = x.cpu().numpy()
    for k in range(nr):
        xe = asm.direct_solve(A, B[k])
        assert np.linalg.norm(X[k] - xe) <= 1e-8 * np.linalg.norm(xe)
    s64 = rz.Riesz(space, p, verts, cells, precond_precision=rz.PREC_FP32, form=form, rtol=1e-11, maxit=3000,
                   nrhs_max=nr)
    x64 = torch.zeros_like(x)
    it64, _, _ = s64.solve(dev(B), x64, nrhs=nr)
    assert it[0] <= it64[0] + 10, (it[0], it64[0])
