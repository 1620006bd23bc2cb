"""Pins of the Hodge-Laplacian oracle (Section 7.2, Appendix C) against what the paper and the
mathematics fix."""
import numpy as np
import pytest
import scipy.sparse.linalg

from oracle import assemble as asm
from oracle import hodge
from oracle.refelem import reference_element
from paper_2506_17406_gb300.inputs import fichera_mesh, kuhn_mesh, normal_vector


def test_fichera_mesh():
    """(0,1)^3 minus (1/2,1)^3: 7/8 of the unit cube's volume, vertex indices increasing along every
    path, boundary vertices unperturbed (the re-entrant faces included)."""
    for n in (2, 4):
        v0, c0 = fichera_mesh(n)
        v, c = fichera_mesh(n, 0.1, 3)
        assert len(c) == 6 * (n ** 3 - (n // 2) ** 3)
        assert np.all(np.diff(c, axis=1) > 0)
        assert len(np.unique(c)) == len(v)
        P = v[c]
        vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])).sum() / 6.0
        assert abs(vol - 7.0 / 8.0) < 1e-12
        moved = np.any(v != v0, axis=1)
        on_outer = np.any((v0 == 0.0) | (v0 == 1.0), axis=1)
        on_inner = np.all(v0 >= 0.5, axis=1) & np.any(v0 == 0.5, axis=1)
        assert not np.any(moved & (on_outer | on_inner))
        assert n == 2 or np.all(moved | on_outer | on_inner)


def test_mixed_block_is_mass_times_gradient_map():
    """k = 1: B = (grad sigma, v) = M_1 G with G the exact gradient map of Eq. (5.3) -- an assembly of
    B by quadrature of the trial gradients checked against the Ned1 mass and the incidence map."""
    v, c = kuhn_mesh(2, 0.1, 5)
    h = hodge.HodgeSystem(1, 3, v, c)
    G = asm.gradient_matrix(h.md1, h.md0)
    assert abs(h.B - h.M1 @ G).max() <= 1e-12 * abs(h.B).max()
    # d o d = 0: the curl of every gradient vanishes, so B_2 B_1-type coupling K_1 G is zero
    assert abs(h.K1 @ G).max() <= 1e-11 * abs(h.K1).max()


@pytest.mark.parametrize("k,p,gamma", [(1, 1, 1.0), (1, 2, 1e3), (2, 1, 1.0), (2, 2, 1e3)])
def test_theorem_c1_spectrum(k, p, gamma):
    """Theorem C.1: with the exact block preconditioner of Eq. (7.6), the eigenvalues of P^{-1} A are
    -1 (multiplicity dim X^{k-1}), mu gamma/(mu gamma + 1) and nu gamma/(nu gamma + 1) for the nonzero
    generalized eigenvalues of (K_k, M_k) and (K_{k-1}, M_{k-1}); the Fichera corner is contractible,
    so there are no harmonic forms."""
    v, c = fichera_mesh(2, 0.1, 2)
    h = hodge.HodgeSystem(k, p, v, c, gamma)
    P = scipy.sparse.block_diag([h.P0, h.P1]).toarray()
    lam = np.sort(scipy.linalg.eigh(h.A.toarray(), P, eigvals_only=True))
    exp = hodge.predicted_spectrum(h)
    assert len(lam) == len(exp) == h.n0 + h.n1
    assert np.abs(lam - exp).max() <= 1e-8
    assert lam.min() >= -1.0 - 1e-9 and lam.max() < 1.0


def test_minres_matches_direct_solve_and_exact_preconditioner_counts():
    """MINRES reaches the sparse direct solution of the indefinite system; with the exact augmented-
    Lagrangian preconditioner and gamma = 1e3 the spectrum clusters at -1 and near 1, so it takes a
    handful of iterations (the paper reports 3 at p = 1, where its preconditioner is exact)."""
    v, c = fichera_mesh(2, 0.1, 1)
    for k in (1, 2):
        for gamma, bound in ((1.0, 12), (1e3, 6)):
            h = hodge.HodgeSystem(k, 2, v, c, gamma)
            b = h.rhs(normal_vector(h.n1, 4))
            x, it, res = hodge.minres(h.A, b, h.exact_preconditioner(), rtol=1e-10)
            xe = scipy.sparse.linalg.splu(h.A.tocsc()).solve(b)
            assert np.linalg.norm(x - xe) <= 1e-7 * np.linalg.norm(xe)
            assert it <= bound, (k, gamma, it)


def test_minres_equals_dense_krylov_minimiser():
    """The k-th MINRES iterate minimises the M^{-1}-norm of the residual over the Krylov space
    K_k(M^{-1}A, M^{-1}b): checked against a dense least-squares solve over an explicit basis."""
    rng = np.random.default_rng(0)
    n = 30
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(np.concatenate([-rng.uniform(1, 3, 10), rng.uniform(0.5, 4, 20)])) @ Q.T
    Mh = rng.standard_normal((n, n))
    M = Mh @ Mh.T + n * np.eye(n)
    Minv = lambda r: np.linalg.solve(M, r)
    b = rng.standard_normal(n)
    L = np.linalg.cholesky(np.linalg.inv(M))  # M^{-1} = L L^T
    for kk in (1, 3, 7):
        x, it, res = hodge.minres(A, b, Minv, rtol=0.0, maxit=kk)
        assert it == kk
        K = [Minv(b)]
        for _ in range(kk - 1):
            K.append(Minv(A @ K[-1]))
        K = np.linalg.qr(np.stack(K, 1))[0]
        y = np.linalg.lstsq(L.T @ A @ K, L.T @ b, rcond=None)[0]
        xe = K @ y
        assert np.linalg.norm(x - xe) <= 1e-8 * np.linalg.norm(xe)
        assert abs(res - np.linalg.norm(L.T @ (b - A @ x)) / np.linalg.norm(L.T @ b)) <= 1e-10


@pytest.mark.parametrize("k", [1, 2])
def test_schwarz_block_preconditioner(k):
    """The per-space Schwarz preconditioners (CG vertex stars, Ned1 Hiptmair-Toselli, RT edge stars,
    each with W^k) replace the exact Riesz maps: SPD blocks, MINRES still reaches the direct solution,
    and gamma = 1e3 takes about as many iterations as gamma = 1 (Table 6: the weight costs nothing once
    the blocks are Schwarz preconditioners; with the additive blocks here, whose spectra span about
    [0.5, 6], MINRES needs 2-3x the paper's counts for its multiplicative hybrid)."""
    v, c = fichera_mesh(2, 0.1, 1)
    its = []
    for gamma in (1.0, 1e3):
        h = hodge.HodgeSystem(k, 2, v, c, gamma)
        for blk, P in zip(h.schwarz_blocks(), (h.P0, h.P1)):
            ev = np.linalg.eigvals(blk.dense() @ P.toarray())
            assert np.abs(ev.imag).max() < 1e-8 and ev.real.min() > 0
        b = h.rhs(normal_vector(h.n1, 4))
        x, it, _ = hodge.minres(h.A, b, h.schwarz_preconditioner(), rtol=1e-10, maxit=500)
        xe = scipy.sparse.linalg.splu(h.A.tocsc()).solve(b)
        assert np.linalg.norm(x - xe) <= 1e-7 * np.linalg.norm(xe)
        its.append(it)
    assert its[1] <= 1.1 * its[0] + 2


def test_dg_basis_orthogonal_and_div_map():
    """X^3 = DG_{p-1} (the abstract DOFs with k = d): its reference mass matrix is diagonal (the paper's
    reason for point-Jacobi on DG in Section 7.2), and div maps RT_p onto DG_{p-1} with an exact
    coefficient map -- the signed face-cell incidence on the Whitney functions and the identity from
    the RT interior type-I functions onto the DG type-II functions (Lemma 4.3 at k = 2) -- so the
    coupling of the k = 3 problem is B = M_3 D."""
    for p in (1, 3):
        M, _ = reference_element("DG", p).ref_matrices()
        assert np.abs(M - np.diag(np.diag(M))).max() <= 1e-13 * np.abs(M).max()
    v, c = fichera_mesh(2, 0.1, 5)
    h = hodge.HodgeSystem(3, 3, v, c)
    assert abs(h.K1).max() == 0.0
    # D = M_3^{-1} B must be the structured map: integer entries, identity on the interior type-I DOFs
    D = scipy.sparse.diags(1.0 / h.M1.diagonal()) @ h.B
    Dd = D.toarray()
    assert np.abs(Dd - np.round(Dd)).max() <= 1e-9
    rt, dg = h.md0, h.md1
    nI = dg.per_entity[3] - 1  # RT interior type-I (div-type) DOFs = DG type-II DOFs
    for cell in range(len(c)):
        # the DG Whitney row: the Whitney DOFs of the cell's four faces with +-1, nothing else
        row = Dd[dg.cell_dofs[cell, 0]]
        nz = np.nonzero(np.abs(row) > 1e-9)[0]
        assert len(nz) == 4 and np.all(np.abs(np.abs(row[nz]) - 1.0) <= 1e-9)
        assert set(nz) <= set(rt._offsets[2] + rt.per_entity[2] * rt.cell_faces[cell])
        # the DG type-II rows: the identity onto the cell's RT interior type-I DOFs
        for m in range(nI):
            row = Dd[dg.cell_dofs[cell, 1 + m]]
            nz = np.nonzero(np.abs(row) > 1e-9)[0]
            assert list(nz) == [rt.n_interface + rt.per_entity[3] * cell + m]
            assert abs(row[nz[0]] - 1.0) <= 1e-9


@pytest.mark.parametrize("p,gamma", [(1, 1.0), (2, 1e3)])
def test_theorem_c1_spectrum_k3(p, gamma):
    """Theorem C.1 for the mixed Poisson problem (k = 3): -1 with multiplicity dim RT_p and
    nu gamma / (nu gamma + 1) for the nonzero div-div/mass eigenvalues nu of RT_p (one per DG DOF)."""
    v, c = fichera_mesh(2, 0.1, 2)
    h = hodge.HodgeSystem(3, p, v, c, gamma)
    P = scipy.sparse.block_diag([h.P0, h.P1]).toarray()
    lam = np.sort(scipy.linalg.eigh(h.A.toarray(), P, eigvals_only=True))
    exp = hodge.predicted_spectrum(h)
    assert len(exp) == h.n0 + h.n1
    assert np.abs(lam - exp).max() <= 1e-8


def test_minres_k3():
    """Mixed Poisson: MINRES reaches the direct solution with the exact preconditioner in a handful of
    iterations at gamma = 1e3 (the paper: 3 at p = 1) and with the Schwarz/Jacobi blocks."""
    v, c = fichera_mesh(2, 0.1, 1)
    for gamma, bound in ((1.0, 12), (1e3, 6)):
        h = hodge.HodgeSystem(3, 2, v, c, gamma)
        b = h.rhs(normal_vector(h.n1, 4))
        xe = scipy.sparse.linalg.splu(h.A.tocsc()).solve(b)
        x, it, _ = hodge.minres(h.A, b, h.exact_preconditioner(), rtol=1e-10)
        assert np.linalg.norm(x - xe) <= 1e-7 * np.linalg.norm(xe) and it <= bound
        x, it, _ = hodge.minres(h.A, b, h.schwarz_preconditioner(True), rtol=1e-10, maxit=1000)
        assert np.linalg.norm(x - xe) <= 1e-7 * np.linalg.norm(xe)


@pytest.mark.parametrize("k,bound", [(1, 45), (2, 55), (3, 20)])
def test_hybrid_blocks_reach_the_papers_range(k, bound):
    """With the paper's hybrid Schwarz form in each Riesz block (Eqs. (7.2)-(7.3)), MINRES at p = 2,
    gamma = 1e3 needs about as many iterations as Table 6 reports (37, 56, 14 for k = 1, 2, 3 on the
    paper's graded Fichera mesh; here 35, 41, 10 on the 2^3-cube Fichera mesh), well below the additive
    blocks, and still reaches the direct solution."""
    v, c = fichera_mesh(2, 0.1, 1)
    h = hodge.HodgeSystem(k, 2, v, c, 1e3)
    b = h.rhs(np.ones(h.n1))
    x, ih, _ = hodge.minres(h.A, b, h.schwarz_preconditioner(True, form="hybrid"), rtol=1e-10, maxit=2000)
    xe = scipy.sparse.linalg.splu(h.A.tocsc()).solve(b)
    assert np.linalg.norm(x - xe) <= 1e-7 * np.linalg.norm(xe)
    _, ih8, _ = hodge.minres(h.A, b, h.schwarz_preconditioner(True, form="hybrid"), rtol=1e-8, maxit=2000)
    _, ia8, _ = hodge.minres(h.A, b, h.schwarz_preconditioner(True), rtol=1e-8, maxit=2000)
    assert ih8 <= bound and 2 * ih8 <= ia8
