"""Pins of the oracle's assembly, preconditioner and solvers."""
import numpy as np
import pytest
import scipy.sparse

from oracle import assemble as asm
from oracle.mesh import MeshDofs
from oracle.polys import REF_VERTS, quadrature
from oracle.refelem import reference_element, eigenbasis
from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_coeffs, normal_vector


def _poly(deg, ncomp, seed):
    """Random polynomial field of total degree <= deg in physical coordinates (value, jacobian)."""
    exps = [(a, b, c) for a in range(deg + 1) for b in range(deg + 1 - a)
            for c in range(deg + 1 - a - b)]
    C = normal_coeffs((ncomp, len(exps)), seed)

    def val(x):
        return np.stack([sum(C[m, k] * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c
                             for k, (a, b, c) in enumerate(exps)) for m in range(ncomp)], 1)

    def jac(x):
        J = np.zeros((x.shape[0], ncomp, 3))
        for m in range(ncomp):
            for k, (a, b, c) in enumerate(exps):
                if a:
                    J[:, m, 0] += C[m, k] * a * x[:, 0] ** (a - 1) * x[:, 1] ** b * x[:, 2] ** c
                if b:
                    J[:, m, 1] += C[m, k] * b * x[:, 0] ** a * x[:, 1] ** (b - 1) * x[:, 2] ** c
                if c:
                    J[:, m, 2] += C[m, k] * c * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** (c - 1)
        return J
    return val, jac


@pytest.mark.parametrize("space,p", [("CG", 3), ("CG", 4), ("N1curl", 3), ("RT", 3)])
def test_manufactured_solution_reproduced(space, p):
    """u in V_h solves the discrete problem exactly: CG_p contains P_p, N1curl_p and RT_p contain P_{p-1}^3."""
    ref = reference_element(space, p)
    v, c = kuhn_mesh(2, 0.1, 7)
    md = MeshDofs(v, c, ref)
    if space == "CG":
        val, jac = _poly(p, 1, 11)
        du = lambda x: jac(x)[:, 0, :]
    else:
        val, jac = _poly(p - 1, 3, 12)
        if space == "N1curl":
            du = lambda x: np.stack([jac(x)[:, 2, 1] - jac(x)[:, 1, 2], jac(x)[:, 0, 2] - jac(x)[:, 2, 0],
                                     jac(x)[:, 1, 0] - jac(x)[:, 0, 1]], 1)
        else:
            du = lambda x: np.trace(jac(x), axis1=1, axis2=2)[:, None]
    A = asm.assemble(md, asm.element_matrices(ref, v, c))
    b = asm.load_function(ref, md, val, du)
    x = asm.direct_solve(A, b)
    Xr, _ = quadrature(3, 3)
    xq, uh = asm.evaluate(ref, md, x, Xr)
    ue = val(xq.reshape(-1, 3)).reshape(uh.shape)
    assert np.abs(uh - ue).max() < 1e-9 * np.abs(ue).max()


def _dense(md, Ae):
    A = np.zeros((md.ndofs, md.ndofs))
    for e in range(md.cells.shape[0]):
        A[np.ix_(md.cell_dofs[e], md.cell_dofs[e])] += Ae[e]
    return A


@pytest.mark.parametrize("ncell", [1, 2])
@pytest.mark.parametrize("space,p", [("CG", 3), ("N1curl", 2), ("RT", 3)])
def test_brute_force_dense_one_and_two_tets(ncell, space, p):
    """Dense numpy.linalg.solve on 1- and 2-tet meshes vs the sparse direct solve and PCG."""
    ref = reference_element(space, p)
    rng = np.random.Generator(np.random.PCG64(5))
    if ncell == 1:
        v = rng.standard_normal((4, 3))
        c = np.array([[0, 1, 2, 3]])
    else:
        v = rng.standard_normal((5, 3))
        c = np.array([[0, 1, 2, 3], [1, 2, 3, 4]])
    md = MeshDofs(v, c, ref)
    Ae = asm.element_matrices(ref, v, c)
    Ad = _dense(md, Ae)
    As = asm.assemble(md, Ae)
    assert np.abs(As.toarray() - Ad).max() < 1e-12 * np.abs(Ad).max()
    b = normal_vector(md.ndofs, 3)
    xd = np.linalg.solve(Ad, b)
    assert np.linalg.norm(asm.direct_solve(As, b) - xd) < 1e-10 * np.linalg.norm(xd)
    P = asm.Preconditioner(As, md)
    xp, it, rr = asm.pcg(As, b, P.apply, rtol=1e-12, maxit=500)
    assert rr <= 1e-12
    assert np.linalg.norm(xp - xd) < 1e-8 * np.linalg.norm(xd)


def test_global_complex_d_of_d_is_zero():
    """Eq. (5.3): grad CG_p = [signed incidence | identity] in N1curl_p, and curl grad = 0,
    curl N1curl_p lies in RT_p with div curl = 0 (the global bases are conforming)."""
    p = 3
    v, c = kuhn_mesh(2, 0.1, 9)
    cg, ned, rt = (reference_element(s, p) for s in ("CG", "N1curl", "RT"))
    mcg, mned, mrt = MeshDofs(v, c, cg), MeshDofs(v, c, ned), MeshDofs(v, c, rt)
    Mn, Kn = asm.mass_and_stiffness(ned, mned)
    Mr, Kr = asm.mass_and_stiffness(rt, mrt)
    _, Kc = asm.mass_and_stiffness(cg, mcg)
    B = asm.mixed_matrix(ned, mned, cg, mcg).toarray()
    G = np.linalg.solve(Mn.toarray(), B)
    # exact representation: ||grad phi_j - P grad phi_j||^2 = K_cg[j,j] - b_j . G_j
    resid = Kc.diagonal() - np.einsum("ij,ij->j", B, G)
    assert np.abs(resid).max() < 1e-10 * Kc.diagonal().max()
    # structure: vertex columns = signed edge incidence on the Whitney DOFs, others unit vectors
    Gexp = np.zeros_like(G)
    ne_d = mned.per_entity[1]
    for e, (a, b) in enumerate(mned.edges):
        Gexp[ne_d * e, a] = -1.0
        Gexp[ne_d * e, b] = 1.0
        for m in range(1, ne_d):
            Gexp[ne_d * e + m, mcg.nverts + (ne_d - 1) * e + m - 1] = 1.0
    nfI = mned.per_entity[2] - mcg.per_entity[2]
    for f in range(len(mned.faces)):
        for m in range(mcg.per_entity[2]):
            Gexp[mned._offsets[2] + mned.per_entity[2] * f + nfI + m,
                 mcg._offsets[2] + mcg.per_entity[2] * f + m] = 1.0
    assert np.abs(G - Gexp).max() < 1e-10
    assert np.abs(Kn @ G).max() < 1e-10
    Bc = asm.mixed_matrix(rt, mrt, ned, mned).toarray()
    C = np.linalg.solve(Mr.toarray(), Bc)
    resid = Kn.diagonal() - np.einsum("ij,ij->j", Bc, C)
    assert np.abs(resid).max() < 1e-10 * Kn.diagonal().max()
    assert np.abs(Kr @ C).max() < 1e-9
    assert np.abs(C @ G).max() < 1e-10


def test_preconditioner_reduces_to_jacobi_at_lowest_order():
    """CG_1: every vertex patch holds one DOF, so P^{-1} = diag(A)^{-1}."""
    ref = reference_element("CG", 1)
    v, c = kuhn_mesh(3, 0.1, 2)
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c))
    P = asm.Preconditioner(A, md)
    r = normal_vector(md.ndofs, 4)
    assert np.allclose(P.apply(r), r / A.diagonal(), rtol=1e-13, atol=0)


@pytest.mark.parametrize("space,p", [("CG", 5), ("N1curl", 4), ("RT", 4)])
def test_interior_diagonal_on_reference_cell(space, p):
    """Lemma 4.5 on the reference cell as a one-cell mesh: diag(A_II) = [lambda + 1, 1]."""
    ref = reference_element(space, p)
    v = REF_VERTS[3].copy()
    c = np.array([[0, 1, 2, 3]])
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c)).toarray()
    fam = {"CG": "CG", "N1curl": "N1", "RT": "RT"}[space]
    lam = eigenbasis(fam, p, 3)[2]
    d = np.diag(A)[md.n_interface:]
    exp = np.ones(len(d))
    exp[:len(lam)] = lam + 1.0
    assert np.abs(d - exp).max() < 1e-12
    AII = A[md.n_interface:, md.n_interface:]
    assert np.abs(AII - np.diag(np.diag(AII))).max() < 1e-12


def test_patch_matrices_from_cells_equal_global_restriction():
    """A_V assembled cell by cell over the star equals A restricted to the patch."""
    ref = reference_element("N1curl", 2)
    v, c = kuhn_mesh(2, 0.1, 4)
    md = MeshDofs(v, c, ref)
    Ae = asm.element_matrices(ref, v, c)
    A = asm.assemble(md, Ae)
    for vi, idx in enumerate(md.patches()):
        pos = {g: k for k, g in enumerate(idx)}
        AV = np.zeros((len(idx), len(idx)))
        _, _, cells = md.vertex_star(vi)
        for e in cells:
            loc = [j for j in range(ref.ndofs) if md.cell_dofs[e, j] in pos]
            gl = [pos[md.cell_dofs[e, j]] for j in loc]
            AV[np.ix_(gl, gl)] += Ae[e][np.ix_(loc, loc)]
        assert np.abs(AV - A[idx][:, idx].toarray()).max() < 1e-12 * np.abs(AV).max()


@pytest.mark.parametrize("space,p", [("CG", 2), ("N1curl", 2), ("RT", 2)])
def test_additive_schwarz_spectrum(space, p):
    """P^{-1} A is similar to an SPD matrix with eigenvalues in (0, 4 + max_T lambda_max(D_T^{-1} A_T,II)]:
    at most four vertex patches meet on a cell (Section 6, additive Schwarz theory)."""
    ref = reference_element(space, p)
    v, c = kuhn_mesh(2, 0.1, 6)
    md = MeshDofs(v, c, ref)
    Ae = asm.element_matrices(ref, v, c)
    A = asm.assemble(md, Ae).toarray()
    P = asm.Preconditioner(scipy.sparse.csr_matrix(A), md).dense()
    ev = np.linalg.eigvals(P @ A)
    assert np.abs(ev.imag).max() < 1e-8
    I = ref.interior
    jac = 1.0
    if I:
        dI = np.diag(A)[md.n_interface:]
        for e in range(len(c)):
            ae = Ae[e][np.ix_(I, I)]
            de = dI[md.cell_dofs[e, I] - md.n_interface]
            jac = max(jac, np.linalg.eigvalsh(ae / np.sqrt(np.outer(de, de))).max())
    assert ev.real.min() > 0
    assert ev.real.max() <= 4 + jac + 1e-10


def test_cg_field_load_matches_function_load():
    """(f, phi_i) for f in [CG_p]^3 via CG coefficients equals quadrature of the same polynomial."""
    p = 2
    v, c = kuhn_mesh(2)  # unperturbed: CG_p interpolates the polynomial exactly
    ned, cg = reference_element("N1curl", p), reference_element("CG", p)
    mned, mcg = MeshDofs(v, c, ned), MeshDofs(v, c, cg)
    val, _ = _poly(1, 3, 21)
    # CG_p coefficients of a linear field: vertex DOFs are point values, higher DOFs of a
    # linear function vanish (Lemma 4.1: the vertex functions are the P1 hat functions)
    f = np.zeros((3, mcg.ndofs))
    f[:, :mcg.nverts] = val(v).T
    b1 = asm.load_cg_field(ned, mned, cg, mcg, f)
    b2 = asm.load_function(ned, mned, val)
    assert np.abs(b1 - b2).max() < 1e-12 * np.abs(b2).max()


def test_sampled_oracle_rows_match_full_oracle():
    """The sampled apply/preconditioner helpers used at full size equal the assembled ones."""
    ref = reference_element("RT", 3)
    v, c = kuhn_mesh(3, 0.1, 2)
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c))
    P = asm.Preconditioner(A, md)
    x = normal_vector(md.ndofs, 1)
    d = np.sort(np.random.Generator(np.random.PCG64(0)).choice(md.ndofs, 40, replace=False))
    assert np.abs(asm.sampled_apply(ref, md, d, x) - (A @ x)[d]).max() < 1e-12 * np.abs(A @ x).max()
    ze = P.apply(x)
    assert np.abs(asm.sampled_precond(ref, md, d, x) - ze[d]).max() < 1e-11 * np.abs(ze).max()


@pytest.mark.parametrize("space,p", [("CG", 3), ("N1curl", 2), ("RT", 2)])
def test_coarse_dofs_are_the_first_dof_of_each_entity(space, p):
    """W^k (Lemma 4.1): one DOF per vertex / edge / face, the entity's first type-I DOF in every cell."""
    ref = reference_element(space, p)
    v, c = kuhn_mesh(2, 0.1, 4)
    md = MeshDofs(v, c, ref)
    W = asm.coarse_dofs(md)
    k = {"CG": 0, "N1curl": 1, "RT": 2}[space]
    nent = {0: md.nverts, 1: len(md.edges), 2: len(md.faces)}[k]
    assert len(W) == nent == len(np.unique(W))
    seen = set()
    for e in range(len(c)):
        for s in range({0: 4, 1: 6, 2: 4}[k]):
            seen.add(int(md.cell_dofs[e, ref.entity_dofs[(k, s)][0]]))
    assert seen == set(int(w) for w in W)


@pytest.mark.parametrize("space,p", [("CG", 3), ("N1curl", 3), ("RT", 3)])
def test_coarse_correction_reproduces_coarse_functions(space, p):
    """For u = R_0^T w in W^k and r = A u, the coarse summand returns u exactly (A_0 = R_0 A R_0^T)."""
    ref = reference_element(space, p)
    v, c = kuhn_mesh(3, 0.1, 5)
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c))
    P2 = asm.TwoLevelPreconditioner(A, md)
    w = normal_vector(len(P2.W), 3)
    u = np.zeros(md.ndofs)
    u[P2.W] = w
    z = P2.coarse(A @ u)
    assert np.abs(z - u).max() <= 1e-10 * np.abs(u).max()


@pytest.mark.parametrize("space,p", [("CG", 2), ("N1curl", 2), ("RT", 2)])
def test_two_level_spectrum(space, p):
    """Adding the PSD coarse term to P^{-1} can only raise every eigenvalue of P^{-1} A (Courant-Fischer in
    the A inner product), and raises the additive upper bound by one summand: 5 + lambda_J."""
    ref = reference_element(space, p)
    v, c = kuhn_mesh(2, 0.1, 6)
    md = MeshDofs(v, c, ref)
    Ae = asm.element_matrices(ref, v, c)
    A = asm.assemble(md, Ae)
    Ad = A.toarray()
    e1 = np.sort(np.linalg.eigvals(asm.Preconditioner(A, md).dense() @ Ad).real)
    e2 = np.sort(np.linalg.eigvals(asm.TwoLevelPreconditioner(A, md).dense() @ Ad).real)
    assert e1.min() > 0
    assert np.all(e2 >= e1 * (1 - 1e-10))
    I = ref.interior
    jac = 1.0
    if I:
        dI = np.diag(Ad)[md.n_interface:]
        for e in range(len(c)):
            ae = Ae[e][np.ix_(I, I)]
            de = dI[md.cell_dofs[e, I] - md.n_interface]
            jac = max(jac, np.linalg.eigvalsh(ae / np.sqrt(np.outer(de, de))).max())
    assert e2.max() <= 5 + jac + 1e-10


def test_two_level_iterations_do_not_grow_with_refinement():
    """With W^k the iteration count stays flat from 2^3 to 4^3 cubes while the one-level count grows."""
    ref = reference_element("CG", 3)
    its1, its2 = [], []
    for n in (2, 4):
        v, c = kuhn_mesh(n, 0.1, 1)
        md = MeshDofs(v, c, ref)
        A = asm.assemble(md, asm.element_matrices(ref, v, c))
        b = normal_vector(md.ndofs, 3)
        its1.append(asm.pcg(A, b, asm.Preconditioner(A, md).apply)[1])
        its2.append(asm.pcg(A, b, asm.TwoLevelPreconditioner(A, md).apply)[1])
    assert its1[1] > 1.3 * its1[0]
    assert its2[1] <= 1.15 * its2[0] + 1
    assert its2[1] < its1[1]


@pytest.mark.parametrize("space,p", [("CG", 3), ("N1curl", 3), ("RT", 2)])
def test_coarse_matrix_by_quadrature_equals_restriction(space, p):
    """A_0 from the lowest-order basis functions alone equals R_0 A R_0^T of the full assembly."""
    ref = reference_element(space, p)
    v, c = kuhn_mesh(2, 0.1, 8)
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c))
    W = asm.coarse_dofs(md)
    A0 = asm.coarse_matrix(ref, md).toarray()
    ref0 = A.tocsr()[W][:, W].toarray()
    assert np.abs(A0 - ref0).max() <= 1e-12 * np.abs(ref0).max()


@pytest.mark.parametrize("space,p", [("CG", 2), ("CG", 3), ("N1curl", 2), ("N1curl", 3), ("RT", 2), ("RT", 3)])
def test_dirichlet_dofs_count_and_place(space, p):
    """The fixed DOFs of a whole-boundary Dirichlet condition: their number is the closed form
    nv (6n^2+2) + ne 18 n^2 + nf 12 n^2 of the cube's surface triangulation (6n^2+2 vertices, 18n^2
    edges, 12n^2 triangles), and every one belongs to an entity whose vertices lie on one cube face."""
    ref = reference_element(space, p)
    for n in (1, 2):
        v, c = kuhn_mesh(n, 0.0, 1)
        md = MeshDofs(v, c, ref)
        D = asm.dirichlet_dofs(md)
        nv, ne, nf, _ = md.per_entity
        assert len(D) == nv * (6 * n * n + 2) + ne * 18 * n * n + nf * 12 * n * n
        for d in D:
            X = md.verts[md.vertices_of_dof(int(d))]
            assert any(np.all(np.isclose(X[:, a], b)) for a in range(3) for b in (0.0, 1.0))


def _bubble():
    def u(x):
        return (x[:, 0] * (1 - x[:, 0]) * x[:, 1] * (1 - x[:, 1]) * x[:, 2] * (1 - x[:, 2]))[:, None]

    def grad(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        bx, by, bz = X * (1 - X), Y * (1 - Y), Z * (1 - Z)
        return np.stack([(1 - 2 * X) * by * bz, bx * (1 - 2 * Y) * bz, bx * by * (1 - 2 * Z)], 1)
    return u, grad


@pytest.mark.parametrize("space", ["CG", "N1curl"])
def test_dirichlet_manufactured_solution(space):
    """u with zero trace lying in V_h (CG_6: the cubic bubble xyz(1-x)(1-y)(1-z); Ned1_6: its gradient,
    whose tangential trace vanishes and whose curl is zero) is reproduced by the constrained system."""
    p = 6
    ref = reference_element(space, p)
    v, c = kuhn_mesh(1, 0.0, 1)
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c))
    D = asm.dirichlet_dofs(md)
    ub, gb = _bubble()
    if space == "CG":
        f, df = ub, gb
    else:
        f, df = gb, (lambda x: np.zeros((x.shape[0], 3)))
    b = asm.load_function(ref, md, f, df)
    b[D] = 0.0
    x = asm.direct_solve(asm.constrained(A, D), b)
    assert np.abs(x[D]).max() == 0.0
    X, _ = quadrature(3, 3)
    xq, val = asm.evaluate(ref, md, x, X)
    ue = f(xq.reshape(-1, 3)).reshape(val.shape)
    assert np.abs(val - ue).max() <= 1e-10 * np.abs(ue).max()


def test_dirichlet_solution_has_zero_trace():
    """For a random right-hand side the constrained solution vanishes at points of boundary faces."""
    ref = reference_element("CG", 3)
    v, c = kuhn_mesh(2, 0.1, 3)
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c))
    D = asm.dirichlet_dofs(md)
    b = normal_vector(md.ndofs, 4)
    b[D] = 0.0
    x = asm.direct_solve(asm.constrained(A, D), b)
    # points on the reference faces, mapped in every cell; keep those on the cube's surface
    Vr = REF_VERTS[3]
    rng = np.random.default_rng(0)
    pts = []
    for f in [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]:
        lam = rng.dirichlet(np.ones(3), 5)
        pts.append(lam @ Vr[list(f)])
    xq, val = asm.evaluate(ref, md, x, np.concatenate(pts))
    xq = xq.reshape(-1, 3)
    on = np.any(np.isclose(xq, 0.0) | np.isclose(xq, 1.0), axis=1)
    assert on.sum() > 20
    assert np.abs(val.reshape(-1)[on]).max() <= 1e-12 * np.abs(x).max()
    assert np.abs(val.reshape(-1)[~on]).max() > 1e-3 * np.abs(x).max()


def test_ht_potential_matrices_are_cg_stiffness():
    """G^T A G on the CG interface DOFs is beta times the CG_p stiffness (d o d = 0 removes the curl
    term), assembled independently from CG element matrices."""
    p = 3
    v, c = kuhn_mesh(2, 0.1, 4)
    rn, rc = reference_element("N1curl", p), reference_element("CG", p)
    mn, mc = MeshDofs(v, c, rn), MeshDofs(v, c, rc)
    A = asm.assemble(mn, asm.element_matrices(rn, v, c, alpha=1.3, beta=0.7))
    G = asm.gradient_matrix(mn, mc)
    K = (G.T @ A @ G).toarray()[:mc.n_interface, :mc.n_interface]
    Kc = asm.assemble(mc, asm.element_matrices(rc, v, c, alpha=0.7, beta=0.0)).toarray()
    Kc = Kc[:mc.n_interface, :mc.n_interface]
    assert np.abs(K - Kc).max() <= 1e-11 * np.abs(Kc).max()


def test_ht_edge_stars():
    """Edge-star type-I DOFs: the edge's Whitney DOF and the type-I DOFs of each face containing it."""
    p = 4
    v, c = kuhn_mesh(2, 0.1, 4)
    rn, rc = reference_element("N1curl", p), reference_element("CG", p)
    mn, mc = MeshDofs(v, c, rn), MeshDofs(v, c, rc)
    stars = asm.edge_star_type1_dofs(mn, mc)
    nfI = mn.per_entity[2] - mc.per_entity[2]  # face type-I DOFs: the face DOFs that are not gradients
    assert nfI > 0
    for e, (a, b) in enumerate(mn.edges):
        nf = int(np.sum(np.isin(mn.faces, [a, b]).sum(1) == 2))
        assert len(stars[e]) == 1 + nfI * nf
        assert stars[e][0] == mn._offsets[1] + mn.per_entity[1] * e


def test_ht_preconditioner_spd_and_refinement_robust():
    """The HT preconditioner is SPD on A (positive spectrum of P^{-1}A) and its PCG count stays
    flat from 2^3 to 4^3 cubes, like the vertex-star two-level one."""
    rn, rc = reference_element("N1curl", 2), reference_element("CG", 2)
    v, c = kuhn_mesh(2, 0.1, 6)
    mn, mc = MeshDofs(v, c, rn), MeshDofs(v, c, rc)
    A = asm.assemble(mn, asm.element_matrices(rn, v, c))
    ev = np.linalg.eigvals(asm.HTPreconditioner(A, mn, mc).dense() @ A.toarray())
    assert np.abs(ev.imag).max() < 1e-8 and ev.real.min() > 0
    its = []
    for n in (2, 4):
        v, c = kuhn_mesh(n, 0.1, 1)
        mn, mc = MeshDofs(v, c, rn), MeshDofs(v, c, rc)
        A = asm.assemble(mn, asm.element_matrices(rn, v, c))
        b = normal_vector(mn.ndofs, 3)
        its.append(asm.pcg(A, b, asm.HTPreconditioner(A, mn, mc).apply)[1])
    assert its[1] <= 1.2 * its[0] + 2


def test_hdiv_edge_stars_cover_faces():
    """PAFW_1 edge stars for RT_p (Eq. (6.24)): exactly the DOFs of the faces containing the edge, so
    every interface (face) DOF lies in the stars of its face's three edges and nowhere else."""
    p = 3
    v, c = kuhn_mesh(2, 0.1, 4)
    md = MeshDofs(v, c, reference_element("RT", p))
    stars = asm.edge_star_dofs(md)
    nf_d = md.per_entity[2]
    cnt = np.zeros(md.n_interface, dtype=int)
    for e, (a, b) in enumerate(md.edges):
        nf = int(np.sum(np.isin(md.faces, [a, b]).sum(1) == 2))
        assert len(stars[e]) == nf * nf_d
        np.add.at(cnt, stars[e], 1)
    assert np.all(cnt == 3)
    # every edge star lies inside the vertex stars of both endpoints
    vp = md.patches()
    for e, (a, b) in enumerate(md.edges):
        assert set(stars[e]) <= set(vp[a]) and set(stars[e]) <= set(vp[b])


def test_hdiv_edge_star_preconditioner_spd_and_refinement_robust():
    """PAFW_1(X^2_Gamma)+J(X^2_I) with W^2 (Eq. (6.24)): SPD on A and a PCG count that stays flat from
    2^3 to 4^3 cubes (h-robust with the coarse space, alpha = beta = 1)."""
    ref = reference_element("RT", 2)
    v, c = kuhn_mesh(2, 0.1, 6)
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c))
    P = asm.TwoLevelPreconditioner(A, md, asm.edge_star_dofs(md))
    ev = np.linalg.eigvals(P.dense() @ A.toarray())
    assert np.abs(ev.imag).max() < 1e-8 and ev.real.min() > 0
    its = []
    for n in (2, 4):
        v, c = kuhn_mesh(n, 0.1, 1)
        md = MeshDofs(v, c, ref)
        A = asm.assemble(md, asm.element_matrices(ref, v, c))
        b = normal_vector(md.ndofs, 3)
        its.append(asm.pcg(A, b, asm.TwoLevelPreconditioner(A, md, asm.edge_star_dofs(md)).apply)[1])
    assert its[1] <= 1.2 * its[0] + 2


def test_lanczos_extremes_bracket_the_spectrum():
    """10 CG/Lanczos steps (the paper's eigenvalue estimate for the hybrid weights, Eq. (7.3)): the Ritz
    values lie inside the spectrum of B^{-1}A and the largest is within a few percent of lambda_max."""
    rng = np.random.default_rng(4)
    n = 60
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    lam = np.concatenate([[0.3], rng.uniform(0.5, 3.0, n - 2), [4.0]])
    A = Q @ np.diag(lam) @ Q.T
    d = rng.uniform(0.5, 2.0, n)  # B = diag(d)^-1 similarity keeps the pencil SPD
    B = np.diag(1.0 / d)
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(B, A)).real)
    lo, hi = asm.lanczos_extremes(lambda x: A @ x, lambda x: d * x, n, iters=10)
    assert ev[0] - 1e-12 <= lo <= hi <= ev[-1] + 1e-12
    assert hi >= 0.95 * ev[-1]


@pytest.mark.parametrize("space,p", [("CG", 2), ("N1curl", 2), ("RT", 2)])
def test_hybrid_preconditioner_symmetric_and_bounded(space, p):
    """The symmetric multiplicative sweep X_1, X_2, X_3, X_2, X_1 with rho_m = (lambda_min + 3 lambda_max)/4
    (Eqs. (7.2)-(7.3)): every damped step contracts in the energy norm (rho_m > lambda_max / 2), so the
    preconditioner is symmetric and the spectrum of P^{-1}A lies in (0, 1]."""
    v, c = kuhn_mesh(2, 0.1, 1)
    ref = reference_element(space, p)
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c))
    H = asm.HybridPreconditioner(A, md)
    P = H.dense()
    assert np.abs(P - P.T).max() <= 1e-12 * np.abs(P).max()
    ev = np.linalg.eigvals(P @ A.toarray())
    assert np.abs(ev.imag).max() < 1e-10
    assert ev.real.min() > 0.05 and ev.real.max() <= 1.0 + 1e-10
    assert abs(H.rho[3] - 1.0) < 1e-10  # exact coarse solver: a = a~ on W^k


def test_hybrid_preconditioner_iterations():
    """With the paper's hybrid form the PCG counts drop well below the additive two-level ones
    (Ned1_3 on 4^3 cubes: 12 against 31) and match the range of the paper's Tables 3-5."""
    v, c = kuhn_mesh(4, 0.1, 1)
    ref = reference_element("N1curl", 3)
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c))
    b = normal_vector(md.ndofs, 7)
    it_add = asm.pcg(A, b, asm.TwoLevelPreconditioner(A, md).apply)[1]
    it_hyb = asm.pcg(A, b, asm.HybridPreconditioner(A, md).apply)[1]
    assert it_hyb <= 15 and 2 * it_hyb <= it_add


@pytest.mark.parametrize("space,p,ht", [("CG", 2, False), ("CG", 4, False), ("RT", 2, False), ("N1curl", 2, True),
                                        ("N1curl", 3, True)])
def test_hybrid_sweep_equals_error_propagation_product(space, p, ht):
    """The residual-update sweep of HybridPreconditioner equals the closed form of a multiplicative
    Schwarz method (Section 7.1, Eq. (7.2)): P^{-1} = (I - E) A^{-1} with the error propagation
    E = (I - T_1)(I - T_2)(I - T_3)(I - T_2)(I - T_1), T_m = rho_m^{-1} B_m A and B_m the subspace solver
    extended by zero (X_1: interior point-Jacobi; X_2: the interface solver on interface residuals,
    interface output only, also for the Hiptmair-Toselli splitting; X_3: the exact W^k solve)."""
    v, c = kuhn_mesh(2, 0.1, 1)
    ref = reference_element(space, p)
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c)).tocsr()
    iface = None
    if ht:
        mc = MeshDofs(v, c, reference_element("CG", p))
        iface = asm.HTPreconditioner(A, md, mc, weight=0.0)
    H = asm.HybridPreconditioner(A, md, interface=iface)
    N = A.shape[0]
    nI = md.n_interface
    Ad = A.toarray()
    I = np.eye(N)
    B1 = np.zeros((N, N))
    B1[nI:, nI:] = np.diag(1.0 / np.diag(Ad)[nI:])
    solver = asm.Preconditioner(A, md) if iface is None else iface
    B2 = np.zeros((N, N))
    for j in range(nI):
        e = np.zeros(N)
        e[j] = 1.0
        B2[:nI, j] = solver.apply(e)[:nI]
    W = asm.coarse_dofs(md)
    B3 = np.zeros((N, N))
    B3[np.ix_(W, W)] = np.linalg.inv(Ad[np.ix_(W, W)])
    T = {m: B @ Ad / H.rho[m] for m, B in ((1, B1), (2, B2), (3, B3)) if m in H.rho}
    assert H.sweep == [m for m in [1, 2, 3, 2, 1] if m in T]  # X_1 only where there are interior DOFs
    E = I
    for m in H.sweep:
        E = (I - T[m]) @ E
    P = (I - E) @ np.linalg.inv(Ad)
    assert np.abs(H.dense() - P).max() <= 1e-9 * np.abs(P).max()
