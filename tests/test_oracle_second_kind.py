"""Pins of the oracle's second-kind spaces NedTwo_p and BDM_p (Eq. (2.6)) as solution spaces.

Each pin is fixed by the mathematics, not by the oracle itself: dimensions of P_p^3 and of its
bubble spaces, the Whitney forms (Lemma 4.1), the exterior derivative of the lower space's type-I
functions (Lemma 4.3 with X^0 = CG_{p+1} for NedTwo_p and X^1 = NedTwo_{p+1} for BDM_p, Section 3.4),
the block structure of Lemma 4.5, and exact reproduction of a full degree-p field (which lies in the
second-kind space but not in the first-kind one of the same degree).
"""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle.mesh import MeshDofs
from oracle.polys import REF_VERTS, quadrature
from oracle.refelem import EDGES, FACES, eigenbasis, reference_element
from paper_2506_17406_gb300.inputs import kuhn_mesh, normal_vector

from test_oracle_solve import _poly


def _bary(X):
    V = REF_VERTS[3]
    A = np.vstack([V.T, np.ones(4)])
    lam = np.linalg.solve(A, np.vstack([X.T, np.ones(X.shape[0])])).T
    return lam, np.linalg.inv(A)[:, :3]


def _counts(space, p):
    """(edge, face, interior) DOFs per entity: P_p^3 has 3 (p+1)(p+2)(p+3)/6 functions; an edge of
    NedTwo_p carries a degree-p tangential trace (p+1 DOFs), a face the tangential bubbles of the
    face's NedTwo_p ((p+1)(p-1)); a face of BDM_p its degree-p normal trace ((p+1)(p+2)/2)."""
    n = (p + 1) * (p + 2) * (p + 3) // 2
    if space == "N2curl":
        ne, nf = p + 1, (p + 1) * (p - 1)
        return ne, nf, n - 6 * ne - 4 * nf
    nf = (p + 1) * (p + 2) // 2
    return 0, nf, n - 4 * nf


@pytest.mark.parametrize("space", ["N2curl", "BDM"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_dimensions_and_unisolvence(space, p):
    R = reference_element(space, p)
    assert R.ndofs == (p + 1) * (p + 2) * (p + 3) // 2
    ne, nf, ni = _counts(space, p)
    assert all(len(R.entity_dofs.get((1, e), [])) == ne for e in range(6))
    assert all(len(R.entity_dofs.get((2, f), [])) == nf for f in range(4))
    assert len(R.interior) == ni
    assert R.dof_cond < 1e4


@pytest.mark.parametrize("p", [1, 2, 3])
def test_lemma_4_1_whitney(p):
    """The first function of each edge (NedTwo_p) / face (BDM_p) is the Whitney form."""
    X, _ = quadrature(3, 4)
    lam, G = _bary(X)
    R = reference_element("N2curl", p)
    v, _ = R.tabulate(X)
    for e, (a, b) in enumerate(EDGES):
        w = lam[:, a, None] * G[b][None, :] - lam[:, b, None] * G[a][None, :]
        assert np.abs(v[:, R.entity_dofs[(1, e)][0], :] - w).max() < 1e-12
    R = reference_element("BDM", p)
    v, _ = R.tabulate(X)
    for f, (a, b, c) in enumerate(FACES):
        w = 2 * (lam[:, a, None] * np.cross(G[b], G[c])[None, :]
                 + lam[:, b, None] * np.cross(G[c], G[a])[None, :]
                 + lam[:, c, None] * np.cross(G[a], G[b])[None, :])
        assert np.abs(v[:, R.entity_dofs[(2, f)][0], :] - w).max() < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lemma_4_3_type_two_is_d_of_type_one(p):
    """NedTwo_p type-II functions are the gradients of the CG_{p+1} type-I functions of the same entity;
    BDM_p type-II functions are the curls of the NedTwo_{p+1} type-I functions of the same entity."""
    X, _ = quadrature(3, 4)
    cg = reference_element("CG", p + 1)
    n2 = reference_element("N2curl", p)
    _, gcg = cg.tabulate(X)
    vn, _ = n2.tabulate(X)
    checked = 0
    for key, dofs in n2.entity_dofs.items():
        cd = cg.entity_dofs.get(key, []) if key[0] > 0 else []
        if cd:
            assert np.abs(vn[:, dofs[-len(cd):], :] - gcg[:, cd, :]).max() < 1e-11
            checked += len(cd)
    assert checked == sum(len(d) for k, d in cg.entity_dofs.items() if k[0] > 0)
    n2p = reference_element("N2curl", p + 1)
    bdm = reference_element("BDM", p)
    _, cn2 = n2p.tabulate(X)
    vb, _ = bdm.tabulate(X)
    for f in range(4):
        nd = n2p.entity_dofs[(2, f)]
        nI = len(nd) - len(reference_element("CG", p + 2).entity_dofs[(2, f)])
        assert nI == len(bdm.entity_dofs[(2, f)]) - 1
        assert np.abs(vb[:, bdm.entity_dofs[(2, f)][1:], :] - cn2[:, nd[:nI], :]).max() < 1e-11
    nd = n2p.entity_dofs.get((3, 0), [])
    nI = len(nd) - len(reference_element("CG", p + 2).entity_dofs.get((3, 0), []))
    if nI:
        assert np.abs(vb[:, bdm.interior[-nI:], :] - cn2[:, nd[:nI], :]).max() < 1e-11


@pytest.mark.parametrize("space,p", [("N2curl", 3), ("N2curl", 4), ("BDM", 3), ("BDM", 4)])
def test_lemma_4_5_block_structure(space, p):
    """K_II = [I 0; 0 0], K_IG = 0, M_II = [Lambda 0; 0 I], and type-II rows of K vanish."""
    R = reference_element(space, p)
    M, K = R.ref_matrices()
    I = R.interior
    G = [i for i in range(R.ndofs) if i not in I]
    _, _, lam = eigenbasis("N2" if space == "N2curl" else "BDM", p, 3)
    nI = len(lam)
    Kexp = np.zeros((len(I), len(I)))
    Kexp[:nI, :nI] = np.eye(nI)
    Mexp = np.eye(len(I))
    Mexp[:nI, :nI] = np.diag(lam)
    assert np.abs(K[np.ix_(I, I)] - Kexp).max() < 1e-12
    assert np.abs(M[np.ix_(I, I)] - Mexp).max() < 1e-12 * max(1.0, np.abs(M).max())
    assert np.abs(K[np.ix_(I, G)]).max() < 1e-12
    typeII = list(I[nI:])
    for key, dofs in R.entity_dofs.items():
        if key[0] in (1, 2) and key[0] >= R.k:
            nfI = 1 if key[0] == R.k else len(eigenbasis("N2", p, 2)[2])
            typeII += list(dofs[nfI:])
    assert len(typeII) > 0
    assert np.abs(K[typeII, :]).max() < 1e-12


def _curl(jac):
    return np.stack([jac[:, 2, 1] - jac[:, 1, 2], jac[:, 0, 2] - jac[:, 2, 0], jac[:, 1, 0] - jac[:, 0, 1]], 1)


@pytest.mark.parametrize("space,p", [("N2curl", 1), ("N2curl", 2), ("N2curl", 3), ("BDM", 1), ("BDM", 2),
                                     ("BDM", 3)])
def test_full_degree_field_reproduced(space, p):
    """A random field in P_p^3 on a perturbed mesh lies in NedTwo_p / BDM_p, so the discrete Riesz map of
    its own right-hand side a(u, .) returns it exactly; the first-kind space of the same degree
    (Ned1_p, RT_p) does not contain it and misses it by a visible amount."""
    v, c = kuhn_mesh(2, 0.1, 7)
    val, jac = _poly(p, 3, 21 + p)
    du = (lambda x: _curl(jac(x))) if space == "N2curl" else (lambda x: np.trace(jac(x), axis1=1, axis2=2)[:, None])
    Xr, _ = quadrature(3, 3)
    errs = []
    for sp in (space, {"N2curl": "N1curl", "BDM": "RT"}[space]):
        ref = reference_element(sp, p)
        md = MeshDofs(v, c, ref)
        A = asm.assemble(md, asm.element_matrices(ref, v, c, alpha=1.3, beta=0.7))
        b = asm.load_function(ref, md, val, du, alpha=1.3, beta=0.7)
        x = asm.direct_solve(A, b)
        xq, uh = asm.evaluate(ref, md, x, Xr)
        ue = val(xq.reshape(-1, 3)).reshape(uh.shape)
        errs.append(np.abs(uh - ue).max() / np.abs(ue).max())
    assert errs[0] < 1e-9
    assert errs[1] > 1e-3


@pytest.mark.parametrize("p", [2, 3])
def test_ht_potentials_for_nedtwo_are_cg_p_plus_1_stiffness(p):
    """Gradients of CG_{p+1} interface functions (signed incidence + identity onto the type-II DOFs) lie in
    NedTwo_p: G^T A G on the CG_{p+1} interface DOFs is beta times the CG_{p+1} stiffness, and curl G = 0."""
    v, c = kuhn_mesh(2, 0.1, 4)
    rn, rc = reference_element("N2curl", p), reference_element("CG", p + 1)
    mn, mc = MeshDofs(v, c, rn), MeshDofs(v, c, rc)
    A = asm.assemble(mn, asm.element_matrices(rn, v, c, alpha=1.3, beta=0.7))
    G = asm.gradient_matrix(mn, mc)
    K = (G.T @ A @ G).toarray()[:mc.n_interface, :mc.n_interface]
    Kc = asm.assemble(mc, asm.element_matrices(rc, v, c, alpha=0.7, beta=0.0)).toarray()
    Kc = Kc[:mc.n_interface, :mc.n_interface]
    assert np.abs(K - Kc).max() <= 1e-11 * np.abs(Kc).max()


@pytest.mark.parametrize("space,p", [("N2curl", 2), ("BDM", 2), ("N2curl", 3), ("BDM", 3)])
def test_coarse_space_is_whitney_and_exact(space, p):
    """W^k by injection (Lemma 4.1): A_0 from the Whitney functions alone equals R_0 A R_0^T, and the coarse
    summand returns every u in W^k from r = A u."""
    ref = reference_element(space, p)
    v, c = kuhn_mesh(2, 0.1, 8)
    md = MeshDofs(v, c, ref)
    A = asm.assemble(md, asm.element_matrices(ref, v, c))
    W = asm.coarse_dofs(md)
    assert len(W) == (len(md.edges) if space == "N2curl" else len(md.faces))
    A0 = asm.coarse_matrix(ref, md).toarray()
    ref0 = A.tocsr()[W][:, W].toarray()
    assert np.abs(A0 - ref0).max() <= 1e-12 * np.abs(ref0).max()
    # the same matrix as the lowest-order first-kind space (Ned1_1 / RT_1 are the Whitney forms)
    r1 = reference_element({"N2curl": "N1curl", "BDM": "RT"}[space], 1)
    m1 = MeshDofs(v, c, r1)
    A1 = asm.assemble(m1, asm.element_matrices(r1, v, c)).toarray()
    assert np.abs(A0 - A1).max() <= 1e-12 * np.abs(A1).max()
    P2 = asm.TwoLevelPreconditioner(A, md)
    u = np.zeros(md.ndofs)
    u[P2.W] = normal_vector(len(P2.W), 3)
    assert np.abs(P2.coarse(A @ u) - u).max() <= 1e-10 * np.abs(u).max()


@pytest.mark.parametrize("space", ["N2curl", "BDM"])
def test_preconditioners_spd_and_refinement_robust(space):
    """Two-level vertex stars (both spaces), HT with CG_{p+1} potentials (NedTwo_p) and PAFW_1 edge stars
    (BDM_p): SPD on A, PCG counts flat from 2^3 to 4^3 cubes."""
    p = 2
    ref = reference_element(space, p)
    rc = reference_element("CG", p + 1)
    its = {}
    for n in (2, 4):
        v, c = kuhn_mesh(n, 0.1, 1)
        md = MeshDofs(v, c, ref)
        A = asm.assemble(md, asm.element_matrices(ref, v, c))
        b = normal_vector(md.ndofs, 3)
        if space == "N2curl":
            mc = MeshDofs(v, c, rc)
            Ps = {"vertex": asm.TwoLevelPreconditioner(A, md), "ht": asm.HTPreconditioner(A, md, mc)}
        else:
            Ps = {"vertex": asm.TwoLevelPreconditioner(A, md),
                  "edge": asm.TwoLevelPreconditioner(A, md, patches=asm.edge_star_dofs(md))}
        if n == 2:
            for P in Ps.values():
                ev = np.linalg.eigvals(P.dense() @ A.toarray())
                assert np.abs(ev.imag).max() < 1e-8 and ev.real.min() > 0
        for k, P in Ps.items():
            its.setdefault(k, []).append(asm.pcg(A, b, P.apply)[1])
    for k, (i2, i4) in its.items():
        assert i4 <= 1.2 * i2 + 2, (k, i2, i4)
