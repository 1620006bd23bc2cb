"""Pins of the oracle's reference element against what Sections 3-4 fix."""
import numpy as np
import pytest

from oracle.polys import REF_VERTS, OrthoBasis, quadrature, simplex_volume
from oracle.refelem import (EDGES, FACES, reference_element, eigenbasis, face_frames,
                            edge_frames, to_face, dcurl2, dcurl3)


def _bary(X):
    V = REF_VERTS[3]
    A = np.vstack([V.T, np.ones(4)])
    lam = np.linalg.solve(A, np.vstack([X.T, np.ones(X.shape[0])])).T
    G = np.linalg.inv(A)[:, :3]  # grad lambda_i (4, 3)
    return lam, G


def test_quadrature_monomials_closed_form():
    """Barycentric monomial integrals: int lam^a = a! d! |T| / (|a| + d)!."""
    from math import factorial
    X, w = quadrature(3, 7)
    lam, _ = _bary(X)
    vol = simplex_volume(REF_VERTS[3])
    for a in [(0, 0, 0, 0), (2, 1, 0, 3), (4, 0, 4, 2), (1, 1, 1, 1), (0, 6, 5, 0)]:
        if sum(a) > 11:
            continue
        exact = np.prod([factorial(x) for x in a]) * factorial(3) * vol / factorial(sum(a) + 3)
        num = np.sum(w * np.prod(lam ** np.array(a)[None, :], axis=1))
        assert abs(num - exact) < 1e-14 * max(1.0, exact)


def test_expansion_orthonormal():
    for dim in (1, 2, 3):
        B = OrthoBasis(dim, 9)
        X, w = quadrature(dim, 14)
        V, _ = B.eval(X)
        assert np.abs(V.T @ (w[:, None] * V) - np.eye(B.n)).max() < 1e-12


@pytest.mark.parametrize("space,p,n_ref", [("CG", 3, 20), ("CG", 5, 56), ("N1curl", 2, 20),
                                           ("N1curl", 4, 84), ("RT", 2, 15), ("RT", 4, 70),
                                           ("N2curl", 3, 60)])
def test_dimensions_and_unisolvence(space, p, n_ref):
    """n_ref from Eq. (2.5)/(2.6) and a nonsingular DOF matrix (Lemma 3.1)."""
    R = reference_element(space, p)
    assert R.ndofs == n_ref
    assert R.dof_cond < 1e4


def _n_interior(space, p):
    return {"CG": (p - 1) * (p - 2) * (p - 3) // 6,
            "N1curl": p * (p + 2) * (p + 3) // 2 - 6 * p - 4 * p * (p - 1),
            "RT": p * (p + 1) * (p - 1) // 2}[space]


@pytest.mark.parametrize("space,p", [("CG", 4), ("CG", 6), ("N1curl", 3), ("N1curl", 5),
                                     ("RT", 3), ("RT", 5)])
def test_lemma_4_5_block_structure(space, p):
    """Lemma 4.5: K_II = [I 0; 0 0], K_IG = 0, M_II = [Lambda 0; 0 I]."""
    R = reference_element(space, p)
    M, K = R.ref_matrices()
    I = R.interior
    assert len(I) == _n_interior(space, p)
    G = [i for i in range(R.ndofs) if i not in I]
    fam = {"CG": "CG", "N1curl": "N1", "RT": "RT"}[space]
    _, _, lam = eigenbasis(fam, p, 3)
    nI = nI_cell = len(lam)
    KII, MII = K[np.ix_(I, I)], M[np.ix_(I, I)]
    Kexp = np.zeros((len(I), len(I)))
    Kexp[:nI, :nI] = np.eye(nI)
    Mexp = np.eye(len(I))
    Mexp[:nI, :nI] = np.diag(lam)
    assert np.abs(KII - Kexp).max() < 1e-12
    assert np.abs(MII - Mexp).max() < 1e-12 * max(1.0, np.abs(M).max())
    assert np.abs(K[np.ix_(I, G)]).max() < 1e-12
    # type-II functions have zero stiffness rows everywhere (d phi^II = 0, Lemma 4.3)
    typeII = []
    for key, dofs in R.entity_dofs.items():
        if R.k == 1:
            nI = {1: 1, 2: len(eigenbasis("N1", p, 2)[2]), 3: nI_cell}.get(key[0], len(dofs))
        elif R.k == 2:
            nI = {2: 1, 3: nI_cell}[key[0]]
        else:
            nI = len(dofs)
        typeII += list(dofs[nI:])
    if R.k > 0:
        assert len(typeII) > 0
        assert np.abs(K[typeII, :]).max() < 1e-12


@pytest.mark.parametrize("p", [1, 2, 4])
def test_lemma_4_1_whitney(p):
    """Lemma 4.1: the first function of each k-entity is the Whitney form."""
    X, _ = quadrature(3, 4)
    lam, G = _bary(X)
    # H(grad): vertex functions are the barycentric coordinates
    R = reference_element("CG", p)
    v, _ = R.tabulate(X)
    for a in range(4):
        j = R.entity_dofs[(0, a)][0]
        assert np.abs(v[:, j, 0] - lam[:, a]).max() < 1e-12
    # H(curl): lam_a grad lam_b - lam_b grad lam_a
    R = reference_element("N1curl", p)
    v, _ = R.tabulate(X)
    for e, (a, b) in enumerate(EDGES):
        j = R.entity_dofs[(1, e)][0]
        w = lam[:, a, None] * G[b][None, :] - lam[:, b, None] * G[a][None, :]
        assert np.abs(v[:, j, :] - w).max() < 1e-12
    # H(div): 2 (lam_a gl_b x gl_c + lam_b gl_c x gl_a + lam_c gl_a x gl_b)
    R = reference_element("RT", p)
    v, _ = R.tabulate(X)
    for f, (a, b, c) in enumerate(FACES):
        j = R.entity_dofs[(2, f)][0]
        w = 2 * (lam[:, a, None] * np.cross(G[b], G[c])[None, :]
                 + lam[:, b, None] * np.cross(G[c], G[a])[None, :]
                 + lam[:, c, None] * np.cross(G[a], G[b])[None, :])
        assert np.abs(v[:, j, :] - w).max() < 1e-12


def _face_points():
    xi, _ = quadrature(2, 5)
    return xi


@pytest.mark.parametrize("p", [3, 5])
def test_lemma_4_2_traces_are_eigenfunctions(p):
    """Lemma 4.2: tr_S phi^I_{S,j} = psi_{S,j}; tr_S phi^II_{S,n} = d_S psi^{k-1}_{S,n}."""
    xi = _face_points()
    s = np.linspace(-0.9, 0.9, 7)
    # H(grad): face and edge type-I functions
    R = reference_element("CG", p)
    Ef, Yf, _ = eigenbasis("CG", p, 2)
    pf = Ef.tab(xi)[0][:, :, 0] @ Yf
    for f, fr in enumerate(face_frames()):
        v, _ = R.tabulate(to_face(xi, fr))
        dofs = R.entity_dofs[(2, f)]
        assert np.abs(v[:, dofs, 0] - pf).max() < 1e-11
        # functions of other faces vanish on this face
        other = [j for g in range(4) if g != f for j in R.entity_dofs[(2, g)]]
        assert np.abs(v[:, other, 0]).max() < 1e-11
    Ee, Ye, _ = eigenbasis("CG", p, 1)
    pe = Ee.tab(s[:, None])[0][:, :, 0] @ Ye
    for e, (mid, t) in enumerate(edge_frames()):
        v, _ = R.tabulate(mid[None, :] + s[:, None] * t[None, :])
        assert np.abs(v[:, R.entity_dofs[(1, e)], 0] - pe).max() < 1e-11
    # H(curl): tangential trace of face type-I = Psi_F, of face type-II = grad_F psi_F
    R = reference_element("N1curl", p)
    EN, YN, _ = eigenbasis("N1", p, 2)
    PsiF = np.einsum("pnc,nj->pjc", EN.tab(xi)[0], YN)
    gpsi = np.einsum("pncd,nj->pjd", Ef.tab(xi)[1], Yf)
    nI = YN.shape[1]
    for f, fr in enumerate(face_frames()):
        _, B, _ = fr
        v, _ = R.tabulate(to_face(xi, fr))
        tv = np.einsum("pjc,cd->pjd", v, B)
        dofs = R.entity_dofs[(2, f)]
        assert np.abs(tv[:, dofs[:nI], :] - PsiF).max() < 1e-11
        assert np.abs(tv[:, dofs[nI:], :] - gpsi).max() < 1e-11
    # H(div): normal trace of face type-II = curl_F Psi_F (second-kind Nedelec bubbles)
    R = reference_element("RT", p)
    E2, Y2, _ = eigenbasis("N2", p, 2)
    cps = dcurl2(E2.tab(xi)[1]) @ Y2
    for f, fr in enumerate(face_frames()):
        _, _, n = fr
        v, _ = R.tabulate(to_face(xi, fr))
        nv = np.einsum("pjc,c->pj", v, n)
        dofs = R.entity_dofs[(2, f)]
        assert np.abs(nv[:, dofs[1:]] - cps).max() < 1e-11
        assert np.abs(nv[:, dofs[0]] - 1.0 / np.sqrt(3.0)).max() < 1e-11  # Whitney: flux 1 / area


@pytest.mark.parametrize("p", [2, 3, 4])
def test_lemma_4_3_type_two_is_d_of_type_one(p):
    """Lemma 4.3: phi^{k,II}_{S,n} = d phi^{k-1,I}_{S,n} (H(curl) from CG_p, H(div) from NedTwo_p)."""
    X, _ = quadrature(3, 4)
    cg = reference_element("CG", p)
    ned = reference_element("N1curl", p)
    _, gcg = cg.tabulate(X)
    vn, _ = ned.tabulate(X)
    for key, dofs in ned.entity_dofs.items():
        if key[0] == 0:
            continue
        cdofs = cg.entity_dofs.get(key, [])
        nII = len(cdofs)
        if nII == 0:
            continue
        assert np.abs(vn[:, dofs[-nII:], :] - gcg[:, cdofs, :]).max() < 1e-11
    n2 = reference_element("N2curl", p)
    rt = reference_element("RT", p)
    _, cn2 = n2.tabulate(X)
    vr, _ = rt.tabulate(X)
    for key, dofs in rt.entity_dofs.items():
        n2d = n2.entity_dofs.get(key, [])
        if key[0] == 2:
            nI = len(n2d) - len(reference_element("CG", p + 1).entity_dofs[key])
            assert np.abs(vr[:, dofs[1:], :] - cn2[:, n2d[:nI], :]).max() < 1e-11
        if key[0] == 3:
            nI = len(n2d) - len(reference_element("CG", p + 1).entity_dofs.get(key, []))
            if nI:
                assert np.abs(vr[:, dofs[-nI:], :] - cn2[:, n2d[:nI], :]).max() < 1e-11


def test_eigenbasis_equation_3_9():
    """(d psi_i, d psi_j) = delta_ij and (psi_i, psi_j) = lambda_i delta_ij on the cell."""
    from oracle.refelem import d_gram
    for fam, p in [("CG", 6), ("N1", 4), ("RT", 4), ("N2", 3)]:
        E, Y, lam = eigenbasis(fam, p, 3)
        K = Y.T @ d_gram(E, fam, 3) @ Y
        M = Y.T @ Y  # the expansion is L2-orthonormal
        assert np.abs(K - np.eye(len(lam))).max() < 1e-11
        assert np.abs(M - np.diag(lam)).max() < 1e-13
        assert np.all(np.diff(lam) <= 1e-12 * lam[0])
