"""The paper's orthogonality-promoting reference element (Sections 3-4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Section 3 in the paper's order:

1. the local spaces of Eq. (2.5) (first kind) and Eq. (2.6) (second kind:
   NedTwo_p and BDM_p as solution spaces, and NedTwo bubbles inside the
   H(div) degrees of freedom, Section 3.4.3);
2. the bubble spaces of Section 3.1 on every subsimplex;
3. the augmented eigenproblem Eq. (3.10) on the bubble space, dropping the
   kernel of d (the type-II part, Eq. (3.5)) and rescaling the rest so that
   Eq. (3.9) holds;
4. the degrees of freedom Eq. (3.14) (H(grad)), Eq. (3.16) (H(curl)),
   Eq. (3.18) (H(div));
5. the Ciarlet dual basis (Section 4, first display).

Readings of what the paper leaves open (each also listed in the design notes):

* Reference simplices: equilateral, edge length 2, centroid 0
  (``polys.REF_VERTS``).  A face (edge) of the tetrahedron is parametrised by
  the isometric affine map sending the reference triangle's (interval's)
  vertices, in order, onto the face's (edge's) vertices in increasing order.
* Edge tangent t = (x_b - x_a)/|x_b - x_a| and face normal
  n = (x_b - x_a) x (x_c - x_a)/|.| for increasing local vertex order a<b<c.
  The surface curl of a tangential field is n . curl.
* Kernel selection in Eq. (3.10): the eigenpairs with the smallest mu are
  dropped, exactly as many as dim d X^{k-1}(S) (known from Eq. (3.8)).
* Eigenvectors are fixed up to sign and, on the symmetric face and cell, up
  to rotations inside degenerate eigenspaces.  They are ordered by increasing
  mu; eigenvalues whose relative spread is below ``CLUSTER_RTOL`` form one
  cluster, whose basis is made unique by the echelon rule: the j-th vector of
  a cluster of size m is annihilated by probe functionals 1..j-1 and is
  positive on probe j (probes: point values, or point values of the field
  dotted with a fixed direction, at fixed interior points).
* Order of the degrees of freedom: vertices 0..3; edges 01,02,03,12,13,23;
  faces 012,013,023,123; interior.  Inside an entity: Whitney, type I,
  type II, each in eigen order.
"""
import numpy as np

from .polys import REF_VERTS, OrthoBasis, quadrature, dim_P

CLUSTER_RTOL = 1e-8

EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
FACES = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]


# ---------------------------------------------------------------------------
# probe functionals used to make degenerate eigenbases unique
# ---------------------------------------------------------------------------
def probe_points(dim, m):
    """m fixed interior points of the reference simplex of dimension dim."""
    V = REF_VERTS[dim]
    pts = []
    for i in range(m):
        b = np.array([1.0 + 0.5 * np.sin(1.7 * (i + 1) * (j + 1) + 0.3 * (j + 1) ** 2)
                      for j in range(dim + 1)])
        b /= b.sum()
        pts.append(b @ V)
    return np.array(pts)


def probe_dirs(dim, m):
    """m fixed unit directions in R^dim."""
    out = []
    for i in range(m):
        c = np.array([np.cos(0.9 * (i + 1) * (l + 1) + 0.5 * l + 0.25) for l in range(dim)])
        out.append(c / np.linalg.norm(c))
    return np.array(out)


# ---------------------------------------------------------------------------
# vector-valued expansions: coefficient index = component * nP + k
# ---------------------------------------------------------------------------
class Expansion:
    """Scalar (ncomp=1) or vector (ncomp=dim) polynomials of degree <= deg."""

    def __init__(self, dim, deg, ncomp):
        self.dim, self.deg, self.ncomp = dim, deg, ncomp
        self.B = OrthoBasis(dim, deg)
        self.nP = self.B.n
        self.n = ncomp * self.nP

    def tab(self, Y):
        """values (npt, n, ncomp) and Jacobians (npt, n, ncomp, dim) of the expansion."""
        V, G = self.B.eval(Y)
        npt = V.shape[0]
        val = np.zeros((npt, self.n, self.ncomp))
        jac = np.zeros((npt, self.n, self.ncomp, self.dim))
        for c in range(self.ncomp):
            val[:, c * self.nP:(c + 1) * self.nP, c] = V
            jac[:, c * self.nP:(c + 1) * self.nP, c, :] = G
        return val, jac

    def project(self, F, X, w):
        """L2 projection coefficients of fields with values F (npt, nf, ncomp) at rule (X, w)."""
        val, _ = self.tab(X)
        return np.einsum("pnc,pfc,p->nf", val, F, w, optimize=True)


def dcurl3(jac):
    """curl from Jacobian (..., 3, 3) with jac[..., c, d] = d f_c / d x_d."""
    return np.stack([jac[..., 2, 1] - jac[..., 1, 2],
                     jac[..., 0, 2] - jac[..., 2, 0],
                     jac[..., 1, 0] - jac[..., 0, 1]], -1)


def dcurl2(jac):
    """scalar 2D curl d f_2/dx_1 - d f_1/dx_2."""
    return jac[..., 1, 0] - jac[..., 0, 1]


def ddiv(jac):
    return np.trace(jac, axis1=-2, axis2=-1)


def range_basis(S, rank, what):
    """Orthonormal basis of the column space of S with known rank (SVD)."""
    U, s, _ = np.linalg.svd(S, full_matrices=False)
    if rank < len(s):
        assert s[rank] < 1e-9 * s[0], (what, s[rank] / s[0])
    assert s[rank - 1] > 1e-7 * s[0], (what, s[rank - 1] / s[0])
    return U[:, :rank]


def null_basis(C, dim, what):
    """Orthonormal basis of the null space of C with known dimension (SVD)."""
    _, s, Vt = np.linalg.svd(C, full_matrices=True)
    n = C.shape[1]
    sv = np.zeros(n)
    sv[:len(s)] = s
    # singular values sorted descending; the last ``dim`` must vanish
    assert sv[n - dim - 1] > 1e-8 * sv[0], (what, sv[n - dim - 1] / sv[0])
    if dim > 0:
        assert sv[n - dim] < 1e-10 * sv[0], (what, sv[n - dim] / sv[0])
    return Vt[n - dim:].T


# ---------------------------------------------------------------------------
# the spaces of Eqs. (2.5)-(2.6) on the reference simplex of dimension dim
# ---------------------------------------------------------------------------
def space(family, p, dim):
    """Return (Expansion, U) with U an L2-orthonormal basis of the space.

    family: 'CG' (P_p), 'N1' (first-kind Nedelec, P_{p-1}^d + P_{p-1}^d x x,
    in 2D P_{p-1}^2 + P_{p-1} x^perp), 'N2' (second kind, P_p^d),
    'RT' (P_{p-1}^3 + P_{p-1} x, 3D only), 'BDM' (second kind, P_p^3, Eq. (2.6)).
    """
    if family == "CG":
        E = Expansion(dim, p, 1)
        return E, np.eye(E.n)
    if family == "DG":  # the last space of the complex whose X^{d-1} is RT_p: P_{p-1}
        E = Expansion(dim, p - 1, 1)
        return E, np.eye(E.n)
    E = Expansion(dim, p, dim)
    if family in ("N2", "BDM"):
        return E, np.eye(E.n)
    X, w = quadrature(dim, p + 2)
    Elow = Expansion(dim, p - 1, 1)
    low, _ = Elow.tab(X)
    low = low[:, :, 0]  # (npt, nlow)
    fields = []
    for c in range(dim):  # P_{p-1}^dim
        F = np.zeros((X.shape[0], Elow.n, dim))
        F[:, :, c] = low
        fields.append(F)
    if family == "N1" and dim == 3:
        for c in range(dim):  # (q e_c) x x
            e = np.zeros(3)
            e[c] = 1.0
            ex = np.cross(e[None, :], X)  # (npt, 3)
            fields.append(low[:, :, None] * ex[:, None, :])
        rank = p * (p + 2) * (p + 3) // 2
    elif family == "N1" and dim == 2:
        xp = np.stack([-X[:, 1], X[:, 0]], 1)
        fields.append(low[:, :, None] * xp[:, None, :])
        rank = p * (p + 2)
    elif family == "RT" and dim == 3:
        fields.append(low[:, :, None] * X[:, None, :])
        rank = p * (p + 1) * (p + 3) // 2
    else:
        raise ValueError(family)
    F = np.concatenate(fields, 1)
    S = E.project(F, X, w)
    return E, range_basis(S, rank, (family, p, dim))


# ---------------------------------------------------------------------------
# bubbles and the eigenproblems Eqs. (3.9)-(3.10)
# ---------------------------------------------------------------------------
def _edge_points_of_simplex(dim, npts):
    """points on every edge of the reference simplex (dim 2 or 3) with unit tangents."""
    V = REF_VERTS[dim]
    g, _ = np.polynomial.legendre.leggauss(npts)
    out = []
    for a in range(dim + 1):
        for b in range(a + 1, dim + 1):
            t = (V[b] - V[a]) / np.linalg.norm(V[b] - V[a])
            X = 0.5 * (V[a] + V[b])[None, :] + 0.5 * g[:, None] * (V[b] - V[a])[None, :]
            out.append((X, t))
    return out


def face_frames():
    """For each face of the reference tetrahedron: (origin map, B (3x2), n).

    x(xi) = V_a + B (xi - r_0), B = [V_b - V_a, V_c - V_a] R^{-1}, with R the
    edge vectors of the reference triangle.  B is an isometry.
    """
    V = REF_VERTS[3]
    r = REF_VERTS[2]
    R = np.stack([r[1] - r[0], r[2] - r[0]], 1)
    out = []
    for (a, b, c) in FACES:
        E = np.stack([V[b] - V[a], V[c] - V[a]], 1)
        B = E @ np.linalg.inv(R)
        n = np.cross(B[:, 0], B[:, 1])
        out.append((V[a], B, n))
    return out


def edge_frames():
    """For each edge of the reference tetrahedron: (midpoint, unit tangent)."""
    V = REF_VERTS[3]
    return [(0.5 * (V[a] + V[b]), 0.5 * (V[b] - V[a])) for (a, b) in EDGES]


def to_face(xi, frame):
    r0 = REF_VERTS[2][0]
    Va, B, _ = frame
    return Va[None, :] + (xi - r0[None, :]) @ B.T


def bubbles(family, p, dim):
    """Expansion and L2-orthonormal basis Z of the bubble space (vanishing trace on the boundary)."""
    E, U = space(family, p, dim)
    if dim == 1:
        val, _ = E.tab(REF_VERTS[1])
        C = val[:, :, 0]
        bdim = p - 1
    elif dim == 2:
        rows = []
        for X, t in _edge_points_of_simplex(2, p + 1):
            val, _ = E.tab(X)
            if family == "CG":
                rows.append(val[:, :, 0])
            else:
                rows.append(np.einsum("pnc,c->pn", val, t, optimize=True))
        C = np.concatenate(rows, 0)
        bdim = {"CG": (p - 1) * (p - 2) // 2, "N1": p * (p - 1), "N2": (p + 1) * (p - 1)}[family]
    else:
        xi, _ = quadrature(2, p + 1)
        rows = []
        for fr in face_frames():
            X = to_face(xi, fr)
            val, _ = E.tab(X)
            _, B, n = fr
            if family == "CG":
                rows.append(val[:, :, 0])
            elif family in ("N1", "N2"):
                tv = np.einsum("pnc,cd->pnd", val, B, optimize=True)
                rows.append(tv[:, :, 0])
                rows.append(tv[:, :, 1])
            else:
                rows.append(np.einsum("pnc,c->pn", val, n, optimize=True))
        C = np.concatenate(rows, 0)
        nsp = U.shape[1]
        bdim = {"CG": (p - 1) * (p - 2) * (p - 3) // 6,
                "N1": nsp - 6 * p - 4 * p * (p - 1),
                "N2": nsp - 6 * (p + 1) - 4 * (p + 1) * (p - 1),
                "RT": nsp - 4 * p * (p + 1) // 2,
                "BDM": nsp - 4 * (p + 1) * (p + 2) // 2}[family]
    if bdim == 0:
        return E, np.zeros((E.n, 0))
    Zs = null_basis(C @ U, bdim, ("bubbles", family, p, dim))
    return E, U @ Zs


def d_gram(E, family, dim):
    """Gram matrix of d (grad, curl or div) of the expansion on the reference simplex."""
    X, w = quadrature(dim, E.deg + 2)
    val, jac = E.tab(X)
    if family == "CG":
        D = jac[:, :, 0, :]  # gradient (npt, n, dim)
    elif family in ("N1", "N2"):
        D = dcurl3(jac) if dim == 3 else dcurl2(jac)[..., None]
    else:
        D = ddiv(jac)[..., None]
    return np.einsum("pnc,pmc,p->nm", D, D, w, optimize=True)


def kernel_dim(family, p, dim):
    """dim d X^{k-1}(S) inside the bubble space (Eq. (3.8)): the dropped eigenpairs."""
    if family == "CG":
        return 0
    if family == "N1":  # grad of CG_p bubbles
        return {2: (p - 1) * (p - 2) // 2, 3: (p - 1) * (p - 2) * (p - 3) // 6}[dim]
    if family == "N2":  # grad of CG_{p+1} bubbles
        return {2: p * (p - 1) // 2, 3: p * (p - 1) * (p - 2) // 6}[dim]
    if family == "RT":  # RT bubbles minus div range (mean-free P_{p-1})
        nb = p * (p + 1) * (p - 1) // 2
        return nb - (dim_P(3, p - 1) - 1)
    if family == "BDM":  # BDM bubbles minus div range (mean-free P_{p-1}, as for RT_p)
        nb = (p + 1) * (p + 2) * (p - 1) // 2
        return nb - (dim_P(3, p - 1) - 1)
    raise ValueError(family)


def canonicalize(E, Y, mu, dim):
    """Order by mu and make each eigen-cluster basis unique (echelon rule on probes)."""
    order = np.argsort(mu, kind="stable")
    mu = mu[order]
    Y = Y[:, order]
    ncols = Y.shape[1]
    out = Y.copy()
    i = 0
    while i < ncols:
        j = i + 1
        while j < ncols and (mu[j] - mu[j - 1]) <= CLUSTER_RTOL * abs(mu[j]):
            j += 1
        m = j - i
        P = probe_points(dim, m)
        val, _ = E.tab(P)
        if E.ncomp == 1:
            Pm = val[:, :, 0]
        else:
            Pm = np.einsum("pnc,pc->pn", val, probe_dirs(dim, m), optimize=True)
        G = Pm @ Y[:, i:j]  # (m, m)
        Q, R = np.linalg.qr(G.T)
        s = np.sign(np.diag(R))
        assert np.all(np.abs(np.diag(R)) > 1e-8 * np.abs(G).max()), "probe matrix singular"
        out[:, i:j] = Y[:, i:j] @ (Q * s[None, :])
        i = j
    return out, mu


def eigenbasis(family, p, dim):
    """Type-I eigenbasis psi_j of Eq. (3.9) on the reference simplex of dimension dim.

    Returns (E, coefficients (E.n, N), lambda (N,)).  Solves the augmented
    problem Eq. (3.10) on the L2-orthonormal bubble basis (so the mass matrix
    is the identity), drops the kernel and rescales psi = psi_hat / sqrt(mu).
    """
    E, Z = bubbles(family, p, dim)
    if Z.shape[1] == 0:
        return E, Z, np.zeros(0)
    K = Z.T @ d_gram(E, family, dim) @ Z
    K = 0.5 * (K + K.T)
    mu, v = np.linalg.eigh(K)
    nk = kernel_dim(family, p, dim)
    if nk > 0:
        assert mu[nk - 1] < 1e-9 * mu[-1], ("kernel", family, p, dim, mu[nk - 1] / mu[-1])
    assert mu[nk] > 1e-7 * mu[-1], ("gap", family, p, dim)
    mu = mu[nk:]
    Y = (Z @ v[:, nk:]) / np.sqrt(mu)[None, :]
    Y, mu = canonicalize(E, Y, mu, dim)
    return E, Y, 1.0 / mu


# ---------------------------------------------------------------------------
# degrees of freedom (Eqs. (3.14), (3.16), (3.18)) and the dual basis
# ---------------------------------------------------------------------------
class RefElement:
    """Reference element of the paper for space in {'CG', 'N1curl', 'N2curl', 'RT', 'BDM', 'DG'}, degree p.

    First kind (Eq. (2.5)): CG_p, Ned1_p ('N1curl'), RT_p.  Second kind (Eq. (2.6)): NedTwo_p = P_p^3
    ('N2curl'), whose gradient moments use the CG_{p+1} eigenbasis (Section 3.4.2), and BDM_p = P_p^3
    ('BDM'), whose face and curl moments use the NedTwo_{p+1} eigenbasis and whose divergence moments use
    the eigenbasis of its own interior bubbles (Section 3.4.3).  RT_p's face and curl moments use the
    NedTwo_p eigenbasis (the second-kind choice of Section 3.4.3).  'DG' is
    X^3 = DG_{p-1} of the complex ending in RT_p (the k = 3 Hodge-Laplace problem):
    the cell DOFs of the abstract definition with k = d, i.e. the mean (1, v)_T and
    the moments (div Phi_{C,j}, v)_T against the divergences of the RT_p interior
    eigenbasis; v pulls back as a 3-form, v = v_hat / det J.

    Attributes
    ----------
    E       : 3D expansion (scalar for CG, vector otherwise)
    Phi     : (E.n, n_ref) coefficients of the dual basis phi_j
    ndofs   : n_ref
    entity_dofs : dict (dim, local entity index) -> list of local DOF indices
    interior: list of local DOF indices of the cell interior
    """

    def __init__(self, space_name, p):
        self.space, self.p = space_name, p
        fam = {"CG": "CG", "N1curl": "N1", "N2curl": "N2", "RT": "RT", "BDM": "BDM", "DG": "DG"}[space_name]
        self.k = {"CG": 0, "N1curl": 1, "N2curl": 1, "RT": 2, "BDM": 2, "DG": 3}[space_name]
        self.fam = fam
        # the H(grad) degree of the complex X^0 -> X^1 used by the H(curl) DOFs
        self.p0 = p + 1 if fam == "N2" else p
        # the degree of the second-kind H(curl) space X^1 -> X^2 used by the H(div) DOFs
        self.p1 = p + 1 if fam == "BDM" else p
        E, U = space(fam, p, 3)
        self.E = E
        L, ent = self._functionals(E)
        D = L @ U
        self.ndofs = D.shape[0]
        assert D.shape == (U.shape[1], U.shape[1]), (D.shape, U.shape)
        self.dof_cond = np.linalg.cond(D)
        self.Phi = U @ np.linalg.inv(D)
        self.entity_dofs = ent
        self.interior = ent[(3, 0)]

    # ----- the functionals, entity by entity, in the documented order -----
    def _functionals(self, E):
        p, k = self.p, self.k
        rows = []
        ent = {}

        def add(key, R):
            start = sum(r.shape[0] for r in rows)
            rows.append(R)
            ent.setdefault(key, []).extend(range(start, start + R.shape[0]))

        if k == 3:  # DG_{p-1}: only cell DOFs
            Xc, wc = quadrature(3, p + 2)
            val, _ = E.tab(Xc)
            add((3, 0), (wc[:, None] * val[:, :, 0]).sum(0)[None, :])  # Whitney (1, v)_T
            ER, YR, _ = eigenbasis("RT", p, 3)
            if YR.shape[1]:
                _, jR = ER.tab(Xc)
                dphi = np.einsum("pn,nj->pj", ddiv(jR), YR, optimize=True)
                add((3, 0), np.einsum("pj,pn,p->jn", dphi, val[:, :, 0], wc, optimize=True))  # type II
            return np.concatenate(rows, 0), ent

        V3 = REF_VERTS[3]
        # edge and face rules (intrinsic coordinates)
        s, ws = np.polynomial.legendre.leggauss(p + 2)
        xi, wf = quadrature(2, p + 2)
        Xc, wc = quadrature(3, p + 2)

        if k == 0:
            for a in range(4):
                val, _ = E.tab(V3[a:a + 1])
                add((0, a), val[:, :, 0])
        if k in (0, 1):
            Eb, Y, _ = eigenbasis("CG", self.p0, 1)
            vb, gb = Eb.tab(s[:, None])
            dpsi = np.einsum("pn,nj->pj", gb[:, :, 0, 0], Y, optimize=True)  # d psi / ds
            for e, (mid, t) in enumerate(edge_frames()):
                X = mid[None, :] + s[:, None] * t[None, :]
                val, jac = E.tab(X)
                if k == 0:  # (grad_E psi, grad_E v)_E
                    tg = np.einsum("pnd,d->pn", jac[:, :, 0, :], t, optimize=True)
                    add((1, e), np.einsum("pj,pn,p->jn", dpsi, tg, ws, optimize=True))
                else:
                    tv = np.einsum("pnc,c->pn", val, t, optimize=True)
                    add((1, e), (ws[:, None] * tv).sum(0)[None, :])  # Whitney (1, t.v)_E
                    add((1, e), np.einsum("pj,pn,p->jn", dpsi, tv, ws, optimize=True))  # type II
        if k == 0:
            Ef, Y, _ = eigenbasis("CG", p, 2)
            _, gf = Ef.tab(xi)
            gpsi = np.einsum("pnd,nj->pjd", gf[:, :, 0, :], Y, optimize=True)
            for f, fr in enumerate(face_frames()):
                val, jac = E.tab(to_face(xi, fr))
                _, B, _ = fr
                tg = np.einsum("pnd,de->pne", jac[:, :, 0, :], B, optimize=True)
                add((2, f), np.einsum("pjd,pnd,p->jn", gpsi, tg, wf, optimize=True))
        elif k == 1:
            EN, YN, _ = eigenbasis(self.fam, p, 2)
            _, jN = EN.tab(xi)
            cpsi = np.einsum("pn,nj->pj", dcurl2(jN), YN, optimize=True)
            Ef, Y, _ = eigenbasis("CG", self.p0, 2)
            _, gf = Ef.tab(xi)
            gpsi = np.einsum("pnd,nj->pjd", gf[:, :, 0, :], Y, optimize=True)
            for f, fr in enumerate(face_frames()):
                val, jac = E.tab(to_face(xi, fr))
                _, B, n = fr
                nc = np.einsum("pnc,c->pn", dcurl3(jac), n, optimize=True)
                add((2, f), np.einsum("pj,pn,p->jn", cpsi, nc, wf, optimize=True))  # type I
                tv = np.einsum("pnc,cd->pnd", val, B, optimize=True)
                add((2, f), np.einsum("pjd,pnd,p->jn", gpsi, tv, wf, optimize=True))  # type II
        else:
            EN, YN, _ = eigenbasis("N2", self.p1, 2)
            _, jN = EN.tab(xi)
            cpsi = np.einsum("pn,nj->pj", dcurl2(jN), YN, optimize=True)
            for f, fr in enumerate(face_frames()):
                val, _ = E.tab(to_face(xi, fr))
                _, B, n = fr
                nv = np.einsum("pnc,c->pn", val, n, optimize=True)
                add((2, f), (wf[:, None] * nv).sum(0)[None, :])  # Whitney (1, n.v)_F
                add((2, f), np.einsum("pj,pn,p->jn", cpsi, nv, wf, optimize=True))  # type II
        # interior
        val, jac = E.tab(Xc)
        if k == 0:
            Ec, Y, _ = eigenbasis("CG", p, 3)
            if Y.shape[1]:
                _, gc = Ec.tab(Xc)
                gpsi = np.einsum("pnd,nj->pjd", gc[:, :, 0, :], Y, optimize=True)
                add((3, 0), np.einsum("pjd,pnd,p->jn", gpsi, jac[:, :, 0, :], wc, optimize=True))
        elif k == 1:
            EN, YN, _ = eigenbasis(self.fam, p, 3)
            if YN.shape[1]:
                _, jN = EN.tab(Xc)
                cpsi = np.einsum("pnc,nj->pjc", dcurl3(jN), YN, optimize=True)
                add((3, 0), np.einsum("pjc,pnc,p->jn", cpsi, dcurl3(jac), wc, optimize=True))
            Ec, Y, _ = eigenbasis("CG", self.p0, 3)
            if Y.shape[1]:
                _, gc = Ec.tab(Xc)
                gpsi = np.einsum("pnd,nj->pjd", gc[:, :, 0, :], Y, optimize=True)
                add((3, 0), np.einsum("pjd,pnd,p->jn", gpsi, val, wc, optimize=True))
        else:
            ER, YR, _ = eigenbasis(self.fam, p, 3)
            if YR.shape[1]:
                _, jR = ER.tab(Xc)
                dphi = np.einsum("pn,nj->pj", ddiv(jR), YR, optimize=True)
                add((3, 0), np.einsum("pj,pn,p->jn", dphi, ddiv(jac), wc, optimize=True))
            EN, YN, _ = eigenbasis("N2", self.p1, 3)
            if YN.shape[1]:
                _, jN = EN.tab(Xc)
                cpsi = np.einsum("pnc,nj->pjc", dcurl3(jN), YN, optimize=True)
                add((3, 0), np.einsum("pjc,pnc,p->jn", cpsi, val, wc, optimize=True))
        ent.setdefault((3, 0), [])
        return np.concatenate(rows, 0), ent

    # ----- tabulation of the dual basis -----
    def tabulate(self, X):
        """Reference basis at points X (npt, 3): values (npt, n_ref, ncomp) and
        d (npt, n_ref, dcomp): gradient (3), curl (3) or div (1)."""
        val, jac = self.E.tab(X)
        v = np.einsum("pnc,nj->pjc", val, self.Phi, optimize=True)
        J = np.einsum("pncd,nj->pjcd", jac, self.Phi, optimize=True)
        if self.k == 0:
            d = J[:, :, 0, :]
        elif self.k == 1:
            d = dcurl3(J)
        elif self.k == 2:
            d = ddiv(J)[..., None]
        else:  # d^3 = 0
            d = np.zeros(v.shape[:2] + (1,))
        return v, d

    def ref_matrices(self):
        """Reference mass and d-stiffness matrices on the reference tetrahedron."""
        X, w = quadrature(3, self.p + 2)
        v, d = self.tabulate(X)
        M = np.einsum("pic,pjc,p->ij", v, v, w, optimize=True)
        K = np.einsum("pic,pjc,p->ij", d, d, w, optimize=True)
        return M, K


_CACHE = {}


def reference_element(space_name, p):
    """Cached RefElement."""
    key = (space_name, p)
    if key not in _CACHE:
        _CACHE[key] = RefElement(space_name, p)
    return _CACHE[key]
