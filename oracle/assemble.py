"""Assembly, preconditioner and solvers for the Riesz maps (Eq. (2.8), Sections 6-7).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Element matrices are computed by quadrature of the reference basis under
  the pullbacks of Eq. (2.7) (not through precomputed geometric factors):
  A_T[i, j] = sum_q w_q |det J| (beta v_i . v_j + alpha d v_i . d v_j) with
  v = pullback of the reference function at the mapped quadrature point.
* The preconditioner is the interior/interface splitting of Eq. (6.11) read
  as one-level additive Schwarz: P^{-1} = D_II^{-1} (+) sum_V R_V^T A_V^{-1} R_V,
  A_V the assembled matrix restricted to the patch of vertex V, factorised by
  dense Cholesky.  (The paper's W^k coarse space and multiplicative hybrid
  weighting, Section 7.1, are not part of this reading.)
* PCG (Section 7.1) from x0 = 0, stopped when the true relative residual
  ||b - A x||_2 / ||b||_2 <= rtol.
"""
import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from .polys import REF_VERTS, quadrature


def jacobians(verts, cells):
    """J_T (nc, 3, 3) of the affine maps from the reference tetrahedron to sorted cells."""
    cells = np.sort(cells, axis=1)
    X = verts[cells]  # (nc, 4, 3)
    Ep = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], 2)
    V = REF_VERTS[3]
    Er = np.stack([V[1] - V[0], V[2] - V[0], V[3] - V[0]], 1)
    J = Ep @ np.linalg.inv(Er)
    return J, X[:, 0]


def physical_tabulation(ref, J, vhat, dhat):
    """Pullbacks (Eq. (2.7)) of reference values/derivatives for every cell.

    vhat (npt, n, ncomp), dhat (npt, n, dcomp) -> v (nc, npt, n, ncomp), d (nc, npt, n, dcomp)
    """
    det = np.linalg.det(J)
    if ref.k == 0:
        v = np.broadcast_to(vhat[None], (J.shape[0],) + vhat.shape)
        JiT = np.linalg.inv(J).transpose(0, 2, 1)
        d = np.einsum("cab,pnb->cpna", JiT, dhat)
    elif ref.k == 1:
        JiT = np.linalg.inv(J).transpose(0, 2, 1)
        v = np.einsum("cab,pnb->cpna", JiT, vhat)
        d = np.einsum("cab,pnb->cpna", J, dhat) / det[:, None, None, None]
    elif ref.k == 2:
        v = np.einsum("cab,pnb->cpna", J, vhat) / det[:, None, None, None]
        d = dhat[None] / det[:, None, None, None]
    else:  # 3-forms (DG): v = v_hat / det J, d = 0
        v = vhat[None] / det[:, None, None, None]
        d = np.zeros((J.shape[0],) + dhat.shape)
    return v, d, det


def element_matrices(ref, verts, cells, alpha=1.0, beta=1.0, chunk=256):
    """A_T for every cell by quadrature, (nc, n_ref, n_ref)."""
    X, w = quadrature(3, ref.p + 2)
    vhat, dhat = ref.tabulate(X)
    J, _ = jacobians(verts, cells)
    nc = J.shape[0]
    out = np.zeros((nc, ref.ndofs, ref.ndofs))
    for s in range(0, nc, chunk):
        v, d, det = physical_tabulation(ref, J[s:s + chunk], vhat, dhat)
        wq = w[None, :] * np.abs(det)[:, None]
        vw = v * wq[:, :, None, None]
        dw = d * wq[:, :, None, None]
        out[s:s + chunk] = (beta * np.einsum("epia,epja->eij", vw, v, optimize=True)
                            + alpha * np.einsum("epia,epja->eij", dw, d, optimize=True))
    return out


def assemble(md, Ae):
    """Global CSR matrix from element matrices and the cell DOF map."""
    nc, n, _ = Ae.shape
    rows = np.repeat(md.cell_dofs, n, axis=1).ravel()
    cols = np.tile(md.cell_dofs, (1, n)).ravel()
    A = scipy.sparse.coo_matrix((Ae.ravel(), (rows, cols)), shape=(md.ndofs, md.ndofs))
    return A.tocsr()


def load_cg_field(ref, md, ref_cg, md_cg, fcoef):
    """b_i = (f, phi_i) for f with components in the CG_p space of the same mesh.

    fcoef: (ncomp_f, N_CG) global coefficients of each Cartesian component of f
    in the paper's CG_p basis (a scalar space takes one component).
    """
    X, w = quadrature(3, ref.p + 2)
    vhat, dhat = ref.tabulate(X)
    chat, _ = ref_cg.tabulate(X)  # (npt, n_cg, 1)
    J, _ = jacobians(md.verts, md.cells)
    v, _, det = physical_tabulation(ref, J, vhat, dhat)
    fq = np.einsum("pa,mea->epm", chat[:, :, 0], fcoef[:, md_cg.cell_dofs])  # (nc, npt, ncomp)
    be = np.einsum("epm,epim,p,e->ei", fq, v, w, np.abs(det))
    b = np.zeros(md.ndofs)
    np.add.at(b, md.cell_dofs, be)
    return b


def load_function(ref, md, f, df=None, alpha=1.0, beta=1.0):
    """b_i = a(u, phi_i) (df given) or (f, phi_i) for a function of physical x.

    f(x) -> (npt, ncomp); df(x) -> (npt, dcomp) the exterior derivative of f.
    """
    X, w = quadrature(3, ref.p + 3)
    vhat, dhat = ref.tabulate(X)
    J, x0 = jacobians(md.verts, md.cells)
    V = REF_VERTS[3]
    xq = x0[:, None, :] + np.einsum("cab,pb->cpa", J, X - V[0][None, :])
    v, d, det = physical_tabulation(ref, J, vhat, dhat)
    nc, npt = xq.shape[:2]
    fx = f(xq.reshape(-1, 3)).reshape(nc, npt, -1)
    be = beta * np.einsum("epm,epim,p,e->ei", fx, v, w, np.abs(det))
    if df is not None:
        dx = df(xq.reshape(-1, 3)).reshape(nc, npt, -1)
        be += alpha * np.einsum("epm,epim,p,e->ei", dx, d, w, np.abs(det))
    b = np.zeros(md.ndofs)
    np.add.at(b, md.cell_dofs, be)
    return b


def evaluate(ref, md, x, Xref):
    """Values of the finite element function with coefficients x at mapped reference points."""
    vhat, dhat = ref.tabulate(Xref)
    J, x0 = jacobians(md.verts, md.cells)
    v, _, _ = physical_tabulation(ref, J, vhat, dhat)
    V = REF_VERTS[3]
    xq = x0[:, None, :] + np.einsum("cab,pb->cpa", J, Xref - V[0][None, :])
    return xq, np.einsum("epia,ei->epa", v, x[md.cell_dofs])


class Preconditioner:
    """P^{-1} = D_II^{-1} (+) sum_V R_V^T A_V^{-1} R_V (Eq. (6.11), one-level additive)."""

    def __init__(self, A, md, patches=None):
        self.N = A.shape[0]
        self.n_interface = md.n_interface
        d = A.diagonal()
        self.dinv_I = 1.0 / d[md.n_interface:]
        self.patches = md.patches() if patches is None else patches
        self.factors = []
        A = A.tocsr()
        for idx in self.patches:
            if len(idx) == 0:
                self.factors.append(None)
                continue
            AV = A[idx][:, idx].toarray()
            self.factors.append(scipy.linalg.cho_factor(AV, lower=True))

    def apply(self, r):
        z = np.zeros_like(r)
        z[self.n_interface:] = self.dinv_I * r[self.n_interface:]
        for idx, fac in zip(self.patches, self.factors):
            if fac is not None:
                z[idx] += scipy.linalg.cho_solve(fac, r[idx])
        return z

    def dense(self):
        """The explicit matrix P^{-1} (small problems only)."""
        I = np.eye(self.N)
        return np.stack([self.apply(I[:, j]) for j in range(self.N)], 1)


def coarse_dofs(md):
    """Global indices of the lowest-order DOFs: the first type-I DOF of every vertex (H1), edge
    (H(curl)) or face (H(div)).  By Lemma 4.1 their basis functions are the Whitney forms, so
    they span W^k, the first summand of the PAFW decomposition (Section 6.2)."""
    nv_d, ne_d, nf_d, _ = md.per_entity
    off_v, off_e, off_f = md._offsets
    if nv_d:
        return off_v + nv_d * np.arange(md.nverts)
    if ne_d:
        return off_e + ne_d * np.arange(len(md.edges))
    return off_f + nf_d * np.arange(len(md.faces))


def coarse_matrix(ref, md, alpha=1.0, beta=1.0):
    """A_0 = R_0 A R_0^T by quadrature of the lowest-order basis functions only (one per k-entity
    of each cell), assembled in the numbering of coarse_dofs; cheap at any mesh size."""
    k = ref.k
    nloc = {0: 4, 1: 6, 2: 4}[k]
    loc = [ref.entity_dofs[(k, s)][0] for s in range(nloc)]
    X, w = quadrature(3, ref.p + 2)
    vhat, dhat = ref.tabulate(X)
    J, _ = jacobians(md.verts, md.cells)
    v, d, det = physical_tabulation(ref, J, vhat[:, loc], dhat[:, loc])
    wq = w[None, :] * np.abs(det)[:, None]
    Ae = (beta * np.einsum("epia,epja,ep->eij", v, v, wq) + alpha * np.einsum("epia,epja,ep->eij", d, d, wq))
    W = coarse_dofs(md)
    cidx = -np.ones(md.ndofs, dtype=np.int64)
    cidx[W] = np.arange(len(W))
    ce = cidx[md.cell_dofs[:, loc]]
    rows = np.repeat(ce, nloc, axis=1).ravel()
    cols = np.tile(ce, (1, nloc)).ravel()
    return scipy.sparse.coo_matrix((Ae.ravel(), (rows, cols)), shape=(len(W), len(W))).tocsr()


def dirichlet_dofs(md, vertex_mask=None):
    """DOFs fixed by a homogeneous Dirichlet condition (X_{p,D} of Eq. (2.8)): every DOF of a vertex, edge
    or face of a face of Gamma_D.  Gamma_D is the whole boundary (the faces of exactly one cell), or, with
    vertex_mask (one flag per mesh vertex), the boundary faces whose three vertices are all flagged: a part
    of the boundary together with its closure."""
    _, cnt = np.unique(md.cell_faces.ravel(), return_counts=True)
    bfaces = np.nonzero(cnt == 1)[0]
    if vertex_mask is not None:
        vm = np.asarray(vertex_mask).astype(bool)
        bfaces = bfaces[np.all(vm[md.faces[bfaces]], axis=1)]
    nv_d, ne_d, nf_d, _ = md.per_entity
    off_v, off_e, off_f = md._offsets
    tri = md.faces[bfaces]
    bverts = np.unique(tri.ravel())
    pairs = np.unique(np.concatenate([tri[:, [0, 1]], tri[:, [0, 2]], tri[:, [1, 2]]]), axis=0)
    eidx = {tuple(e): i for i, e in enumerate(md.edges.tolist())}
    bedges = np.array([eidx[tuple(e)] for e in pairs.tolist()], dtype=np.int64)
    d = [off_v + nv_d * v + m for v in bverts for m in range(nv_d)]
    d += [off_e + ne_d * e + m for e in bedges for m in range(ne_d)]
    d += [off_f + nf_d * f + m for f in bfaces for m in range(nf_d)]
    return np.array(sorted(d), dtype=np.int64)


def constrained(A, D):
    """[A_ff 0; 0 I]: the Dirichlet DOFs D decoupled, with unit diagonal."""
    A = A.tocsr()
    keep = np.ones(A.shape[0])
    keep[D] = 0.0
    K = scipy.sparse.diags(keep)
    I_D = scipy.sparse.diags(1.0 - keep)
    return (K @ A @ K + I_D).tocsr()


class DirichletPreconditioner:
    """The one- or two-level preconditioner of the free DOFs (patches and W^k without the fixed DOFs)
    with the identity on the fixed DOFs."""

    def __init__(self, A, md, D, two_level=True, weight=0.5, patches=None):
        self.D = np.asarray(D)
        fixed = np.zeros(md.ndofs, dtype=bool)
        fixed[self.D] = True
        patches = [p[~fixed[p]] for p in (md.patches() if patches is None else patches)]
        Ac = constrained(A, self.D)
        if two_level:
            self.P = TwoLevelPreconditioner(Ac, md, patches, weight, W=coarse_dofs(md)[~fixed[coarse_dofs(md)]])
        else:
            self.P = Preconditioner(Ac, md, patches)

    def apply(self, r):
        z = self.P.apply(r)
        z[self.D] = r[self.D]
        return z


def gradient_matrix(md_ned, md_cg):
    """Ned1_p coefficients of the gradients of the CG_p basis functions on the same mesh: signed
    vertex-edge incidence on the Whitney DOFs and the identity from CG type-I edge/face DOFs onto
    Ned1_p type-II edge/face DOFs (Eq. (5.3), Lemma 4.3: type II = d of type I).  Interface part only."""
    rows, cols, vals = [], [], []
    ne_d, nf_d = md_ned.per_entity[1], md_ned.per_entity[2]
    ce, cf = md_cg.per_entity[1], md_cg.per_entity[2]
    off_e, off_f = md_ned._offsets[1], md_ned._offsets[2]
    coff_e, coff_f = md_cg._offsets[1], md_cg._offsets[2]
    for e, (a, b) in enumerate(md_ned.edges):
        rows += [off_e + ne_d * e] * 2
        cols += [int(a), int(b)]
        vals += [-1.0, 1.0]
        for m in range(ce):
            rows.append(off_e + ne_d * e + 1 + m)
            cols.append(coff_e + ce * e + m)
            vals.append(1.0)
    nfI = nf_d - cf
    for f in range(len(md_ned.faces)):
        for m in range(cf):
            rows.append(off_f + nf_d * f + nfI + m)
            cols.append(coff_f + cf * f + m)
            vals.append(1.0)
    return scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(md_ned.ndofs, md_cg.ndofs))


def edge_star_type1_dofs(md_ned, md_cg):
    """Per edge L: the Whitney DOF of L and the type-I DOFs of every face containing L (interface
    DOFs of X^{1,I} on the star of L), sorted."""
    ne_d, nf_d = md_ned.per_entity[1], md_ned.per_entity[2]
    nfI = nf_d - md_cg.per_entity[2]
    off_e, off_f = md_ned._offsets[1], md_ned._offsets[2]
    faces_of = {}
    for f, tri in enumerate(md_ned.faces.tolist()):
        for a, b in ((tri[0], tri[1]), (tri[0], tri[2]), (tri[1], tri[2])):
            faces_of.setdefault((a, b), []).append(f)
    out = []
    for e, (a, b) in enumerate(md_ned.edges.tolist()):
        d = [off_e + ne_d * e]
        for f in faces_of.get((a, b), []):
            d += [off_f + nf_d * f + m for m in range(nfI)]
        out.append(np.array(sorted(d), dtype=np.int64))
    return out


def edge_star_dofs(md, exclude=None):
    """Per edge E: the interface DOFs of E and of every face containing E, i.e. the interface functions
    supported in the star of E (the edge-star subspaces X^k_Gamma|_{star E} of the PAFW_1 decomposition,
    Eq. (6.24) for H(div), where only the face DOFs are present), sorted.  DOFs in `exclude` (fixed
    Dirichlet DOFs) are left out."""
    ne_d, nf_d = md.per_entity[1], md.per_entity[2]
    off_e, off_f = md._offsets[1], md._offsets[2]
    drop = set() if exclude is None else set(int(d) for d in exclude)
    faces_of = {}
    for f, tri in enumerate(md.faces.tolist()):
        for a, b in ((tri[0], tri[1]), (tri[0], tri[2]), (tri[1], tri[2])):
            faces_of.setdefault((a, b), []).append(f)
    out = []
    for e, (a, b) in enumerate(md.edges.tolist()):
        d = [off_e + ne_d * e + m for m in range(ne_d)]
        for f in faces_of.get((a, b), []):
            d += [off_f + nf_d * f + m for m in range(nf_d)]
        out.append(np.array(sorted(x for x in d if x not in drop), dtype=np.int64))
    return out


class HTPreconditioner:
    """The Hiptmair-Toselli splitting of Eq. (6.19) for H(curl) with the interface/interior split:
    P^{-1} = D_II^{-1} + sum_L R_L^T A_L^{-1} R_L (edge stars of type-I interface DOFs)
           + G sum_J R_J^T (G^T A G)_J^{-1} R_J G^T (gradients of CG_p interface functions on vertex
             stars, the potential problems of Eq. (6.18)) + w R_0^T A_0^{-1} R_0 (W^1).
    Additive; the coarse weight w = 1/2 as for the vertex-star preconditioner."""

    def __init__(self, A, md_ned, md_cg, weight=0.5):
        self.N = A.shape[0]
        A = A.tocsr()
        self.nI = md_ned.n_interface
        self.dinv_I = 1.0 / A.diagonal()[self.nI:]
        self.G = gradient_matrix(md_ned, md_cg).tocsc()
        K = (self.G.T @ A @ self.G).tocsr()
        self.pot = [(idx, scipy.linalg.cho_factor(K[idx][:, idx].toarray(), lower=True))
                    for idx in md_cg.patches() if len(idx)]
        self.est = [(idx, scipy.linalg.cho_factor(A[idx][:, idx].toarray(), lower=True))
                    for idx in edge_star_type1_dofs(md_ned, md_cg)]
        self.W = coarse_dofs(md_ned)
        self.weight = weight
        self.fac0 = scipy.linalg.cho_factor(A[self.W][:, self.W].toarray(), lower=True)

    def apply(self, r):
        z = np.zeros_like(r)
        z[self.nI:] = self.dinv_I * r[self.nI:]
        for idx, f in self.est:
            z[idx] += scipy.linalg.cho_solve(f, r[idx])
        rc = self.G.T @ r
        zc = np.zeros_like(rc)
        for idx, f in self.pot:
            zc[idx] += scipy.linalg.cho_solve(f, rc[idx])
        z += self.G @ zc
        z[self.W] += self.weight * scipy.linalg.cho_solve(self.fac0, r[self.W])
        return z

    def dense(self):
        I = np.eye(self.N)
        return np.stack([self.apply(I[:, j]) for j in range(self.N)], 1)


class TwoLevelPreconditioner:
    """P^{-1} = D_II^{-1} (+) sum_V R_V^T A_V^{-1} R_V + w R_0^T A_0^{-1} R_0: the one-level operator
    plus an exact solve on W^k (the PAFW decomposition's coarse summand, Section 6.2), with
    A_0 = R_0 A R_0^T the restriction of A to the lowest-order DOFs.  Additive, with the coarse
    correction weighted by w = 1/2 (the paper combines the summands multiplicatively with weights
    from eigenvalue estimates; every W^k function also lies in the vertex-star spaces, so the plain
    sum over-corrects, most for H(div))."""

    def __init__(self, A, md, patches=None, weight=0.5, W=None):
        self.weight = weight
        self.one = Preconditioner(A, md, patches)
        self.N = self.one.N
        self.W = coarse_dofs(md) if W is None else np.asarray(W)
        A = A.tocsr()
        self.A0 = A[self.W][:, self.W].toarray()
        self.fac0 = scipy.linalg.cho_factor(self.A0, lower=True)

    def coarse(self, r):
        """R_0^T A_0^{-1} R_0 r"""
        z = np.zeros_like(r)
        z[self.W] = scipy.linalg.cho_solve(self.fac0, r[self.W])
        return z

    def apply(self, r):
        return self.one.apply(r) + self.weight * self.coarse(r)

    def dense(self):
        I = np.eye(self.N)
        return np.stack([self.apply(I[:, j]) for j in range(self.N)], 1)


def lanczos_extremes(A_apply, Binv_apply, n, iters=10, seed=0):
    """Estimates of the extreme eigenvalues of B^{-1} A (A and B SPD on R^n) from `iters` steps of
    preconditioned CG with a random right-hand side: the eigenvalues of the Lanczos tridiagonal
    assembled from the CG step lengths alpha_j and ratios beta_j (diagonal 1/alpha_j +
    beta_{j-1}/alpha_{j-1}, off-diagonal sqrt(beta_j)/alpha_j)."""
    rng = np.random.default_rng(seed)
    r = rng.standard_normal(n)
    z = Binv_apply(r)
    p = z.copy()
    rz = r @ z
    al, be = [], []
    for _ in range(min(iters, n)):
        Ap = A_apply(p)
        a = rz / (p @ Ap)
        r = r - a * Ap
        z = Binv_apply(r)
        rz_new = r @ z
        al.append(a)
        be.append(rz_new / rz)
        if rz_new <= 0.0 or not np.isfinite(rz_new):
            break
        p = z + be[-1] * p
        rz = rz_new
    m = len(al)
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / al[j] + (be[j - 1] / al[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(be[j]) / al[j]
    ev = np.linalg.eigvalsh(T)
    return ev[0], ev[-1]


class HybridPreconditioner:
    """The paper's symmetric hybrid Schwarz preconditioner (Section 7.1, Eq. (7.2)): the spaces
    X_1 = interior DOFs (point-Jacobi), X_2 = interface DOFs (additive patches with exact solvers),
    X_3 = W^k (exact solve here; the paper uses a geometric-multigrid V-cycle), each inexact solver
    weighted by rho_m = (lambda_min + 3 lambda_max) / 4 from 10 Lanczos/CG steps of
    a(u, v) = lambda a~_m(u, v) on X_m (Eq. (7.3)), and combined multiplicatively in the sweep
    X_1, X_2, X_3, X_2, X_1 (X_1, X_2, X_1 without the coarse space)."""

    def __init__(self, A, md, patches=None, coarse=True, iters=10, seed=0, interface=None):
        """interface: an additive preconditioner whose restriction to the interface DOFs is the X_2
        solver (default: exact solves on `patches`, vertex stars if None); e.g. an HTPreconditioner
        with weight 0 for the Hiptmair-Toselli splitting.  The X_2 correction is that solver's
        output on the interface DOFs for a residual restricted to the interface DOFs (interior
        entries zeroed on input, dropped on output): for Hiptmair-Toselli this is the interface
        restriction of the HT operator, so the interior Ned1 components of its gradient corrections
        G (potential solves) are not part of X_2; the interior DOFs belong to X_1 alone."""
        A = A.tocsr()
        self.A = A
        self.N = A.shape[0]
        nI = md.n_interface
        self.I = np.arange(nI, self.N)
        self.G = np.arange(nI)
        self.one = Preconditioner(A, md, patches) if interface is None else interface
        AII, AGG = A[self.I][:, self.I], A[self.G][:, self.G]
        self.dinv = 1.0 / AII.diagonal() if len(self.I) else np.zeros(0)

        def patch_apply(rg):
            r = np.zeros(self.N)
            r[self.G] = rg
            return self.one.apply(r)[self.G]

        self.rho = {}
        if len(self.I):
            lo, hi = lanczos_extremes(lambda x: AII @ x, lambda x: self.dinv * x, len(self.I), iters, seed)
            self.rho[1] = (lo + 3.0 * hi) / 4.0
        lo, hi = lanczos_extremes(lambda x: AGG @ x, patch_apply, nI, iters, seed + 1)
        self.rho[2] = (lo + 3.0 * hi) / 4.0
        self.patch_apply = patch_apply
        self.sweep = [1, 2, 3, 2, 1] if coarse else [1, 2, 1]
        if not len(self.I):
            self.sweep = [m for m in self.sweep if m != 1]
        if coarse:
            self.W = coarse_dofs(md)
            A0 = A[self.W][:, self.W].toarray()
            self.fac0 = scipy.linalg.cho_factor(A0, lower=True)
            lo, hi = lanczos_extremes(lambda x: A0 @ x, lambda x: scipy.linalg.cho_solve(self.fac0, x),
                                      len(self.W), iters, seed + 2)
            self.rho[3] = (lo + 3.0 * hi) / 4.0

    def correction(self, m, res):
        z = np.zeros(self.N)
        if m == 1:
            z[self.I] = self.dinv * res[self.I] / self.rho[1]
        elif m == 2:
            z[self.G] = self.patch_apply(res[self.G]) / self.rho[2]
        else:
            z[self.W] = scipy.linalg.cho_solve(self.fac0, res[self.W]) / self.rho[3]
        return z

    def apply(self, r):
        z = np.zeros_like(r)
        for m in self.sweep:
            z = z + self.correction(m, r - self.A @ z)
        return z

    def dense(self):
        I = np.eye(self.N)
        return np.stack([self.apply(I[:, j]) for j in range(self.N)], 1)


def pcg(A, b, M=None, rtol=1e-8, maxit=1000):
    """PCG from x0 = 0; stops on the true relative residual.  Returns (x, iters, relres)."""
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0:
        return x, 0, 0.0
    r = b.copy()
    z = M(r) if M is not None else r.copy()
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        Ap = A @ p
        a = rz / (p @ Ap)
        x += a * p
        r -= a * Ap
        it += 1
        if np.linalg.norm(r) <= rtol * nb:
            rt = b - A @ x
            if np.linalg.norm(rt) <= rtol * nb:
                break
            r = rt
        z = M(r) if M is not None else r.copy()
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, np.linalg.norm(b - A @ x) / nb


def direct_solve(A, b):
    """Sparse direct solve (SuperLU)."""
    return scipy.sparse.linalg.splu(A.tocsc()).solve(b)


def mixed_matrix(ref_test, md_test, ref_trial, md_trial):
    """B[i, j] = (d phi^trial_j, phi^test_i) on a mesh shared by both spaces.

    Used to check that d maps one space of the complex into the next (Eq. (5.3)).
    """
    X, w = quadrature(3, max(ref_test.p, ref_trial.p) + 2)
    vt, dt = ref_test.tabulate(X)
    vr, dr = ref_trial.tabulate(X)
    J, _ = jacobians(md_test.verts, md_test.cells)
    v_te, _, det = physical_tabulation(ref_test, J, vt, dt)
    _, d_tr, _ = physical_tabulation(ref_trial, J, vr, dr)
    Be = np.einsum("epia,epja,p,e->eij", v_te, d_tr, w, np.abs(det))
    nc, n, m = Be.shape
    rows = np.repeat(md_test.cell_dofs, m, axis=1).ravel()
    cols = np.tile(md_trial.cell_dofs, (1, n)).ravel()
    B = scipy.sparse.coo_matrix((Be.ravel(), (rows, cols)), shape=(md_test.ndofs, md_trial.ndofs))
    return B.tocsr()


def mass_and_stiffness(ref, md):
    """Global mass and d-stiffness matrices separately (beta, alpha parts of Eq. (2.8))."""
    M = assemble(md, element_matrices(ref, md.verts, md.cells, alpha=0.0, beta=1.0))
    K = assemble(md, element_matrices(ref, md.verts, md.cells, alpha=1.0, beta=0.0))
    return M, K


def cells_of_dofs(md, dofs):
    """For each DOF: the (cell, local index) pairs that touch it."""
    out = []
    for d in dofs:
        c, j = np.nonzero(md.cell_dofs == d)
        out.append(list(zip(c.tolist(), j.tolist())))
    return out


def sampled_apply(ref, md, dofs, x):
    """(A x)[dofs] from the element matrices of the cells touching each DOF only."""
    touch = cells_of_dofs(md, dofs)
    cells = sorted({c for t in touch for c, _ in t})
    Ae = element_matrices(ref, md.verts, md.cells[cells])
    k = {c: i for i, c in enumerate(cells)}
    y = np.zeros(len(dofs))
    for m, t in enumerate(touch):
        for c, j in t:
            y[m] += Ae[k[c]][j] @ x[md.cell_dofs[c]]
    return y


def patch_matrix(ref, md, v):
    """A_V for vertex v assembled from the element matrices of its star cells."""
    idx = md.patches_of([v])[0]
    pos = {g: i for i, g in enumerate(idx)}
    _, _, cells = md.vertex_star(v)
    Ae = element_matrices(ref, md.verts, md.cells[cells])
    AV = np.zeros((len(idx), len(idx)))
    for a, c in enumerate(cells):
        loc = [j for j in range(ref.ndofs) if md.cell_dofs[c, j] in pos]
        gl = [pos[md.cell_dofs[c, j]] for j in loc]
        AV[np.ix_(gl, gl)] += Ae[a][np.ix_(loc, loc)]
    return idx, AV


def sampled_precond(ref, md, dofs, r):
    """(P^{-1} r)[dofs] for the preconditioner of Eq. (6.11), patch by patch."""
    z = np.zeros(len(dofs))
    cache = {}
    for m, d in enumerate(dofs):
        if d >= md.n_interface:
            (c, j), = cells_of_dofs(md, [d])[0]
            Ae = element_matrices(ref, md.verts, md.cells[[c]])[0]
            z[m] = r[d] / Ae[j, j]
            continue
        for v in md.vertices_of_dof(d):
            if v not in cache:
                idx, AV = patch_matrix(ref, md, v)
                cache[v] = (idx, scipy.linalg.cho_solve(scipy.linalg.cho_factor(AV, lower=True), r[idx]))
            idx, zv = cache[v]
            z[m] += zv[np.searchsorted(idx, d)]
    return z
