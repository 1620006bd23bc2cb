"""Hodge-Laplacians of the de Rham complex in mixed form (Section 7.2, Eq. (7.5)) -- CPU oracle.

Test infrastructure only: the library never imports this module.

For k in {1, 2, 3} find (sigma, u) in X^{k-1} x X^k with
    -(sigma, tau) + (u, d tau)         = 0       for all tau in X^{k-1}
     (d sigma, v) + (d u, d v)         = (f, v)  for all v in X^k,
i.e. the symmetric indefinite block system
    [ -M_{k-1}   B^T ] [sigma]   [0]
    [  B         K_k ] [u    ] = [b],   B_ij = (d phi^{k-1}_j, phi^k_i),
preconditioned by the block-diagonal weighted Riesz maps of Eq. (7.6) (the augmented-Lagrangian
preconditioner): P = diag(M_{k-1} + gamma K_{k-1}, gamma^{-1} M_k + K_k), either solved exactly
or replaced by the paper's Schwarz preconditioners for each block (Section 7.2: PAFW_0 vertex stars
for CG_p, Hiptmair-Toselli for Ned1_p, PAFW_1 edge stars for RT_p, each with W^k).  MINRES (Paige
and Saunders, 1975) is written out below from the Lanczos recurrence and Givens rotations.

k = 3 is the mixed Poisson problem in RT_p x DG_{p-1} (d^3 = 0, so K_3 = 0); the DG block of the
preconditioner is its diagonal mass matrix, inverted exactly (point-Jacobi, Section 7.2).
"""
import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from . import assemble as asm
from .mesh import MeshDofs
from .refelem import reference_element

SPACES = {1: ("CG", "N1curl"), 2: ("N1curl", "RT"), 3: ("RT", "DG")}


class HodgeSystem:
    """Blocks of the Hodge-Laplace problem of Section 7.2 for k in {1, 2, 3} on one mesh."""

    def __init__(self, k, p, verts, cells, gamma=1.0):
        self.k, self.p, self.gamma = k, p, gamma
        s0, s1 = SPACES[k]
        self.ref0, self.ref1 = reference_element(s0, p), reference_element(s1, p)
        self.md0 = MeshDofs(verts, cells, self.ref0)
        self.md1 = MeshDofs(verts, cells, self.ref1)
        self.M0, self.K0 = asm.mass_and_stiffness(self.ref0, self.md0)
        self.M1, self.K1 = asm.mass_and_stiffness(self.ref1, self.md1)
        self.B = asm.mixed_matrix(self.ref1, self.md1, self.ref0, self.md0)  # (d sigma_j, v_i)
        self.n0, self.n1 = self.md0.ndofs, self.md1.ndofs
        self.A = scipy.sparse.bmat([[-self.M0, self.B.T], [self.B, self.K1]]).tocsr()
        # the weighted Riesz maps of Eq. (7.6)
        self.P0 = (self.M0 + gamma * self.K0).tocsr()
        self.P1 = ((1.0 / gamma) * self.M1 + self.K1).tocsr()

    def rhs(self, f1):
        """Block right-hand side [0; b] for a load vector b = (f, v) on X^k."""
        return np.concatenate([np.zeros(self.n0), f1])

    def exact_preconditioner(self):
        """z = P^{-1} r with both weighted Riesz maps solved by sparse LU."""
        l0 = scipy.sparse.linalg.splu(self.P0.tocsc())
        l1 = scipy.sparse.linalg.splu(self.P1.tocsc())

        def apply(r):
            return np.concatenate([l0.solve(r[:self.n0]), l1.solve(r[self.n0:])])

        return apply

    def schwarz_blocks(self, recommended=True, coarse=True, form="additive"):
        """The two Schwarz preconditioners (the paper's per-space decompositions when recommended,
        else vertex stars for both), each with interior Jacobi and, when coarse, the weighted W^k
        summand (one-level otherwise).  form = "hybrid": the paper's symmetric hybrid sweep with
        Lanczos-estimated weights (Eqs. (7.2)-(7.3)) in each Riesz block instead."""
        out = []
        for sp, P, md in ((SPACES[self.k][0], self.P0, self.md0), (SPACES[self.k][1], self.P1, self.md1)):
            if sp == "DG":  # diagonal mass (orthogonal basis): Jacobi is the exact inverse
                out.append(asm.Preconditioner(P, md, patches=[]))
            elif form == "hybrid":
                iface = None
                patches = None
                if recommended and sp == "N1curl":
                    mc = self.md0 if self.k == 1 else MeshDofs(md.verts, md.cells, reference_element("CG", self.p))
                    iface = asm.HTPreconditioner(P, md, mc, weight=0.0)
                elif recommended and sp == "RT":
                    patches = asm.edge_star_dofs(md)
                out.append(asm.HybridPreconditioner(P, md, patches, coarse=coarse, interface=iface))
            elif recommended and sp == "N1curl":
                mc = self.md0 if self.k == 1 else MeshDofs(md.verts, md.cells, reference_element("CG", self.p))
                out.append(asm.HTPreconditioner(P, md, mc, weight=0.5 if coarse else 0.0))
            else:
                patches = asm.edge_star_dofs(md) if (recommended and sp == "RT") else None
                if coarse:
                    out.append(asm.TwoLevelPreconditioner(P, md, patches))
                else:
                    out.append(asm.Preconditioner(P, md, patches))
        return out

    def schwarz_preconditioner(self, recommended=True, coarse=True, form="additive"):
        b0, b1 = self.schwarz_blocks(recommended, coarse, form)

        def apply(r):
            return np.concatenate([b0.apply(r[:self.n0]), b1.apply(r[self.n0:])])

        return apply


def minres(A, b, Minv, rtol=1e-8, maxit=1000, x0=None):
    """Preconditioned MINRES for symmetric A and SPD M.

    Lanczos on M^{-1} A in the M-inner product (v: unpreconditioned Lanczos vectors, u = M^{-1} v),
    the tridiagonal T_k reduced by Givens rotations as it grows, and the iterate updated along the
    directions d_k = (u_k - delta_k d_{k-1} - eps_k d_{k-2}) / gamma_k.  |phibar| is the M^{-1}-norm of
    the residual b - A x_k; stop when it drops below rtol times its initial value.
    Returns (x, iterations, M^{-1}-norm residual ratio)."""
    n = len(b)
    x = np.zeros(n) if x0 is None else x0.copy()
    r = b - A @ x
    z = Minv(r)
    beta = np.sqrt(r @ z)
    beta1 = beta
    if beta1 == 0.0:
        return x, 0, 0.0
    v_prev = np.zeros(n)
    v = r / beta
    u = z / beta
    d_prev = np.zeros(n)
    d_prev2 = np.zeros(n)
    c_prev, s_prev = 1.0, 0.0   # rotation k-1
    c_prev2, s_prev2 = 1.0, 0.0  # rotation k-2
    phibar = beta1
    it = 0
    while it < maxit:
        it += 1
        # Lanczos step: column k of T has beta_k (above), alpha_k, beta_{k+1} (below)
        w = A @ u - beta * v_prev
        alpha = u @ w
        w = w - alpha * v
        zw = Minv(w)
        beta_next = np.sqrt(max(w @ zw, 0.0))
        # the two previous rotations applied to column k
        eps = s_prev2 * beta
        dlt = c_prev2 * beta
        delta = c_prev * dlt + s_prev * alpha
        gbar = -s_prev * dlt + c_prev * alpha
        # the new rotation eliminates beta_{k+1}
        gam = np.hypot(gbar, beta_next)
        c, s = gbar / gam, beta_next / gam
        tau = c * phibar
        phibar = -s * phibar
        d = (u - delta * d_prev - eps * d_prev2) / gam
        x = x + tau * d
        d_prev2, d_prev = d_prev, d
        c_prev2, s_prev2, c_prev, s_prev = c_prev, s_prev, c, s
        if abs(phibar) <= rtol * beta1 or beta_next == 0.0:
            break
        v_prev, v = v, w / beta_next
        u = zw / beta_next
        beta = beta_next
    return x, it, abs(phibar) / beta1


def predicted_spectrum(h):
    """Eigenvalues of P^{-1} A for the exact block preconditioner by Theorem C.1 on a contractible
    domain (no harmonic forms): -1 with multiplicity dim X^{k-1}; mu gamma / (mu gamma + 1) for the
    nonzero generalized eigenvalues mu of (K_k, M_k); nu gamma / (nu gamma + 1) for those nu of
    (K_{k-1}, M_{k-1})."""
    g = h.gamma
    mu = scipy.linalg.eigh(h.K1.toarray(), h.M1.toarray(), eigvals_only=True)
    nu = scipy.linalg.eigh(h.K0.toarray(), h.M0.toarray(), eigvals_only=True)
    tol = 1e-8 * max(mu.max(), nu.max())
    mu, nu = mu[mu > tol], nu[nu > tol]
    return np.sort(np.concatenate([-np.ones(h.n0), mu * g / (mu * g + 1.0), nu * g / (nu * g + 1.0)]))
