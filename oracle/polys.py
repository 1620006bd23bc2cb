"""Reference simplices, quadrature and an orthonormal polynomial expansion.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper works on an equilateral reference simplex (Section 3.3, the
paragraph after Eq. (3.9)); its size and placement are not stated.  Reading
used here: edge length 2, centroid at the origin, vertices listed below.  The
reference interval is [-1, 1] (length 2) and the reference triangle is the
equilateral triangle with the same edge length, vertices counter-clockwise.
With every reference simplex of edge length 2 the affine map that sends the
ordered vertices of the reference triangle (interval) onto the ordered
vertices of a face (edge) of the reference tetrahedron is an isometry.

The expansion is plain Gram--Schmidt on monomials taken in graded order, each
new candidate being x_i times an earlier basis function (the "Arnoldi" form
of Gram--Schmidt, done twice for stability).  It is orthonormal in L2 of the
simplex up to rounding and spans P_n exactly.
"""
import numpy as np

S3 = np.sqrt(3.0)
S6 = np.sqrt(6.0)

#: vertices of the reference interval, triangle and tetrahedron (edge length 2)
REF_VERTS = {
    1: np.array([[-1.0], [1.0]]),
    2: np.array([[-1.0, -1.0 / S3], [1.0, -1.0 / S3], [0.0, 2.0 / S3]]),
    3: np.array([[-1.0, -1.0 / S3, -1.0 / S6], [1.0, -1.0 / S3, -1.0 / S6],
                 [0.0, 2.0 / S3, -1.0 / S6], [0.0, 0.0, 3.0 / S6]]),
}


def simplex_volume(verts):
    """Lebesgue measure of the simplex with the given (d+1, d) vertices."""
    d = verts.shape[1]
    E = (verts[1:] - verts[0]).T
    return abs(np.linalg.det(E)) / np.prod(np.arange(1, d + 1))


def quadrature(dim, npts):
    """Collapsed (Duffy) tensor Gauss--Legendre rule on the reference simplex.

    ``npts`` points per direction; exact for polynomials of degree
    ``2*npts - 1 - (dim - 1)`` on the simplex.
    Returns points (n, dim) and weights (n,).
    """
    g, gw = np.polynomial.legendre.leggauss(npts)
    g = 0.5 * (g + 1.0)
    gw = 0.5 * gw
    V = REF_VERTS[dim]
    if dim == 1:
        lam = np.stack([1.0 - g, g], 1)
        w = gw.copy()
    elif dim == 2:
        a, b = np.meshgrid(g, g, indexing="ij")
        wa, wb = np.meshgrid(gw, gw, indexing="ij")
        u = a
        v = b * (1.0 - a)
        w = (wa * wb * (1.0 - a)).ravel()
        lam = np.stack([1.0 - u - v, u, v], -1).reshape(-1, 3)
    else:
        a, b, c = np.meshgrid(g, g, g, indexing="ij")
        wa, wb, wc = np.meshgrid(gw, gw, gw, indexing="ij")
        u = a
        v = b * (1.0 - a)
        t = c * (1.0 - a) * (1.0 - b)
        w = (wa * wb * wc * (1.0 - a) ** 2 * (1.0 - b)).ravel()
        lam = np.stack([1.0 - u - v - t, u, v, t], -1).reshape(-1, 4)
    X = lam @ V
    # the unit simplex has volume 1/d!; rescale to the reference simplex
    unit = 1.0 / np.prod(np.arange(1, dim + 1))
    w = w * simplex_volume(V) / unit
    return X, w


def graded_exponents(dim, deg):
    """Monomial exponents of total degree <= deg, graded, lexicographic inside."""
    out = []
    for d in range(deg + 1):
        if dim == 1:
            out.append((d,))
        elif dim == 2:
            for a in range(d, -1, -1):
                out.append((a, d - a))
        else:
            for a in range(d, -1, -1):
                for b in range(d - a, -1, -1):
                    out.append((a, b, d - a - b))
    return out


def dim_P(dim, deg):
    """dim P_deg in ``dim`` variables (0 for negative degree)."""
    if deg < 0:
        return 0
    from math import comb
    return comb(deg + dim, dim)


class OrthoBasis:
    """L2-orthonormal basis of P_deg on the reference simplex of dimension dim.

    Built by two passes of classical Gram--Schmidt on candidates x_i * q_parent
    in the discrete inner product of a rule exact to degree 2*deg.  The
    recurrence is stored so the basis and its gradient can be evaluated at any
    point.
    """

    def __init__(self, dim, deg):
        self.dim = dim
        self.deg = deg
        self.exps = graded_exponents(dim, deg)
        self.n = len(self.exps)
        X, w = quadrature(dim, deg + 2)
        index = {e: k for k, e in enumerate(self.exps)}
        Q = np.zeros((X.shape[0], self.n))
        self.rec = []  # (axis, parent, coefficients on previous, norm)
        Q[:, 0] = 1.0
        nrm = np.sqrt(np.sum(w * Q[:, 0] ** 2))
        Q[:, 0] /= nrm
        self.rec.append((None, None, np.zeros(0), nrm))
        for k in range(1, self.n):
            e = self.exps[k]
            axis = max(i for i in range(dim) if e[i] > 0)
            pe = list(e)
            pe[axis] -= 1
            parent = index[tuple(pe)]
            c = X[:, axis] * Q[:, parent]
            h = np.zeros(k)
            for _ in range(2):
                hk = Q[:, :k].T @ (w * c)
                c = c - Q[:, :k] @ hk
                h += hk
            nrm = np.sqrt(np.sum(w * c * c))
            Q[:, k] = c / nrm
            self.rec.append((axis, parent, h, nrm))

    def eval(self, Y):
        """Values (n_pts, n) and gradients (n_pts, n, dim) at points Y (n_pts, dim)."""
        Y = np.atleast_2d(Y)
        npt = Y.shape[0]
        V = np.zeros((npt, self.n))
        G = np.zeros((npt, self.n, self.dim))
        V[:, 0] = 1.0 / self.rec[0][3]
        for k in range(1, self.n):
            axis, parent, h, nrm = self.rec[k]
            v = Y[:, axis] * V[:, parent] - V[:, :k] @ h
            g = Y[:, axis, None] * G[:, parent, :] - np.einsum("pjd,j->pd", G[:, :k, :], h)
            g[:, axis] += V[:, parent]
            V[:, k] = v / nrm
            G[:, k, :] = g / nrm
        return V, G
