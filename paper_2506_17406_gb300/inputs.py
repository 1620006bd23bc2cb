"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the oracle.

This module holds none of the solver's arithmetic: it only generates the
problem data the paper's experiments use (Section 7.1) -- Freudenthal (Kuhn)
meshes of the unit cube, optionally with interior vertices perturbed, and
seeded random coefficient vectors.

Mesh recipe: the unit cube split into n^3 sub-cubes, each cut into the 6
tetrahedra that share its main diagonal (the Freudenthal subdivision shown in
the paper's Fig. 3a).  Vertex (i, j, k) has index i + (n+1)(j + (n+1)k) and
position h(i, j, k), h = 1/n.  Each tetrahedron is the path corner,
corner + h e_a, corner + h e_a + h e_b, corner + h(1,1,1) for one of the 6
orderings (a, b, c) of the axes; its vertex indices increase along the path.
Perturbation: every coordinate of every vertex not on the boundary of the
cube moves by an independent uniform draw in [-amp*h, amp*h].

Fichera corner (Section 7.2): the same Kuhn cubes of (0,1)^3 without the
cubes inside (1/2,1)^3 (n even), unused vertices dropped and the others
renumbered in increasing order, so that vertex indices still increase along
every path; a vertex is interior when all eight cubes around it are kept.
The paper's graded unstructured Fichera mesh is not reproduced: this uniform
Kuhn mesh stands in for it.
"""
import itertools

import numpy as np


def kuhn_mesh(n, perturb=0.0, seed=0):
    """Return (verts float64 (nv, 3), cells int64 (6 n^3, 4))."""
    h = 1.0 / n
    g = np.arange(n + 1, dtype=np.float64) * h
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    if perturb:
        rng = np.random.Generator(np.random.PCG64(seed))
        d = rng.uniform(-perturb * h, perturb * h, size=verts.shape)
        ijk = np.stack(np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1),
                                   indexing="ij")[::-1], -1).reshape(-1, 3)
        interior = np.all((ijk > 0) & (ijk < n), axis=1)
        verts[interior] += d[interior]
    stride = np.array([1, n + 1, (n + 1) ** 2], dtype=np.int64)
    cells = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                c0 = i + (n + 1) * (j + (n + 1) * k)
                for perm in itertools.permutations(range(3)):
                    v = [c0]
                    for a in perm:
                        v.append(v[-1] + stride[a])
                    cells.append(v)
    return verts, np.array(cells, dtype=np.int64)


def fichera_mesh(n, perturb=0.0, seed=0):
    """Return (verts, cells) of the Kuhn mesh of (0,1)^3 minus (1/2,1)^3 with n (even) cubes per edge."""
    if n % 2:
        raise ValueError("n must be even")
    verts, cells = kuhn_mesh(n)
    m = n // 2
    keep_cube = np.ones((n, n, n), dtype=bool)  # [k][j][i]
    keep_cube[m:, m:, m:] = False
    cube = np.repeat(np.arange(n ** 3), 6)
    ci, cj, ck = cube % n, (cube // n) % n, cube // (n * n)
    cells = cells[keep_cube[ck, cj, ci]]
    used = np.zeros(len(verts), dtype=bool)
    used[cells.ravel()] = True
    new = np.cumsum(used) - 1
    ijk = np.stack([np.arange(len(verts)) % (n + 1), (np.arange(len(verts)) // (n + 1)) % (n + 1),
                    np.arange(len(verts)) // (n + 1) ** 2], 1)
    interior = np.ones(len(verts), dtype=bool)
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                a, b, c = ijk[:, 0] - di, ijk[:, 1] - dj, ijk[:, 2] - dk
                inside = (a >= 0) & (a < n) & (b >= 0) & (b < n) & (c >= 0) & (c < n)
                ok = np.zeros(len(verts), dtype=bool)
                ok[inside] = keep_cube[c[inside], b[inside], a[inside]]
                interior &= ok
    verts = verts[used].copy()
    interior = interior[used]
    if perturb:
        h = 1.0 / n
        rng = np.random.Generator(np.random.PCG64(seed))
        d = rng.uniform(-perturb * h, perturb * h, size=verts.shape)
        verts[interior] += d[interior]
    return verts, new[cells].astype(np.int64)


def normal_vector(size, seed):
    """Seeded N(0, 1) float64 vector (the paper's random right-hand side)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(size)


def normal_coeffs(shape, seed):
    """Seeded N(0, 1) float64 array of the given shape."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape)
