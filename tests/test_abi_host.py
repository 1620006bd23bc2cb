"""Host-side parity of libriesz.so (no GPU): exported symbols, reference basis
and mesh maps against the oracle, input validation."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.mesh import MeshDofs
from oracle.polys import quadrature
from oracle.refelem import reference_element
from paper_2506_17406_gb300 import riesz as rz
from paper_2506_17406_gb300.inputs import kuhn_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return rz.load_library(build_if_missing=True)


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "riesz.h")).read()
    names = sorted(set(re.findall(r"\b(riesz_[a-z_0-9]+)\s*\(", hdr)))
    assert len(names) >= 18
    cdll = ctypes.CDLL(rz.library_path())
    for n in names:
        assert hasattr(cdll, n), n


@pytest.mark.parametrize("space", ["CG", "N1curl", "RT"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_reference_basis_matches_oracle(lib, space, p):
    """The library's basis (Dubiner expansion, own eigen/null-space code) equals the
    oracle's (Gram-Schmidt expansion, LAPACK) at points of the reference cell, for every
    degree the configurations draw (1..10).

    Both sides solve the eigenproblems of Eq. (3.9) independently; inside an eigenvalue
    cluster the probe rule fixes the basis, but an eigenvector still moves by about
    eps / (relative gap to the nearest other cluster) under rounding.  Those gaps shrink
    with p (down to 2.6e-5 at p = 10 for Ned1 and RT), so the agreement is 1e-11 up to
    p = 5, a few 1e-11 up to p = 8 and at most 1.5e-9 at p = 9, 10 (measured); a wrong
    cluster, order or sign would differ by O(1)."""
    tol = 1e-11 if p <= 5 else (1e-10 if p <= 8 else 1e-8)
    X, _ = quadrature(3, 4)
    v, d = rz.riesz_ref_tabulate(space, p, X)
    vo, do = reference_element(space, p).tabulate(X)
    assert np.abs(v - vo).max() <= tol * np.abs(vo).max()
    assert np.abs(d - do).max() <= tol * np.abs(do).max()


@pytest.mark.parametrize("space,p", [(s, p) for s in ("N2curl", "BDM") for p in range(1, 9)] +
                         [("N2curl", 9), ("N2curl", 10)])
def test_second_kind_basis_matches_oracle(lib, space, p):
    """NedTwo_p and BDM_p (Eq. (2.6)) from the library equal the oracle's at points of the reference cell;
    same tolerance argument as for the first kind (measured: at most 2e-11 up to p = 8, 6e-10 at p = 9, 10).
    BDM_9 and BDM_10 (about a minute of host eigensolves on each side) are checked through the GPU apply
    against the oracle's assembled matrix (tests/test_gpu_second_kind.py)."""
    tol = 1e-10 if p <= 8 else 1e-8
    X, _ = quadrature(3, 4)
    v, d = rz.riesz_ref_tabulate(space, p, X)
    vo, do = reference_element(space, p).tabulate(X)
    assert v.shape == vo.shape == (X.shape[0], (p + 1) * (p + 2) * (p + 3) // 2, 3)
    assert np.abs(v - vo).max() <= tol * np.abs(vo).max()
    assert np.abs(d - do).max() <= tol * np.abs(do).max()


@pytest.mark.parametrize("space,p,n", [("CG", 3, 4), ("CG", 4, 2), ("N1curl", 3, 3), ("N1curl", 1, 2),
                                       ("RT", 2, 3), ("RT", 4, 2), ("N2curl", 2, 3), ("N2curl", 3, 2),
                                       ("BDM", 1, 3), ("BDM", 3, 2)])
def test_dof_and_patch_maps_bit_exact(lib, space, p, n):
    verts, cells = kuhn_mesh(n, 0.1, 5)
    # present the cells with scrambled vertex order: both sides must sort them
    rng = np.random.Generator(np.random.PCG64(1))
    scr = np.array([rng.permutation(c) for c in cells])
    s = rz.Riesz(space, p, verts, scr, device=False)
    md = MeshDofs(verts, scr, reference_element(space, p))
    assert s.N == md.ndofs and s.n_interior == md.n_interior
    assert np.array_equal(s.dof_map(), md.cell_dofs)
    off, dofs = s.patch_map()
    pts = md.patches()
    assert len(off) == len(pts) + 1
    for v, q in enumerate(pts):
        assert np.array_equal(dofs[off[v]:off[v + 1]], q)


def test_dof_counts_large_mesh(lib):
    """Ned1_6 on 8^3 x 6 tets (405 264 DOFs) and RT_8 on 16^3 x 6 (8 017 920)."""
    v, c = kuhn_mesh(8, 0.1, 1)
    s = rz.Riesz("N1curl", 6, v, c, device=False)
    assert s.N == 405264
    v, c = kuhn_mesh(16, 0.1, 1)
    s = rz.Riesz("RT", 8, v, c, device=False)
    assert s.N == 8017920


def test_input_validation(lib):
    v, c = kuhn_mesh(1)
    with pytest.raises(rz.RieszError) as e:
        rz.Riesz("CG", 0, v, c, device=False)
    assert e.value.code == 1
    with pytest.raises(rz.RieszError) as e:
        rz.Riesz(7, 2, v, c, device=False)
    assert e.value.code == 1
    bad = c.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(rz.RieszError) as e:
        rz.Riesz("CG", 2, v, bad, device=False)
    assert e.value.code == 2
    bad = c.copy()
    bad[0, 1] = len(v)
    with pytest.raises(rz.RieszError) as e:
        rz.Riesz("CG", 2, v, bad, device=False)
    assert e.value.code == 2
    flat = v.copy()
    flat[:, 2] = 0.0  # every cell degenerate
    with pytest.raises(rz.RieszError) as e:
        rz.Riesz("CG", 2, flat, c, device=False)
    assert e.value.code == 2
    nan = v.copy()
    nan[3, 0] = np.nan
    with pytest.raises(rz.RieszError) as e:
        rz.Riesz("CG", 2, nan, c, device=False)
    assert e.value.code == 2


def test_device_calls_fail_loudly_without_device_state(lib):
    v, c = kuhn_mesh(1)
    s = rz.Riesz("CG", 2, v, c, device=False)
    rc = lib.riesz_apply(s.h, ctypes.c_void_p(8), ctypes.c_void_p(8), 1, None)
    assert rc == 8  # RIESZ_ERR_NO_DEVICE, nothing launched


def test_option_validation(lib):
    v, c = kuhn_mesh(1)
    for kw in [dict(loop=2), dict(loop=-1), dict(autotune=3), dict(apply_precision=3), dict(alpha=0.0), dict(beta=-1.0),
               dict(nrhs_max=0), dict(rtol=0.0), dict(coarse=3), dict(form=2), dict(coarse_its=0),
               dict(coarse_its=1001)]:
        with pytest.raises(rz.RieszError) as e:
            rz.Riesz("CG", 2, v, c, device=False, **kw)
        assert e.value.code == 1, kw
    o = rz.default_opts()
    assert o.loop == rz.LOOP_GRAPH and o.apply_precision == rz.PREC_FP64
    assert o.form == rz.FORM_ADDITIVE and o.coarse_its == 4


def test_planned_bytes_count_the_options(lib):
    """riesz_plan_bytes (host-only) grows by the buffers each option adds: a second right-hand side adds
    its Krylov vectors, the hybrid form its three sweep vectors, the sparse coarse route its CSR."""
    v, c = kuhn_mesh(3, 0.1, 1)
    base, na = rz.Riesz("RT", 3, v, c, device=False).plan_bytes()
    assert base > 0 and na > 20
    N = rz.Riesz("RT", 3, v, c, device=False).N
    hyb, _ = rz.Riesz("RT", 3, v, c, device=False, form=rz.FORM_HYBRID).plan_bytes()
    assert hyb - base == 3 * 8 * N
    two, _ = rz.Riesz("RT", 3, v, c, device=False, nrhs_max=2).plan_bytes()
    assert two - base >= 8 * 8 * N
    sp, _ = rz.Riesz("RT", 3, v, c, device=False, coarse=2).plan_bytes()
    assert sp != base


def test_batch_without_device_state(lib):
    v, c = kuhn_mesh(1)
    s = rz.Riesz("CG", 2, v, c, device=False)
    hs = (ctypes.c_void_p * 1)(s.h.value)
    ptrs = (ctypes.c_void_p * 1)(8)
    rc = lib.riesz_solve_batch(ctypes.cast(hs, ctypes.c_void_p), 1, ctypes.cast(ptrs, ctypes.c_void_p),
                               ctypes.cast(ptrs, ctypes.c_void_p), None, None, None, None, None)
    assert rc in (6, 8)  # no CUDA device here (6) or no device state (8); nothing launched


@pytest.mark.parametrize("space,p", [("CG", 3), ("N1curl", 2), ("RT", 3)])
def test_dirichlet_map_bit_exact(lib, space, p):
    """The library's fixed DOFs equal the oracle's, and the patches leave them out."""
    from oracle import assemble as asm
    from oracle.mesh import MeshDofs
    from oracle.refelem import reference_element
    v, c = kuhn_mesh(3, 0.1, 2)
    s = rz.Riesz(space, p, v, c, device=False, dirichlet=1)
    md = MeshDofs(v, c, reference_element(space, p))
    D = asm.dirichlet_dofs(md)
    mask = s.dirichlet_map()
    assert np.array_equal(np.nonzero(mask)[0], D)
    off, dofs = s.patch_map()
    fixed = np.zeros(s.N, dtype=bool)
    fixed[D] = True
    for vv in range(len(off) - 1):
        exp = md.patches_of([vv])[0]
        assert np.array_equal(dofs[off[vv]:off[vv + 1]], exp[~fixed[exp]])
    s0 = rz.Riesz(space, p, v, c, device=False)
    assert s0.dirichlet_map().sum() == 0


def test_ht_validation(lib):
    v, c = kuhn_mesh(2)
    rz.Riesz("N1curl", 2, v, c, device=False, decomposition=rz.DECOMP_HT)
    for space, kw in [("RT", {}), ("CG", {}), ("N1curl", dict(dirichlet=1))]:
        with pytest.raises(rz.RieszError) as e:
            rz.Riesz(space, 2, v, c, device=False, decomposition=rz.DECOMP_HT, **kw)
        assert e.value.code == 1
    rz.Riesz("RT", 2, v, c, device=False, decomposition=rz.DECOMP_EDGE_STAR)
    rz.Riesz("RT", 2, v, c, device=False, decomposition=rz.DECOMP_EDGE_STAR, dirichlet=1)
    for space in ("CG", "N1curl"):
        with pytest.raises(rz.RieszError) as e:
            rz.Riesz(space, 2, v, c, device=False, decomposition=rz.DECOMP_EDGE_STAR)
        assert e.value.code == 1
    with pytest.raises(rz.RieszError):
        rz.Riesz("RT", 2, v, c, device=False, decomposition=3)


@pytest.mark.parametrize("dirichlet", [0, 1])
def test_edge_star_patches_match_oracle(lib, dirichlet):
    """The library's H(div) edge-star patches (Eq. (6.24)) are the oracle's edge-star DOF sets, bit-exact,
    with the fixed Dirichlet DOFs left out."""
    from oracle import assemble as asm
    from oracle.mesh import MeshDofs
    from oracle.refelem import reference_element
    v, c = kuhn_mesh(2, 0.1, 3)
    h = rz.Riesz("RT", 3, v, c, device=False, decomposition=rz.DECOMP_EDGE_STAR, dirichlet=dirichlet)
    off, dofs = h.patch_map()
    md = MeshDofs(v, c, reference_element("RT", 3))
    D = asm.dirichlet_dofs(md) if dirichlet else None
    exp = asm.edge_star_dofs(md, exclude=D)
    assert len(off) == len(md.edges) + 1 == len(exp) + 1
    for e, q in enumerate(exp):
        assert np.array_equal(dofs[off[e]:off[e + 1]], q)
    assert dirichlet == int(any(len(q) == 0 for q in exp))


def test_hodge_validation(lib):
    """Arguments are checked before any device work: k, gamma, Dirichlet; without a GPU the setup
    reports the missing device instead of falling back."""
    from paper_2506_17406_gb300.inputs import fichera_mesh
    v, c = fichera_mesh(2)
    for k, gamma, kw in [(0, 1.0, {}), (4, 1.0, {}), (1, 0.0, {}), (2, -1.0, {}), (3, 1.0, dict(dirichlet=1))]:
        with pytest.raises(rz.RieszError) as e:
            rz.Hodge(k, 2, v, c, gamma, stream=0, **kw)
        assert e.value.code == 1
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(rz.RieszError) as e:
            rz.Hodge(1, 2, v, c, 1.0, stream=0)
        assert e.value.code == 6


@pytest.mark.parametrize("k,p", [(1, 1), (1, 3), (2, 2), (2, 4)])
def test_hodge_coupling_tables_match_oracle(lib, k, p):
    """The library's reference coupling tables, contracted with one cell's metric, give the oracle's
    (d phi^{k-1}_j, phi^k_i) on that cell (oracle: quadrature of the pulled-back functions)."""
    from oracle import assemble as asm
    from oracle.mesh import MeshDofs
    from oracle.refelem import reference_element
    rng = np.random.default_rng(k * 10 + p)
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float) + 0.2 * rng.standard_normal((4, 3))
    cells = np.array([[0, 1, 2, 3]])
    sp = {1: ("CG", "N1curl"), 2: ("N1curl", "RT")}[k]
    r0, r1 = reference_element(sp[0], p), reference_element(sp[1], p)
    B = asm.mixed_matrix(r1, MeshDofs(verts, cells, r1), r0, MeshDofs(verts, cells, r0)).toarray()
    J, _ = asm.jacobians(verts, cells)
    J = J[0]
    d = abs(np.linalg.det(J))
    G = d * np.linalg.inv(J) @ np.linalg.inv(J).T if k == 1 else J.T @ J / d
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    R = rz.riesz_ref_mixed_tables(k, p)
    Bl = sum(G[a, b] * R[q] for q, (a, b) in enumerate(pairs))  # [j][i]
    assert np.abs(Bl.T - B).max() <= 1e-12 * np.abs(B).max()


@pytest.mark.parametrize("p", [2, 4])
def test_ht_edge_star_patches_match_oracle(lib, p):
    """The library's Hiptmair-Toselli edge stars (Eq. (6.19): the edge's Whitney DOF and the type-I DOFs of
    every face containing it) are the oracle's, bit-exact, edge by edge."""
    from oracle import assemble as asm
    from oracle.mesh import MeshDofs
    from oracle.refelem import reference_element
    v, c = kuhn_mesh(2, 0.1, 3)
    h = rz.Riesz("N1curl", p, v, c, device=False, decomposition=rz.DECOMP_HT)
    off, dofs = h.patch_map()
    mn = MeshDofs(v, c, reference_element("N1curl", p))
    mc = MeshDofs(v, c, reference_element("CG", p))
    exp = asm.edge_star_type1_dofs(mn, mc)
    assert len(off) == len(exp) + 1
    for e, q in enumerate(exp):
        assert np.array_equal(dofs[off[e]:off[e + 1]], q)


@pytest.mark.parametrize("p", [1, 3])
def test_ht_gradient_map_matches_oracle(lib, p):
    """The library's gradient map (Eq. (5.3): signed vertex-edge incidence on the Whitney DOFs, identity from CG
    edge/face DOFs onto the Ned1 type-II DOFs) equals the oracle's gradient_matrix on the interface, bit-exact."""
    from oracle import assemble as asm
    from oracle.mesh import MeshDofs
    from oracle.refelem import reference_element
    v, c = kuhn_mesh(2, 0.1, 3)
    h = rz.Riesz("N1curl", p, v, c, device=False, decomposition=rz.DECOMP_HT)
    mn = MeshDofs(v, c, reference_element("N1curl", p))
    mc = MeshDofs(v, c, reference_element("CG", p))
    ptr, idx, sgn = h.ht_gradient_map(mn.n_interface)
    G = asm.gradient_matrix(mn, mc).tocsr()[:mn.n_interface, :mc.n_interface].toarray()
    Gl = np.zeros_like(G)
    for d in range(mn.n_interface):
        for k in range(ptr[d], ptr[d + 1]):
            Gl[d, idx[k]] += sgn[k]
    assert np.array_equal(Gl, G)
    with pytest.raises(rz.RieszError):
        rz.Riesz("N1curl", p, v, c, device=False).ht_gradient_map(mn.n_interface)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_dg_reference_basis_matches_oracle(lib, p):
    """DG_{p-1} (X^3): the library's basis (1/|T| and the divergences of its RT_p interior eigenbasis) equals
    the oracle's dual basis of the cell DOFs at random reference points; d = 0."""
    from oracle.refelem import reference_element
    rng = np.random.default_rng(p)
    lam = rng.dirichlet(np.ones(4), size=40)
    V = np.array([[-1, -1 / np.sqrt(3), -1 / np.sqrt(6)], [1, -1 / np.sqrt(3), -1 / np.sqrt(6)],
                  [0, 2 / np.sqrt(3), -1 / np.sqrt(6)], [0, 0, 3 / np.sqrt(6)]])
    X = lam @ V
    vals, dvals = rz.riesz_ref_tabulate("DG", p, X)
    ve, _ = reference_element("DG", p).tabulate(X)
    assert vals.shape == ve.shape
    assert np.abs(vals - ve).max() <= 1e-11 * np.abs(ve).max()
    assert np.all(dvals == 0.0)
    with pytest.raises(rz.RieszError):
        rz.Riesz("DG", p, *kuhn_mesh(1), device=False)


@pytest.mark.parametrize("p", [1, 3])
def test_hodge_coupling_tables_k3_match_oracle(lib, p):
    """k = 3: (div phi^RT_j, psi^DG_i) on a random cell is the library's reference table over |det J| (the
    3-form and contravariant pullbacks leave a single metric factor)."""
    from oracle import assemble as asm
    from oracle.mesh import MeshDofs
    from oracle.refelem import reference_element
    rng = np.random.default_rng(30 + p)
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float) + 0.2 * rng.standard_normal((4, 3))
    cells = np.array([[0, 1, 2, 3]])
    r0, r1 = reference_element("RT", p), reference_element("DG", p)
    B = asm.mixed_matrix(r1, MeshDofs(verts, cells, r1), r0, MeshDofs(verts, cells, r0)).toarray()
    J, _ = asm.jacobians(verts, cells)
    R = rz.riesz_ref_mixed_tables(3, p)
    assert R.shape[0] == 1
    Bl = R[0] / abs(np.linalg.det(J[0]))
    assert np.abs(Bl.T - B).max() <= 1e-12 * np.abs(B).max()


@pytest.mark.parametrize("space,p", [("CG", 3), ("N1curl", 2), ("RT", 3)])
def test_partial_dirichlet_map_bit_exact(lib, space, p):
    """Dirichlet conditions on a part of the boundary (Eq. (2.8) with Gamma_D a proper part of the
    boundary): Gamma_D = the two faces x = 0 and y = 0 of the cube, chosen by flagging their vertices.
    The library's fixed DOFs equal the oracle's bit for bit, and their count is the closed form over the
    closure of Gamma_D (two n x n squares of 2n^2 triangles each sharing the edge x = y = 0)."""
    n = 3
    v, c = kuhn_mesh(n, 0.1, 2)
    x0 = np.isclose(v[:, 0], 0.0)
    y0 = np.isclose(v[:, 1], 0.0)
    mask = (x0 | y0).astype(np.uint8)
    s = rz.Riesz(space, p, v, c, device=False, dirichlet=1, dirichlet_vertices=mask)
    md = MeshDofs(v, c, reference_element(space, p))
    from oracle import assemble as asm
    D = asm.dirichlet_dofs(md, vertex_mask=mask)
    got = np.nonzero(s.dirichlet_map())[0]
    assert np.array_equal(got, D)
    # closure of two squares glued along an edge: vertices, edges and faces of Gamma_D
    nv_g = 2 * (n + 1) ** 2 - (n + 1)
    ne_g = 2 * (3 * n * n + 2 * n) - n
    nf_g = 2 * (2 * n * n)
    pv, pe, pf, _ = s.per_entity
    assert len(D) == pv * nv_g + pe * ne_g + pf * nf_g
    # a mask that flags no boundary face fixes nothing; the whole-boundary default is unchanged
    none = rz.Riesz(space, p, v, c, device=False, dirichlet=1, dirichlet_vertices=np.zeros(len(v), np.uint8))
    assert none.dirichlet_map().sum() == 0
    full = rz.Riesz(space, p, v, c, device=False, dirichlet=1)
    assert np.array_equal(np.nonzero(full.dirichlet_map())[0], asm.dirichlet_dofs(md))
