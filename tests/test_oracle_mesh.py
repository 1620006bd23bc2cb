"""Pins of the oracle's numbering and patches against the paper's printed counts."""
import os

import numpy as np
import pytest

from oracle.mesh import MeshDofs
from oracle.refelem import reference_element
from paper_2506_17406_gb300.inputs import kuhn_mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            out.append(line.split())
    return out


@pytest.mark.parametrize("space", ["CG", "N1curl", "RT"])
def test_dof_counts_match_paper_tables(space):
    """Every 'dofs' entry of Tables 3-5 (levels 0-2, p = 2..7)."""
    rows = [r for r in _rows("paper_dof_counts.txt") if r[0] == space]
    assert len(rows) == 18
    meshes = {}
    for _, level, p, dofs, *_ in rows:
        n = 3 * 2 ** int(level)
        if n not in meshes:
            meshes[n] = kuhn_mesh(n)
        v, c = meshes[n]
        md = MeshDofs(v, c, reference_element(space, int(p)))
        assert md.ndofs == int(dofs), (space, level, p)


def test_interior_star_counts():
    """Section 6.1: an interior vertex star has 14 edges, 36 faces, 24 cells."""
    v, c = kuhn_mesh(3)
    md = MeshDofs(v, c, reference_element("CG", 1))
    for vi in range(len(v)):
        ijk = np.array([vi % 4, (vi // 4) % 4, vi // 16])
        e, f, cc = md.vertex_star(vi)
        if np.all((ijk > 0) & (ijk < 3)):
            assert (len(e), len(f), len(cc)) == (14, 36, 24)
        else:
            assert len(cc) < 24


class _CountsOnly:
    """Per-entity DOF counts of a reference element (closed forms of Eq. (3.8))."""

    def __init__(self, space, p):
        if space == "CG":
            c = (1, p - 1, (p - 1) * (p - 2) // 2, (p - 1) * (p - 2) * (p - 3) // 6)
        elif space == "N1curl":
            c = (0, p, p * (p - 1), p * (p + 2) * (p + 3) // 2 - 6 * p - 4 * p * (p - 1))
        else:
            c = (0, 0, p * (p + 1) // 2, p * (p + 1) * (p - 1) // 2)
        self.entity_dofs = {}
        k = 0
        for dim, nent in ((0, 4), (1, 6), (2, 4), (3, 1)):
            for e in range(nent):
                self.entity_dofs[(dim, e)] = list(range(k, k + c[dim]))
                k += c[dim]
        self.ndofs = k


@pytest.mark.parametrize("space,p,iface,full", [tuple(r[:1]) + tuple(int(x) for x in r[1:])
                                                for r in _rows("paper_patch_sizes.txt")])
def test_patch_sizes_match_paper(space, p, iface, full):
    """Section 6.1 text and Tables 1-2: interior vertex patch dimensions."""
    v, c = kuhn_mesh(2)
    ref = reference_element(space, p) if p <= 4 else _CountsOnly(space, p)
    if p <= 4:  # the closed-form counts agree with the built element
        cnt = _CountsOnly(space, p)
        for key, d in ref.entity_dofs.items():
            assert len(d) == len(cnt.entity_dofs[key])
    md = MeshDofs(v, c, ref)
    pt = md.patches()
    centre = 1 + 3 * (1 + 3 * 1)
    assert len(pt[centre]) == iface
    assert max(len(q) for q in pt) == iface
    n_int = len(ref.entity_dofs[(3, 0)])
    assert iface + 24 * n_int == full


def test_numbering_layout():
    """Interface DOFs first, interior DOFs last and contiguous per cell; every DOF used."""
    v, c = kuhn_mesh(2, 0.1, 3)
    for space, p in [("CG", 4), ("N1curl", 3), ("RT", 3)]:
        ref = reference_element(space, p)
        md = MeshDofs(v, c, ref)
        used = np.zeros(md.ndofs, dtype=int)
        np.add.at(used, md.cell_dofs.ravel(), 1)
        assert np.all(used > 0)
        I = ref.interior
        assert np.all(md.cell_dofs[:, I] >= md.n_interface)
        if I:
            exp = md.n_interface + np.arange(len(c))[:, None] * len(I) + np.arange(len(I))[None, :]
            assert np.array_equal(md.cell_dofs[:, I], exp)
        assert np.all(used[md.n_interface:] == 1)


@pytest.mark.parametrize("space,p,edge,vert", [tuple(r[:1]) + (int(r[1]), int(r[2]), r[3])
                                               for r in _rows("paper_edge_patch_sizes.txt")])
def test_edge_patch_sizes_match_paper(space, p, edge, vert):
    """Tables 1-2: largest edge-star patches of the HT decomposition (type-I DOFs, Eq. (6.19)) and of
    PAFW_1 for H(div) (Eq. (6.24)); the HT potential problem on the largest vertex star."""
    from oracle import assemble as asm
    v, c = kuhn_mesh(2)
    ref = reference_element(space, p) if p <= 4 else _CountsOnly(space, p)
    md = MeshDofs(v, c, ref)
    if space == "N1curl":
        rc = reference_element("CG", p) if p <= 4 else _CountsOnly("CG", p)
        mc = MeshDofs(v, c, rc)
        stars = asm.edge_star_type1_dofs(md, mc)
        assert max(len(q) for q in mc.patches()) == int(vert)
    else:
        stars = asm.edge_star_dofs(md)
    assert max(len(q) for q in stars) == edge
