"""Global entities, DOF numbering and vertex-star patches (Section 5, Section 6.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Readings (the paper leaves numbering to Firedrake):

* The map F_T of Section 5 sends the reference vertices, in order, to the
  cell's vertices sorted by global index, so shared entities are seen with
  the same vertex order from every cell and no sign or permutation is needed.
* Edges are the sorted vertex pairs of the mesh, numbered in lexicographic
  order; faces the sorted vertex triples, lexicographic.
* Global layout: [vertex DOFs | edge DOFs (edge-major) | face DOFs
  (face-major) | interior DOFs (cell-major)]; inside an entity the reference
  element's order.  Interface DOFs therefore come first and the interior ones
  form one contiguous block at the end.
* The patch of vertex V (Eq. (6.11)) holds the interface DOFs of V and of
  every edge and face that contains V, in increasing global order.
"""
import numpy as np

from .refelem import EDGES, FACES


class MeshDofs:
    def __init__(self, verts, cells, ref):
        self.verts = np.asarray(verts, dtype=np.float64)
        cells = np.sort(np.asarray(cells, dtype=np.int64), axis=1)
        self.cells = cells
        nc = cells.shape[0]
        self.nverts = self.verts.shape[0]
        # entities
        eall = np.concatenate([cells[:, [a, b]] for (a, b) in EDGES], 0)
        self.edges, einv = np.unique(eall, axis=0, return_inverse=True)
        self.cell_edges = einv.reshape(len(EDGES), nc).T
        fall = np.concatenate([cells[:, [a, b, c]] for (a, b, c) in FACES], 0)
        self.faces, finv = np.unique(fall, axis=0, return_inverse=True)
        self.cell_faces = finv.reshape(len(FACES), nc).T
        # DOFs per entity from the reference element
        nv_d = len(ref.entity_dofs.get((0, 0), []))
        ne_d = len(ref.entity_dofs.get((1, 0), []))
        nf_d = len(ref.entity_dofs.get((2, 0), []))
        ni_d = len(ref.entity_dofs.get((3, 0), []))
        self.per_entity = (nv_d, ne_d, nf_d, ni_d)
        off_v = 0
        off_e = off_v + nv_d * self.nverts
        off_f = off_e + ne_d * len(self.edges)
        off_i = off_f + nf_d * len(self.faces)
        self.ndofs = off_i + ni_d * nc
        self.n_interface = off_i
        self.n_interior = ni_d * nc
        cd = np.zeros((nc, ref.ndofs), dtype=np.int64)
        for a in range(4):
            for m, j in enumerate(ref.entity_dofs.get((0, a), [])):
                cd[:, j] = off_v + nv_d * cells[:, a] + m
        for e in range(6):
            for m, j in enumerate(ref.entity_dofs.get((1, e), [])):
                cd[:, j] = off_e + ne_d * self.cell_edges[:, e] + m
        for f in range(4):
            for m, j in enumerate(ref.entity_dofs.get((2, f), [])):
                cd[:, j] = off_f + nf_d * self.cell_faces[:, f] + m
        for m, j in enumerate(ref.entity_dofs.get((3, 0), [])):
            cd[:, j] = off_i + ni_d * np.arange(nc) + m
        self.cell_dofs = cd
        self._offsets = (off_v, off_e, off_f)

    def vertex_star(self, v):
        """(edges, faces, cells) containing vertex v."""
        e = np.nonzero(np.any(self.edges == v, axis=1))[0]
        f = np.nonzero(np.any(self.faces == v, axis=1))[0]
        c = np.nonzero(np.any(self.cells == v, axis=1))[0]
        return e, f, c

    def patches(self):
        """List over vertices of the sorted interface DOFs of the vertex star."""
        nv_d, ne_d, nf_d, _ = self.per_entity
        off_v, off_e, off_f = self._offsets
        out = []
        for v in range(self.nverts):
            e, f, _ = self.vertex_star(v)
            d = [off_v + nv_d * v + m for m in range(nv_d)]
            d += [off_e + ne_d * x + m for x in e for m in range(ne_d)]
            d += [off_f + nf_d * x + m for x in f for m in range(nf_d)]
            out.append(np.array(sorted(d), dtype=np.int64))
        return out

    def patches_of(self, verts):
        """Sorted interface DOFs of the stars of the given vertices."""
        nv_d, ne_d, nf_d, _ = self.per_entity
        off_v, off_e, off_f = self._offsets
        out = []
        for v in verts:
            e, f, _ = self.vertex_star(v)
            d = [off_v + nv_d * v + m for m in range(nv_d)]
            d += [off_e + ne_d * x + m for x in e for m in range(ne_d)]
            d += [off_f + nf_d * x + m for x in f for m in range(nf_d)]
            out.append(np.array(sorted(d), dtype=np.int64))
        return out

    def vertices_of_dof(self, d):
        """Mesh vertices of the entity that owns interface DOF d."""
        nv_d, ne_d, nf_d, _ = self.per_entity
        off_v, off_e, off_f = self._offsets
        if d < off_e:
            return [int((d - off_v) // nv_d)]
        if d < off_f:
            return [int(v) for v in self.edges[(d - off_e) // ne_d]]
        return [int(v) for v in self.faces[(d - off_f) // nf_d]]
