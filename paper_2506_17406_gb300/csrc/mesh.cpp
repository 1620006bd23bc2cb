// Host topology for the Riesz-map solver.
//
// The affine map of every cell sends the reference vertices, in order, to the
// cell's vertices sorted by global index (Section 5: F_T preserves fixed
// global orientations), so a shared edge or face is seen with the same vertex
// order from every cell and gather/scatter need no signs or permutations.
// Numbering: [vertex DOFs | edge DOFs (edge-major) | face DOFs (face-major) |
// interior DOFs (cell-major)], edges and faces in lexicographic order of their
// sorted vertices.  The patch of vertex V (Eq. (6.11)) holds the interface
// DOFs of V and of every edge and face containing V, in increasing order.
#include "mesh.h"

#include <algorithm>
#include <array>
#include <stdexcept>

namespace riesz {

MeshMaps build_mesh(const RefElement& R, int64_t nverts, int64_t ncells, const int64_t* cells_in) {
  MeshMaps M;
  if (nverts <= 0 || ncells <= 0) throw std::runtime_error("mesh: empty mesh");
  if (nverts > (int64_t)1 << 30 || ncells > (int64_t)1 << 28) throw std::runtime_error("mesh: too large");
  M.nverts = nverts;
  M.ncells = ncells;
  M.cells.resize((size_t)ncells * 4);
  for (int64_t c = 0; c < ncells; ++c) {
    std::array<int64_t, 4> v;
    for (int k = 0; k < 4; ++k) {
      v[k] = cells_in[c * 4 + k];
      if (v[k] < 0 || v[k] >= nverts) throw std::runtime_error("mesh: vertex index out of range");
    }
    std::sort(v.begin(), v.end());
    for (int k = 0; k < 3; ++k)
      if (v[k] == v[k + 1]) throw std::runtime_error("mesh: repeated vertex in a cell");
    for (int k = 0; k < 4; ++k) M.cells[c * 4 + k] = (int32_t)v[k];
  }
  static const int E[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  static const int F[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
  // edges
  std::vector<std::array<int32_t, 2>> ev((size_t)ncells * 6);
  for (int64_t c = 0; c < ncells; ++c)
    for (int e = 0; e < 6; ++e) ev[c * 6 + e] = {M.cells[c * 4 + E[e][0]], M.cells[c * 4 + E[e][1]]};
  std::vector<std::array<int32_t, 2>> eu(ev);
  std::sort(eu.begin(), eu.end());
  eu.erase(std::unique(eu.begin(), eu.end()), eu.end());
  M.nedges = (int64_t)eu.size();
  M.edges.resize(eu.size() * 2);
  for (size_t i = 0; i < eu.size(); ++i) {
    M.edges[i * 2] = eu[i][0];
    M.edges[i * 2 + 1] = eu[i][1];
  }
  M.cell_edges.resize((size_t)ncells * 6);
  for (size_t i = 0; i < ev.size(); ++i)
    M.cell_edges[i] = (int32_t)(std::lower_bound(eu.begin(), eu.end(), ev[i]) - eu.begin());
  // faces
  std::vector<std::array<int32_t, 3>> fv((size_t)ncells * 4);
  for (int64_t c = 0; c < ncells; ++c)
    for (int f = 0; f < 4; ++f)
      fv[c * 4 + f] = {M.cells[c * 4 + F[f][0]], M.cells[c * 4 + F[f][1]], M.cells[c * 4 + F[f][2]]};
  std::vector<std::array<int32_t, 3>> fu(fv);
  std::sort(fu.begin(), fu.end());
  fu.erase(std::unique(fu.begin(), fu.end()), fu.end());
  M.nfaces = (int64_t)fu.size();
  M.faces.resize(fu.size() * 3);
  for (size_t i = 0; i < fu.size(); ++i)
    for (int k = 0; k < 3; ++k) M.faces[i * 3 + k] = fu[i][k];
  M.cell_faces.resize((size_t)ncells * 4);
  for (size_t i = 0; i < fv.size(); ++i)
    M.cell_faces[i] = (int32_t)(std::lower_bound(fu.begin(), fu.end(), fv[i]) - fu.begin());
  // numbering
  for (int d = 0; d < 4; ++d) M.per_entity[d] = R.per_entity[d];
  M.nref = R.nref;
  M.off[0] = 0;
  M.off[1] = M.off[0] + (int64_t)R.per_entity[0] * nverts;
  M.off[2] = M.off[1] + (int64_t)R.per_entity[1] * M.nedges;
  M.off[3] = M.off[2] + (int64_t)R.per_entity[2] * M.nfaces;
  M.ndofs = M.off[3] + (int64_t)R.per_entity[3] * ncells;
  if (M.ndofs >= ((int64_t)1 << 31)) throw std::runtime_error("mesh: more than 2^31 DOFs");
  M.n_interface = M.off[3];
  M.n_interior = M.ndofs - M.off[3];
  const int nr = R.nref;
  M.cell_dofs.resize((size_t)ncells * nr);
  for (int64_t c = 0; c < ncells; ++c) {
    int32_t* cd = &M.cell_dofs[c * nr];
    int j = 0;
    for (int a = 0; a < 4; ++a)
      for (int m = 0; m < R.per_entity[0]; ++m) cd[j++] = (int32_t)(M.off[0] + (int64_t)R.per_entity[0] * M.cells[c * 4 + a] + m);
    for (int e = 0; e < 6; ++e)
      for (int m = 0; m < R.per_entity[1]; ++m)
        cd[j++] = (int32_t)(M.off[1] + (int64_t)R.per_entity[1] * M.cell_edges[c * 6 + e] + m);
    for (int f = 0; f < 4; ++f)
      for (int m = 0; m < R.per_entity[2]; ++m)
        cd[j++] = (int32_t)(M.off[2] + (int64_t)R.per_entity[2] * M.cell_faces[c * 4 + f] + m);
    for (int m = 0; m < R.per_entity[3]; ++m) cd[j++] = (int32_t)(M.off[3] + (int64_t)R.per_entity[3] * c + m);
    if (j != nr) throw std::runtime_error("mesh: reference DOF layout mismatch");
  }
  // vertex -> edges, faces, cells (counting sort keeps entity order ascending)
  std::vector<int64_t> ve_ptr(nverts + 1, 0), vf_ptr(nverts + 1, 0);
  M.star_ptr.assign(nverts + 1, 0);
  for (int64_t e = 0; e < M.nedges; ++e)
    for (int k = 0; k < 2; ++k) ve_ptr[M.edges[e * 2 + k] + 1]++;
  for (int64_t f = 0; f < M.nfaces; ++f)
    for (int k = 0; k < 3; ++k) vf_ptr[M.faces[f * 3 + k] + 1]++;
  for (int64_t c = 0; c < ncells; ++c)
    for (int k = 0; k < 4; ++k) M.star_ptr[M.cells[c * 4 + k] + 1]++;
  for (int64_t v = 0; v < nverts; ++v) {
    ve_ptr[v + 1] += ve_ptr[v];
    vf_ptr[v + 1] += vf_ptr[v];
    M.star_ptr[v + 1] += M.star_ptr[v];
  }
  std::vector<int32_t> ve(ve_ptr[nverts]), vf(vf_ptr[nverts]);
  M.star_cells.resize(M.star_ptr[nverts]);
  {
    std::vector<int64_t> a(ve_ptr.begin(), ve_ptr.end() - 1), b(vf_ptr.begin(), vf_ptr.end() - 1),
        s(M.star_ptr.begin(), M.star_ptr.end() - 1);
    for (int64_t e = 0; e < M.nedges; ++e)
      for (int k = 0; k < 2; ++k) ve[a[M.edges[e * 2 + k]]++] = (int32_t)e;
    for (int64_t f = 0; f < M.nfaces; ++f)
      for (int k = 0; k < 3; ++k) vf[b[M.faces[f * 3 + k]]++] = (int32_t)f;
    for (int64_t c = 0; c < ncells; ++c)
      for (int k = 0; k < 4; ++k) M.star_cells[s[M.cells[c * 4 + k]]++] = (int32_t)c;
  }
  M.patch_ptr.assign(nverts + 1, 0);
  for (int64_t v = 0; v < nverts; ++v)
    M.patch_ptr[v + 1] = M.patch_ptr[v] + R.per_entity[0] + (ve_ptr[v + 1] - ve_ptr[v]) * R.per_entity[1] +
                         (vf_ptr[v + 1] - vf_ptr[v]) * R.per_entity[2];
  M.patch_dofs.resize(M.patch_ptr[nverts]);
  for (int64_t v = 0; v < nverts; ++v) {
    int64_t k = M.patch_ptr[v];
    for (int m = 0; m < R.per_entity[0]; ++m) M.patch_dofs[k++] = (int32_t)(M.off[0] + (int64_t)R.per_entity[0] * v + m);
    for (int64_t i = ve_ptr[v]; i < ve_ptr[v + 1]; ++i)
      for (int m = 0; m < R.per_entity[1]; ++m) M.patch_dofs[k++] = (int32_t)(M.off[1] + (int64_t)R.per_entity[1] * ve[i] + m);
    for (int64_t i = vf_ptr[v]; i < vf_ptr[v + 1]; ++i)
      for (int m = 0; m < R.per_entity[2]; ++m) M.patch_dofs[k++] = (int32_t)(M.off[2] + (int64_t)R.per_entity[2] * vf[i] + m);
  }
  return M;
}

}  // namespace riesz
