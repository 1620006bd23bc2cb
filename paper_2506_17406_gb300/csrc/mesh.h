// Host topology: entities, global DOF numbering and vertex-star patches
// (arXiv 2506.17406, Section 5 and Section 6.1, Eq. (6.11)).
#pragma once
#include <cstdint>
#include <vector>

#include "refelem.h"

namespace riesz {

struct MeshMaps {
  int64_t nverts = 0, ncells = 0, nedges = 0, nfaces = 0;
  std::vector<int32_t> cells;       // ncells x 4, vertices sorted increasing
  std::vector<int32_t> edges;       // nedges x 2 (sorted pairs, lexicographic)
  std::vector<int32_t> faces;       // nfaces x 3 (sorted triples, lexicographic)
  std::vector<int32_t> cell_edges;  // ncells x 6 (local order 01,02,03,12,13,23)
  std::vector<int32_t> cell_faces;  // ncells x 4 (local order 012,013,023,123)
  int per_entity[4] = {0, 0, 0, 0};
  int nref = 0;
  int64_t ndofs = 0, n_interface = 0, n_interior = 0;
  int64_t off[4] = {0, 0, 0, 0};    // first DOF of vertices, edges, faces, interiors
  std::vector<int32_t> cell_dofs;   // ncells x nref (cell-major)
  // vertex-star patches: DOFs (ascending) and star cells
  std::vector<int64_t> patch_ptr;   // nverts + 1
  std::vector<int32_t> patch_dofs;
  std::vector<int64_t> star_ptr;    // nverts + 1
  std::vector<int32_t> star_cells;
};

// Throws std::runtime_error on invalid input.
MeshMaps build_mesh(const RefElement& R, int64_t nverts, int64_t ncells, const int64_t* cells);

}  // namespace riesz
