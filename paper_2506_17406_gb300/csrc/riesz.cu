// C ABI of the Riesz-map solver: handle, host/device setup, apply, precond,
// PCG.  See include/riesz.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/riesz.h"
#include "kernels.cuh"
#include "tc_apply.cuh"
#include "mesh.h"
#include "refelem.h"

using namespace riesz;

namespace {

thread_local std::string g_err;

struct Err : std::runtime_error {
  int code;
  Err(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CK(x)                                                                                        \
  do {                                                                                               \
    cudaError_t e_ = (x);                                                                            \
    if (e_ != cudaSuccess)                                                                           \
      throw Err(e_ == cudaErrorMemoryAllocation ? RIESZ_ERR_OOM : RIESZ_ERR_CUDA,                    \
                std::string(#x) + ": " + cudaGetErrorString(e_));                                    \
  } while (0)

#define KCHECK() CK(cudaGetLastError())

template <typename T>
struct DBuf {  // device buffer owned by the handle
  T* p = nullptr;
  size_t n = 0;
  void alloc(size_t count) {
    free();
    n = count;
    if (count) CK(cudaMalloc((void**)&p, count * sizeof(T)));
  }
  void upload(const std::vector<T>& v, cudaStream_t s) {
    alloc(v.size());
    if (n) CK(cudaMemcpyAsync(p, v.data(), n * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  void free() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
};

}  // namespace

struct riesz_handle {
  int space = 0, p = 0;  // space: k (0, 1, 2)
  int kind = 1;          // 1: CG_p / Ned1_p / RT_p (Eq. (2.5)), 2: NedTwo_p / BDM_p (Eq. (2.6))
  riesz_opts opts;
  const RefElement* ref = nullptr;
  const RefElement* refcg = nullptr;  // CG_p: the load's source field
  std::vector<double> verts;
  MeshMaps mesh, meshcg;
  MeshMaps meshpot;  // CG_{p+1}: the Hiptmair-Toselli potentials of NedTwo_p (kind 2 only)
  int nif = 0;  // interface DOFs per cell
  // host-side plans
  std::vector<int64_t> sc_ptr;   // interface DOF -> positions in Ycell
  std::vector<int32_t> sc_pos;
  std::vector<int32_t> p_n;      // patches in launch order (largest first)
  std::vector<int64_t> p_doff, p_foff, p_dioff, p_moff;  // DOF list, factor tiles, diagonal inverses, tile map
  std::vector<int32_t> p_meta;  // per patch: tile index map [nb*nb] (-1 = zero tile) then the block column of each stored tile
  int64_t tile_ops = 0;         // 32x32x32 tile products of the symbolic factorisation (all patches)
  double chol_flops = 0.0;      // flops of the tile-sparse Cholesky (all patches)
  std::vector<int32_t> p_dofs;
  std::vector<int64_t> pz_ptr;   // interface DOF -> positions in zpatch
  std::vector<int32_t> pz_pos;
  std::vector<int64_t> pb_ptr, pb_off;
  std::vector<int32_t> pb_cell, pb_ent;
  int64_t factor_entries = 0, dinv_entries = 0;
  double setup_host_ms = 0.0, setup_dev_ms = 0.0;
  // device state
  bool on_device = false;
  int device = 0;
  DBuf<double> d_verts, d_g, d_jac, d_R, d_Ae, d_Ycell, d_dinv, d_L64, d_D64, d_zpatch, d_X;
  DBuf<float> d_L32, d_D32, d_Ae32;
  DBuf<float> d_L32T, d_D32T;  // tile-transposed FP32 factors (forward sweep of several right-hand sides)
  // Hiptmair-Toselli decomposition (H(curl)): type-I edge-star patches on this
  // handle, gradient potential problems on the CG vertex stars of `aux`, and the
  // gradient map: CG interface DOF -> (Ned1 DOF, sign) and Ned1 interface DOF ->
  // (CG DOF, sign) (Eq. (5.3))
  bool ht = false;
  riesz_handle* aux = nullptr;
  // edge-star patches (Hiptmair-Toselli for H(curl), PAFW_1 for H(div)): CSR edge -> sorted DOFs
  bool edge_star = false;
  bool apply_only = false;  // internal operator handles (Hodge-Laplace blocks): no patches, no coarse space
  std::vector<int64_t> es_ptr;
  std::vector<int32_t> es_dofs;
  std::vector<int64_t> gt_ptr, gg_ptr;
  std::vector<int32_t> gt_idx, gg_idx;
  std::vector<float> gt_sgn, gg_sgn;
  DBuf<int64_t> d_gt_ptr, d_gg_ptr;
  DBuf<int32_t> d_gt_idx, d_gg_idx;
  DBuf<float> d_gt_sgn, d_gg_sgn;
  DBuf<double> d_zcg, d_zg;  // potential corrections [nrhs][n_if(CG)], their gradients [nrhs][n_if]
  // homogeneous Dirichlet DOFs (all DOFs of boundary entities), flag per interface DOF
  std::vector<uint8_t> dir_mask;
  DBuf<uint8_t> d_dmask;
  const uint8_t* dmask() const { return opts.dirichlet ? d_dmask.p : nullptr; }
  // W^k coarse space: coarse DOF -> global DOF, interface DOF -> coarse index,
  // per coarse row the (J, cell, local a | b << 16) contributions of A_0
  bool coarse_on = false;
  int N0 = 0, N0p = 0, coarse_group = 8;
  std::vector<int32_t> c_w, c_idx, c_J, c_cell, c_ab;
  std::vector<int64_t> c_ptr;
  DBuf<int32_t> d_cw, d_cidx, d_cJ, d_ccell, d_cab;
  DBuf<int64_t> d_cptr;
  // the same in FP64 for ill-conditioned coarse matrices (beta/alpha far from 1, and the blocks of
  // the Hodge-Laplace preconditioner), where the FP32 inverse stops being positive definite
  DBuf<double> d_A0d, d_Dinv0d, d_Rb0d, d_r0d;
  DBuf<double> d_X0d;   // FP64 path: X = -(L^{-T} L^{-1}) (the factor and its inverse are built in d_A0d)
  DBuf<int> d_cbad;     // non-positive pivot in the coarse Cholesky
  DBuf<double> d_zc;                  // coarse corrections [nrhs][N0]
  // hybrid form (opts.form): the subspace weights rho_1..3 (index 0 unused), fixed once set by
  // the caller, and the sweep's residual, correction and product vectors [nrhs][N]
  double rho[4] = {0.0, 1.0, 1.0, 1.0};
  bool rho_fixed = false;
  DBuf<double> d_hres, d_hc, d_hAc;
  // BF16x3 tensor-core contraction (apply_precision = RIESZ_PREC_BF16X3): the split reference
  // matrices in the kernel's stage layout, n padded to 16 (tc_np) and the number of 32-wide K chunks
  DBuf<uint16_t> d_Btc;
  int tc_np = 0, tc_kc = 0;
  // coarse solve above the dense limit (or opts.coarse = 2): A_0 is the lowest-order Riesz map
  // on the same mesh (Lemma 4.1), held by an internal p = 1 handle with its own vertex-star
  // patches; a coarse application runs opts.coarse_its PCG steps on it.  c_aux maps coarse index
  // -> that handle's DOF (its entity index)
  bool coarse_sparse = false;
  riesz_handle* caux = nullptr;
  std::vector<int32_t> c_aux;
  DBuf<int32_t> d_caux;
  int multi_group = 8;  // right-hand sides per k_patch_solve_multi launch
  int chol_ctas = 0;    // resident k_cholesky CTAs per SM picked by the autotuner (0: no limit)
  // FP32 sweeps of several right-hand sides over patches of at most 8 tiles: 0 one CTA per patch
  // (bulk-copy ring, k_patch_sweep8), 4 or 8: one warp per patch with that many warps per block
  int sweep_shape = 8;
  int sweep_tuned = 0;  // candidates the autotuner timed
  int chol_tuned = 0;   // candidates the autotuner timed
  int chol_split = 1;   // CTAs per patch in the factorisation (1, or a 2-CTA cluster)
  DBuf<int32_t> d_cells, d_cdofs, d_sc_pos, d_pn, d_pdofs, d_pz_pos, d_pb_cell, d_pb_ent, d_cgdofs, d_meta;
  DBuf<int64_t> d_sc_ptr, d_pdoff, d_pfoff, d_pdioff, d_pmoff, d_pz_ptr, d_pb_ptr, d_pb_off;
  DBuf<int> d_info;  // Cholesky status per patch
  DBuf<unsigned> d_ticket;    // last-block ticket of the fused reductions
  // PCG workspace
  DBuf<double> d_r, d_z, d_zold, d_p, d_Ap, d_part, d_scal, d_tmp, d_xh, d_xw;
  double* h_scal = nullptr;  // pinned
  // device-driven PCG loop: control words, their pinned copy, the capture
  // stream and the instantiated loop graphs (entry after a restart, resume)
  DBuf<int> d_ctl;
  int* h_ctl = nullptr;  // pinned [4]
  DBuf<int> d_flags;     // [0]: a bulk-copy wait of the patch sweeps timed out
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side_stream = nullptr;  // setup work that runs beside the patch factorisation
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_pfork = nullptr, ev_pjoin = nullptr;
  cudaStream_t ht_stream = nullptr;  // the potential problems (setup and per application) beside the edge stars
  cudaEvent_t ev_hfork = nullptr, ev_hjoin = nullptr;
  cudaStream_t batch_stream = nullptr;  // this handle's device setup inside a batched setup
  cudaEvent_t ev_batch = nullptr;
  cudaGraphExec_t g_entry = nullptr, g_resume = nullptr;
  int g_nrhs = 0;
  int64_t g_pro_launches = 0, g_body_launches = 0;
  cudaEvent_t ev_scal = nullptr;  // marks the arrival of h_scal
  int last_iters = 0;
  int64_t launches = 0;
  // per-kernel CUDA-event profiler (riesz_profile)
  bool prof = false;
  unsigned prof_mask = 0;  // kinds recorded by the profiler (bit k = kind k)
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> prof_pending;  // (kind, first event index)
  double prof_ms[RIESZ_NKIND] = {0};
  int64_t prof_cnt[RIESZ_NKIND] = {0};
  int64_t N() const { return mesh.ndofs; }
  int64_t C() const { return mesh.ncells; }
  size_t device_bytes() const {
    return d_verts.bytes() + d_g.bytes() + d_jac.bytes() + d_R.bytes() + d_Ae.bytes() + d_Ycell.bytes() +
           d_dinv.bytes() + d_L64.bytes() + d_L32.bytes() + d_L32T.bytes() + d_D32T.bytes() + d_Ae32.bytes() + d_D64.bytes() + d_D32.bytes() + d_zpatch.bytes() + d_X.bytes() + d_cells.bytes() +
           d_cdofs.bytes() + d_sc_pos.bytes() + d_pn.bytes() + d_pdofs.bytes() + d_pz_pos.bytes() +
           d_pb_cell.bytes() + d_pb_ent.bytes() + d_cgdofs.bytes() + d_sc_ptr.bytes() + d_pdoff.bytes() +
           d_pfoff.bytes() + d_pdioff.bytes() + d_pmoff.bytes() + d_meta.bytes() + d_pz_ptr.bytes() + d_pb_ptr.bytes() + d_pb_off.bytes() + d_r.bytes() + d_z.bytes() +
           d_zold.bytes() + d_p.bytes() + d_Ap.bytes() + d_part.bytes() + d_scal.bytes() + d_tmp.bytes() + d_xh.bytes() +
           d_xw.bytes() + d_ctl.bytes() + d_flags.bytes() + d_dmask.bytes() + d_gt_ptr.bytes() + d_gg_ptr.bytes() +
           d_gt_idx.bytes() + d_gg_idx.bytes() + d_gt_sgn.bytes() + d_gg_sgn.bytes() + d_zcg.bytes() + d_zg.bytes() +
           (aux ? aux->device_bytes() : 0) + d_cw.bytes() + d_cidx.bytes() + d_cJ.bytes() +
           d_ccell.bytes() + d_cab.bytes() + d_cptr.bytes() +
           d_zc.bytes() + d_A0d.bytes() + d_X0d.bytes() + d_Dinv0d.bytes() + d_Rb0d.bytes() + d_r0d.bytes() +
           d_info.bytes() + d_ticket.bytes() + d_cbad.bytes() + d_caux.bytes() + (caux ? caux->device_bytes() : 0) +
           d_hres.bytes() + d_hc.bytes() + d_hAc.bytes() + d_Btc.bytes();
  }
  void drop_graphs() {
    if (g_entry) cudaGraphExecDestroy(g_entry);
    if (g_resume) cudaGraphExecDestroy(g_resume);
    g_entry = g_resume = nullptr;
    g_nrhs = 0;
  }
  void free_device() {
    drop_graphs();
    for (auto* b : {&d_verts, &d_g, &d_jac, &d_R, &d_Ae, &d_Ycell, &d_dinv, &d_L64, &d_D64, &d_zpatch, &d_X, &d_r, &d_z,
                    &d_zold, &d_p, &d_Ap, &d_part, &d_scal, &d_tmp, &d_xh, &d_xw})
      b->free();
    d_ctl.free();
    d_flags.free();
    d_dmask.free();
    d_gt_ptr.free();
    d_gg_ptr.free();
    d_gt_idx.free();
    d_gg_idx.free();
    d_gt_sgn.free();
    d_gg_sgn.free();
    d_zcg.free();
    d_zg.free();
    for (auto* b : {&d_cw, &d_cidx, &d_cJ, &d_ccell, &d_cab}) b->free();
    d_cptr.free();
    d_A0d.free();
    d_X0d.free();
    d_cbad.free();
    d_Dinv0d.free();
    d_Rb0d.free();
    d_r0d.free();
    d_zc.free();
    d_caux.free();
    if (caux) caux->free_device();
    d_hres.free();
    d_hc.free();
    d_hAc.free();
    d_Btc.free();
    if (h_ctl) cudaFreeHost(h_ctl);
    h_ctl = nullptr;
    d_L32.free();
    d_L32T.free();
    d_D32T.free();
    d_D32.free();
    d_Ae32.free();
    for (auto* b : {&d_cells, &d_cdofs, &d_sc_pos, &d_pn, &d_pdofs, &d_pz_pos, &d_pb_cell, &d_pb_ent, &d_cgdofs, &d_meta})
      b->free();
    for (auto* b : {&d_sc_ptr, &d_pdoff, &d_pfoff, &d_pdioff, &d_pmoff, &d_pz_ptr, &d_pb_ptr, &d_pb_off}) b->free();
    d_info.free();
    d_ticket.free();
    if (h_scal) cudaFreeHost(h_scal);
    h_scal = nullptr;
    on_device = false;
  }
  ~riesz_handle() {
    free_device();
    if (ev_scal) cudaEventDestroy(ev_scal);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (side_stream) cudaStreamDestroy(side_stream);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_pfork) cudaEventDestroy(ev_pfork);
    if (ev_pjoin) cudaEventDestroy(ev_pjoin);
    if (ht_stream) cudaStreamDestroy(ht_stream);
    if (ev_hfork) cudaEventDestroy(ev_hfork);
    if (ev_hjoin) cudaEventDestroy(ev_hjoin);
    if (batch_stream) cudaStreamDestroy(batch_stream);
    if (ev_batch) cudaEventDestroy(ev_batch);
    delete aux;
    delete caux;
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  }
};

namespace {

template <typename F>
int guarded(F&& f) {
  try {
    f();
    return RIESZ_OK;
  } catch (const Err& e) {
    g_err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return RIESZ_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return RIESZ_ERR_INVALID_ARG;
  }
}

void need(bool ok, const char* msg, int code = RIESZ_ERR_INVALID_ARG) {
  if (!ok) throw Err(code, msg);
}

// Launch a kernel (callable f) of the given kind on stream s; with the
// profiler on, bracket it with a pair of pooled CUDA events.
template <typename F>
void launch(riesz_handle& h, int kind, cudaStream_t s, F&& f) {
  size_t e = 0;
  const bool rec = h.prof && ((h.prof_mask >> kind) & 1u);
  if (rec) {
    while (h.ev_pool.size() < h.ev_used + 2) {
      cudaEvent_t ev;
      CK(cudaEventCreate(&ev));
      h.ev_pool.push_back(ev);
    }
    e = h.ev_used;
    h.ev_used += 2;
    CK(cudaEventRecord(h.ev_pool[e], s));
  }
  f();
  CK(cudaGetLastError());
  ++h.launches;
  if (rec) {
    CK(cudaEventRecord(h.ev_pool[e + 1], s));
    h.prof_pending.push_back({kind, e});
  }
}

void prof_collect(riesz_handle& h) {
  for (auto& pe : h.prof_pending) {
    CK(cudaEventSynchronize(h.ev_pool[pe.second + 1]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h.ev_pool[pe.second], h.ev_pool[pe.second + 1]));
    h.prof_ms[pe.first] += ms;
    h.prof_cnt[pe.first] += 1;
  }
  h.prof_pending.clear();
  h.ev_used = 0;
}

// reference edge matrix inverse (columns V1-V0, V2-V0, V3-V0 of the reference tetrahedron)
dev::Mat3 ref_edge_inverse() {
  const double s3 = std::sqrt(3.0), s6 = std::sqrt(6.0);
  const double V[4][3] = {{-1.0, -1.0 / s3, -1.0 / s6}, {1.0, -1.0 / s3, -1.0 / s6}, {0.0, 2.0 / s3, -1.0 / s6},
                          {0.0, 0.0, 3.0 / s6}};
  Mat E(3, 3);
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < 3; ++k) E(d, k) = V[k + 1][d] - V[0][d];
  Mat Ei = inverse(E);
  dev::Mat3 m;
  for (int k = 0; k < 9; ++k) m.a[k] = Ei(k / 3, k % 3);
  return m;
}

// Plan one vertex-star patch (Eq. (6.11)): order its DOFs, record the cell
// contributions for the assembly and the tile structure of its Cholesky factor.
//
// The factorisation of P A_V P^T for any permutation P gives the same operator
// R_V^T A_V^{-1} R_V.  Entities (the vertex, edges and faces of the star) are
// ordered by a Fiedler-type vector of their adjacency graph (two entities are
// adjacent when a star cell contains both): power iteration of (c I - Lap)
// started from the entity midpoints projected on (1,1,1) and orthogonal to the
// constant.  The link of a vertex is a sphere-like graph, so this orders the
// DOFs in bands and leaves most 32x32 tiles of the factor zero.  The tile
// pattern of the factor is the symbolic tile-level Cholesky of the pattern of
// A_V; only nonzero tiles are stored, in block-row order.
// Plan one patch: its DOFs pd[0..np) (ascending interface DOFs) and the cells
// of its star (cells whose interface DOFs may touch it); `center` is a point
// of the star (the Fiedler ordering uses coordinates relative to it).  The plan
// depends on the patch alone (build_plans computes the plans of many patches at
// once on host threads), and append_patch adds it to the handle in patch order.
struct PatchPlan {
  int np = 0, nb = 0, nt = 0;
  std::vector<int32_t> dofs;           // the patch DOFs in factor order
  std::vector<int32_t> meta;           // [nb][nb] tile index (-1: zero tile), then the column of every tile
  std::vector<int32_t> cells;          // star cells holding patch DOFs
  std::vector<int64_t> cell_end;       // end of each cell's entries in ent
  std::vector<int32_t> ent;            // (local DOF j) | (factor position << 10) per (cell, patch DOF)
  int64_t tile_ops = 0;
  std::vector<double> col_flops;       // flops of each block column of the factorisation
};

PatchPlan plan_patch(const riesz_handle& h, const int32_t* pd, int np, const int32_t* star, int64_t nstar,
                     const double* center) {
  PatchPlan P;
  const MeshMaps& M = h.mesh;
  const int n = M.nref;
  // entities: contiguous runs of the sorted patch DOF list with the same entity
  std::vector<int> ent_start, ent_len, dof_ent(np);
  std::vector<std::array<double, 3>> mid;
  const double* X = h.verts.data();
  for (int k = 0; k < np;) {
    const int64_t d = pd[k];
    int kind = (d < M.off[1]) ? 0 : (d < M.off[2] ? 1 : 2);
    const int per = M.per_entity[kind];
    const int64_t id = (d - M.off[kind]) / per;
    int run = 1;
    while (k + run < np && pd[k + run] < M.off[kind] + (id + 1) * per && pd[k + run] >= M.off[kind] + id * per) ++run;
    std::array<double, 3> m = {0.0, 0.0, 0.0};
    int nvx = 0;
    int32_t vv[3];
    if (kind == 0) {
      vv[0] = (int32_t)id;
      nvx = 1;
    } else if (kind == 1) {
      vv[0] = M.edges[id * 2];
      vv[1] = M.edges[id * 2 + 1];
      nvx = 2;
    } else {
      for (int q = 0; q < 3; ++q) vv[q] = M.faces[id * 3 + q];
      nvx = 3;
    }
    for (int q = 0; q < nvx; ++q)
      for (int c = 0; c < 3; ++c) m[c] += (X[(size_t)vv[q] * 3 + c] - center[c]) / nvx;
    const int ei = (int)ent_start.size();
    ent_start.push_back(k);
    ent_len.push_back(run);
    mid.push_back(m);
    for (int q = 0; q < run; ++q) dof_ent[k + q] = ei;
    k += run;
  }
  const int ne = (int)ent_start.size();
  // star cells -> patch entities (and DOF positions)
  std::vector<std::vector<int>> cell_ents;
  std::vector<int32_t> cell_ids;
  std::vector<std::vector<std::pair<int, int>>> cell_locs;  // (local j, sorted patch index)
  for (int64_t sidx = 0; sidx < nstar; ++sidx) {
    const int32_t c = star[sidx];
    std::vector<int> ce;
    std::vector<std::pair<int, int>> loc;
    for (int j = 0; j < h.nif; ++j) {
      const int32_t gd = M.cell_dofs[(int64_t)c * n + j];
      const int32_t* it = std::lower_bound(pd, pd + np, gd);
      if (it != pd + np && *it == gd) {
        const int k = (int)(it - pd);
        loc.push_back({j, k});
        if (std::find(ce.begin(), ce.end(), dof_ent[k]) == ce.end()) ce.push_back(dof_ent[k]);
      }
    }
    if (!loc.empty()) {
      cell_ids.push_back(c);
      cell_ents.push_back(ce);
      cell_locs.push_back(loc);
    }
  }
  // entity adjacency and the Fiedler-type ordering
  std::vector<std::vector<int>> adj(ne);
  for (const auto& ce : cell_ents)
    for (int a : ce)
      for (int bb : ce)
        if (a != bb && std::find(adj[a].begin(), adj[a].end(), bb) == adj[a].end()) adj[a].push_back(bb);
  size_t maxdeg = 0;
  for (const auto& l : adj) maxdeg = std::max(maxdeg, l.size());
  const double cshift = 2.0 * (double)maxdeg + 1.0;
  std::vector<double> x(ne), y(ne);
  const double s3 = 1.0 / std::sqrt(3.0);
  for (int a = 0; a < ne; ++a) x[a] = (mid[a][0] + mid[a][1] + mid[a][2]) * s3;
  for (int it = 0; it < 60; ++it) {
    double mean = 0.0;
    for (int a = 0; a < ne; ++a) mean += x[a];
    mean /= ne;
    double nrm = 0.0;
    for (int a = 0; a < ne; ++a) {
      x[a] -= mean;
      nrm += x[a] * x[a];
    }
    if (!(nrm > 0.0)) {
      for (int a = 0; a < ne; ++a) x[a] = a;
      continue;
    }
    nrm = 1.0 / std::sqrt(nrm);
    for (int a = 0; a < ne; ++a) x[a] *= nrm;
    for (int a = 0; a < ne; ++a) {
      double t = (cshift - (double)adj[a].size()) * x[a];
      for (int bb : adj[a]) t += x[bb];
      y[a] = t;
    }
    x.swap(y);
  }
  std::vector<int> eorder(ne);
  for (int a = 0; a < ne; ++a) eorder[a] = a;
  std::stable_sort(eorder.begin(), eorder.end(), [&](int a, int bb) { return x[a] < x[bb]; });
  // new DOF order
  std::vector<int> newpos(np), ent_new_start(ne);
  std::vector<int32_t> dofs_new;
  dofs_new.reserve(np);
  for (int a : eorder) {
    ent_new_start[a] = (int)dofs_new.size();
    for (int q = 0; q < ent_len[a]; ++q) {
      newpos[ent_start[a] + q] = (int)dofs_new.size();
      dofs_new.push_back(pd[ent_start[a] + q]);
    }
  }
  // tile pattern of A_V and its symbolic tile Cholesky
  const int nb = (np + 31) / 32;
  std::vector<char> nz((size_t)nb * nb, 0);
  for (int I = 0; I < nb; ++I) nz[(size_t)I * nb + I] = 1;
  for (const auto& ce : cell_ents)
    for (int a : ce)
      for (int bb : ce) {
        const int r0 = ent_new_start[a] / 32, r1 = (ent_new_start[a] + ent_len[a] - 1) / 32;
        const int c0 = ent_new_start[bb] / 32, c1 = (ent_new_start[bb] + ent_len[bb] - 1) / 32;
        for (int I = r0; I <= r1; ++I)
          for (int J = c0; J <= c1; ++J) nz[(size_t)std::max(I, J) * nb + std::min(I, J)] = 1;
      }
  std::vector<int> col;
  P.col_flops.reserve(nb);
  for (int K = 0; K < nb; ++K) {
    col.clear();
    for (int I = K + 1; I < nb; ++I)
      if (nz[(size_t)I * nb + K]) col.push_back(I);
    P.tile_ops += 1 + (int64_t)col.size() + (int64_t)col.size() * (col.size() + 1) / 2;
    // diagonal factor (n^3/3) + its inverse (n^3/3), panel (triangular, 32*528 FMA per tile),
    // trailing tile products (32^3 FMA each)
    P.col_flops.push_back(2.0 * 32768.0 / 3.0 + 2.0 * 16896.0 * col.size() +
                          65536.0 * (col.size() * (col.size() + 1) / 2));
    for (size_t a = 0; a < col.size(); ++a)
      for (size_t bb = 0; bb <= a; ++bb) nz[(size_t)col[a] * nb + col[bb]] = 1;
  }
  P.meta.assign((size_t)nb * nb, -1);
  int32_t nt = 0;
  std::vector<int32_t> tcol;
  for (int I = 0; I < nb; ++I)
    for (int J = 0; J <= I; ++J)
      if (nz[(size_t)I * nb + J]) {
        P.meta[(size_t)I * nb + J] = nt++;
        tcol.push_back(J);
      }
  P.meta.insert(P.meta.end(), tcol.begin(), tcol.end());
  P.np = np;
  P.nb = nb;
  P.nt = nt;
  P.dofs = std::move(dofs_new);
  for (size_t ci = 0; ci < cell_ids.size(); ++ci) {
    for (const auto& jk : cell_locs[ci]) P.ent.push_back(jk.first | (int32_t)(newpos[jk.second] << 10));
    P.cells.push_back(cell_ids[ci]);
    P.cell_end.push_back((int64_t)P.ent.size());
  }
  return P;
}

// Add a patch plan to the handle: offsets of its factor tiles, inverted diagonal tiles, tile
// map and DOFs, and its cell contributions for the assembly.
void append_patch(riesz_handle& h, const PatchPlan& P, int64_t& foff, int64_t& dioff) {
  const int64_t moff = (int64_t)h.p_meta.size();
  h.p_meta.insert(h.p_meta.end(), P.meta.begin(), P.meta.end());
  h.p_n.push_back(P.np);
  h.p_doff.push_back((int64_t)h.p_dofs.size());
  h.p_foff.push_back(foff);
  h.p_dioff.push_back(dioff);
  h.p_moff.push_back(moff);
  foff += (int64_t)P.nt * 1024;
  dioff += (int64_t)P.nb * 1024;
  h.p_dofs.insert(h.p_dofs.end(), P.dofs.begin(), P.dofs.end());
  const int64_t e0 = (int64_t)h.pb_ent.size();
  h.pb_ent.insert(h.pb_ent.end(), P.ent.begin(), P.ent.end());
  for (size_t ci = 0; ci < P.cells.size(); ++ci) {
    h.pb_cell.push_back(P.cells[ci]);
    h.pb_off.push_back(e0 + P.cell_end[ci]);
  }
  h.pb_ptr.push_back((int64_t)h.pb_cell.size());
  h.tile_ops += P.tile_ops;
  for (double f : P.col_flops) h.chol_flops += f;
}

// Index of the sorted edge (a, b), a < b, in the lexicographic edge list.
int64_t edge_index(const MeshMaps& M, int32_t a, int32_t b) {
  int64_t lo = 0, hi = M.nedges;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    const int32_t* e = &M.edges[mid * 2];
    if (e[0] < a || (e[0] == a && e[1] < b))
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo >= M.nedges || M.edges[lo * 2] != a || M.edges[lo * 2 + 1] != b)
    throw Err(RIESZ_ERR_INTERNAL, "edge not found");
  return lo;
}

// Edge-star patches: per edge E the first `take_e` DOFs of E and the first
// `take_f` DOFs of every face containing E, without fixed Dirichlet DOFs,
// sorted.  All DOFs of both (take_e = 0 edge DOFs of RT_p, all face DOFs) give
// the interface functions supported in the star of E: the PAFW_1 subspaces of
// Eq. (6.24) for H(div).
void plan_edge_stars(riesz_handle& h, int take_e, int take_f) {
  const MeshMaps& M = h.mesh;
  const int ne_d = M.per_entity[1], nf_d = M.per_entity[2];
  std::vector<std::vector<int32_t>> faces_of(M.nedges);
  for (int64_t f = 0; f < M.nfaces; ++f) {
    const int32_t* v = &M.faces[f * 3];
    faces_of[edge_index(M, v[0], v[1])].push_back((int32_t)f);
    faces_of[edge_index(M, v[0], v[2])].push_back((int32_t)f);
    faces_of[edge_index(M, v[1], v[2])].push_back((int32_t)f);
  }
  auto keep = [&](int64_t d) { return h.dir_mask.empty() || !h.dir_mask[d]; };
  h.es_ptr.assign(1, 0);
  h.es_dofs.clear();
  for (int64_t e = 0; e < M.nedges; ++e) {
    std::vector<int32_t> d;
    for (int m = 0; m < take_e; ++m)
      if (keep(M.off[1] + (int64_t)ne_d * e + m)) d.push_back((int32_t)(M.off[1] + (int64_t)ne_d * e + m));
    for (int32_t f : faces_of[e])
      for (int m = 0; m < take_f; ++m)
        if (keep(M.off[2] + (int64_t)nf_d * f + m)) d.push_back((int32_t)(M.off[2] + (int64_t)nf_d * f + m));
    std::sort(d.begin(), d.end());
    h.es_dofs.insert(h.es_dofs.end(), d.begin(), d.end());
    h.es_ptr.push_back((int64_t)h.es_dofs.size());
  }
  h.edge_star = true;
}

// Hiptmair-Toselli decomposition of Eq. (6.19) for H(curl): per edge L the
// Whitney DOF of L and the type-I DOFs of every face containing L (the
// interface DOFs of X^{1,I} on the star of L; inside a face the type-I DOFs
// come first), and the gradient map between CG_p and Ned1_p interface DOFs
// (CG_{p+1} and NedTwo_p for the second kind, whose X^0 is CG_{p+1}):
// the gradient of the CG vertex function v has Whitney coefficient +1 on edges
// ending at v and -1 on edges starting at v; the gradient of the m-th CG edge
// (face) function is the m-th type-II Ned1 function of that edge (face)
// (Eq. (5.3), Lemma 4.3).
void plan_ht(riesz_handle& h) {
  const MeshMaps& M = h.mesh;
  const MeshMaps& Mc = h.kind == 2 ? h.meshpot : h.meshcg;
  const int ne_d = M.per_entity[1], nf_d = M.per_entity[2];
  const int ce = Mc.per_entity[1], cf = Mc.per_entity[2];
  const int nfI = nf_d - cf;
  if (ne_d != ce + 1 || nfI < 0 || Mc.per_entity[0] != 1)
    throw Err(RIESZ_ERR_INTERNAL, "gradient map: unexpected DOF counts");
  plan_edge_stars(h, 1, nfI);
  // G^T rows: CG interface DOF -> (Ned1 DOF, sign)
  const int64_t ncif = Mc.n_interface;
  std::vector<std::vector<std::pair<int32_t, float>>> gt(ncif);
  std::vector<std::vector<std::pair<int32_t, float>>> gg(M.n_interface);
  for (int64_t e = 0; e < M.nedges; ++e) {
    const int32_t a = M.edges[e * 2], b = M.edges[e * 2 + 1];
    const int32_t w = (int32_t)(M.off[1] + (int64_t)ne_d * e);
    gt[Mc.off[0] + a].push_back({w, -1.f});
    gt[Mc.off[0] + b].push_back({w, 1.f});
    gg[w].push_back({(int32_t)(Mc.off[0] + a), -1.f});
    gg[w].push_back({(int32_t)(Mc.off[0] + b), 1.f});
    for (int m = 0; m < ce; ++m) {
      const int32_t nd = w + 1 + m, cd = (int32_t)(Mc.off[1] + (int64_t)ce * e + m);
      gt[cd].push_back({nd, 1.f});
      gg[nd].push_back({cd, 1.f});
    }
  }
  for (int64_t f = 0; f < M.nfaces; ++f)
    for (int m = 0; m < cf; ++m) {
      const int32_t nd = (int32_t)(M.off[2] + (int64_t)nf_d * f + nfI + m), cd = (int32_t)(Mc.off[2] + (int64_t)cf * f + m);
      gt[cd].push_back({nd, 1.f});
      gg[nd].push_back({cd, 1.f});
    }
  auto flatten = [](const std::vector<std::vector<std::pair<int32_t, float>>>& rows, std::vector<int64_t>& ptr,
                    std::vector<int32_t>& idx, std::vector<float>& sgn) {
    ptr.assign(1, 0);
    idx.clear();
    sgn.clear();
    for (const auto& r : rows) {
      for (const auto& q : r) {
        idx.push_back(q.first);
        sgn.push_back(q.second);
      }
      ptr.push_back((int64_t)idx.size());
    }
  };
  flatten(gt, h.gt_ptr, h.gt_idx, h.gt_sgn);
  flatten(gg, h.gg_ptr, h.gg_idx, h.gg_sgn);
  h.ht = true;
}

// Homogeneous Dirichlet conditions on the whole boundary (X_{p,D} with
// Gamma_D the boundary, Eq. (2.8)): a function has zero trace there exactly
// when every DOF of every boundary vertex, edge and face is zero.  Marks those
// DOFs and removes them from the vertex-star patches.
void plan_dirichlet(riesz_handle& h) {
  MeshMaps& M = h.mesh;
  h.dir_mask.assign(M.n_interface, 0);
  std::vector<int> cnt(M.nfaces, 0);
  for (int64_t c = 0; c < M.ncells; ++c)
    for (int f = 0; f < 4; ++f) ++cnt[M.cell_faces[c * 4 + f]];
  auto mark = [&](int k, int64_t ent) {
    const int nd = M.per_entity[k];
    for (int m = 0; m < nd; ++m) h.dir_mask[M.off[k] + (int64_t)nd * ent + m] = 1;
  };
  const uint8_t* vm = h.opts.dirichlet_vertices;  // Gamma_D: the boundary faces with all three vertices flagged
  for (int64_t f = 0; f < M.nfaces; ++f) {
    if (cnt[f] != 1) continue;
    const int32_t* v = &M.faces[f * 3];
    if (vm && !(vm[v[0]] && vm[v[1]] && vm[v[2]])) continue;
    mark(2, f);
    for (int a = 0; a < 3; ++a) mark(0, v[a]);
    mark(1, edge_index(M, v[0], v[1]));
    mark(1, edge_index(M, v[0], v[2]));
    mark(1, edge_index(M, v[1], v[2]));
  }
  std::vector<int64_t> ptr(M.nverts + 1, 0);
  std::vector<int32_t> dofs;
  dofs.reserve(M.patch_dofs.size());
  for (int64_t v = 0; v < M.nverts; ++v) {
    for (int64_t k = M.patch_ptr[v]; k < M.patch_ptr[v + 1]; ++k)
      if (!h.dir_mask[M.patch_dofs[k]]) dofs.push_back(M.patch_dofs[k]);
    ptr[v + 1] = (int64_t)dofs.size();
  }
  M.patch_ptr.swap(ptr);
  M.patch_dofs.swap(dofs);
}

// W^k (Lemma 4.1: the first type-I DOF of each vertex, edge or face carries
// the Whitney form) and the contribution lists of A_0 = R_0 A R_0^T.
// Dense coarse inverse (FP64 Cholesky route, 0.83 N0^3 FP64 flop at setup: 220 ms at 5832 DOFs): up to
// COARSE_DENSE_MAX DOFs for H(curl) and H(div), above that the lowest-order PCG steps; up to
// COARSE_DENSE_MAX_H1 for H1, whose lowest-order vertex stars are single vertices (those steps are
// point-Jacobi PCG and converge slowly); the blocks of the Hodge-Laplace preconditioner (which MINRES needs
// linear) keep the dense inverse up to COARSE_MAX.  An FP32 Gauss-Jordan inverse was
// cheaper to form but its error grows with N0 (measured on RT_1: 2e-3 relative at 1650 DOFs, 6e-3 at
// 4410, where PCG took 217 iterations against 36 with the exact coarse solve and 46 with the PCG steps).
constexpr int COARSE_DENSE_MAX = 2048;
constexpr int COARSE_DENSE_MAX_H1 = 3072;
constexpr int COARSE_MAX = 6144;
// Weight of the additive coarse correction: every W^k function also lies in the
// vertex-star spaces, so the unweighted sum over-corrects (most for H(div)).
constexpr double COARSE_WEIGHT = 0.5;

void plan_coarse(riesz_handle& h, bool hodge_block) {
  const MeshMaps& M = h.mesh;
  const int k = h.space;  // entity dimension of the Whitney DOFs: 0, 1, 2
  const int nd = M.per_entity[k];
  const int64_t nent = k == 0 ? M.nverts : (k == 1 ? M.nedges : M.nfaces);
  h.coarse_on = false;
  if (!h.opts.coarse || nd == 0) return;
  // Dirichlet entities carry no coarse DOF
  std::vector<int32_t> w;
  for (int64_t e = 0; e < nent; ++e) {
    const int64_t gd = M.off[k] + (int64_t)nd * e;
    if (h.dir_mask.empty() || !h.dir_mask[gd]) w.push_back((int32_t)gd);
  }
  if (w.empty()) return;
  const int dense_max = hodge_block ? COARSE_MAX : (k == 0 ? COARSE_DENSE_MAX_H1 : COARSE_DENSE_MAX);
  h.coarse_sparse = h.opts.coarse == 2 || (int64_t)w.size() > dense_max;
  const int N0 = (int)w.size();
  const int nloc = k == 1 ? 6 : 4;
  const int loc0 = k == 0 ? 0 : (k == 1 ? 4 * M.per_entity[0] : 4 * M.per_entity[0] + 6 * M.per_entity[1]);
  h.N0 = N0;
  h.N0p = (N0 + dev::CB - 1) / dev::CB * dev::CB;
  h.c_w.swap(w);
  h.c_idx.assign(M.n_interface, -1);
  for (int e = 0; e < N0; ++e) h.c_idx[h.c_w[e]] = e;
  struct Con {
    int32_t I, J, cell, ab;
  };
  std::vector<Con> con;
  con.reserve((size_t)M.ncells * nloc * nloc);
  for (int64_t c = 0; c < M.ncells; ++c) {
    int32_t loc[6], ce[6];
    for (int t = 0; t < nloc; ++t) {
      loc[t] = loc0 + t * nd;
      const int64_t gd = M.cell_dofs[c * M.nref + loc[t]];
      ce[t] = h.c_idx[gd];
      if (ce[t] < 0 && (h.dir_mask.empty() || !h.dir_mask[gd]))
        throw Err(RIESZ_ERR_INTERNAL, "coarse DOF map inconsistent with the cell DOFs");
    }
    for (int a = 0; a < nloc; ++a)
      for (int b = 0; b < nloc; ++b)
        if (ce[a] >= 0 && ce[b] >= 0) con.push_back({ce[a], ce[b], (int32_t)c, loc[a] | (loc[b] << 16)});
  }
  std::sort(con.begin(), con.end(), [](const Con& x, const Con& y) {
    return x.I != y.I ? x.I < y.I : (x.J != y.J ? x.J < y.J : x.cell < y.cell);
  });
  h.c_ptr.assign(N0 + 1, 0);
  h.c_J.resize(con.size());
  h.c_cell.resize(con.size());
  h.c_ab.resize(con.size());
  for (size_t e = 0; e < con.size(); ++e) {
    ++h.c_ptr[con[e].I + 1];
    h.c_J[e] = con[e].J;
    h.c_cell[e] = con[e].cell;
    h.c_ab[e] = con[e].ab;
  }
  for (int i = 0; i < N0; ++i) h.c_ptr[i + 1] += h.c_ptr[i];
  h.coarse_on = true;
  if (h.coarse_sparse) {  // coarse index -> entity (the DOF of the p = 1 handle)
    h.c_aux.resize(N0);
    for (int j = 0; j < N0; ++j) h.c_aux[j] = (int32_t)((h.c_w[j] - M.off[k]) / nd);
    return;
  }
}

void build_plans(riesz_handle& h) {
  const MeshMaps& M = h.mesh;
  const int n = M.nref;
  const int64_t C = M.ncells;
  h.nif = n - h.ref->ninterior;
  // host check of the cell volumes
  for (int64_t c = 0; c < C; ++c) {
    double X[4][3];
    double emax = 0.0;
    for (int k = 0; k < 4; ++k)
      for (int d = 0; d < 3; ++d) X[k][d] = h.verts[(size_t)M.cells[c * 4 + k] * 3 + d];
    double E[3][3];
    for (int k = 0; k < 3; ++k) {
      double l = 0.0;
      for (int d = 0; d < 3; ++d) {
        E[k][d] = X[k + 1][d] - X[0][d];
        l += E[k][d] * E[k][d];
      }
      emax = std::max(emax, l);
    }
    const double det = E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) -
                       E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
                       E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
    if (!(std::fabs(det) > 1e-12 * std::pow(emax, 1.5)) || !std::isfinite(det))
      throw Err(RIESZ_ERR_BAD_MESH, "degenerate or non-finite cell " + std::to_string(c));
  }
  // interface scatter CSR: DOF d <- (j*C + c) for local interface j
  const int64_t nI = M.n_interface;
  h.sc_ptr.assign(nI + 1, 0);
  for (int64_t c = 0; c < C; ++c)
    for (int j = 0; j < h.nif; ++j) h.sc_ptr[M.cell_dofs[c * n + j] + 1]++;
  for (int64_t d = 0; d < nI; ++d) h.sc_ptr[d + 1] += h.sc_ptr[d];
  h.sc_pos.assign(h.sc_ptr[nI], 0);
  {
    std::vector<int64_t> cur(h.sc_ptr.begin(), h.sc_ptr.end() - 1);
    for (int64_t c = 0; c < C; ++c)  // cell order fixes the summation order
      for (int j = 0; j < h.nif; ++j) h.sc_pos[cur[M.cell_dofs[c * n + j]]++] = (int32_t)((int64_t)j * C + c);
  }
  // patches, largest first
  const int64_t nv = M.nverts;
  std::vector<int64_t> order(nv);
  for (int64_t v = 0; v < nv; ++v) order[v] = v;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return (M.patch_ptr[a + 1] - M.patch_ptr[a]) > (M.patch_ptr[b + 1] - M.patch_ptr[b]);
  });
  h.p_n.clear();
  h.p_doff.clear();
  h.p_foff.clear();
  h.p_dioff.clear();
  h.p_moff.clear();
  h.p_meta.clear();
  h.p_dofs.clear();
  h.pb_ptr.assign(1, 0);
  h.pb_off.assign(1, 0);
  h.pb_cell.clear();
  h.pb_ent.clear();
  h.tile_ops = 0;
  h.chol_flops = 0.0;
  int64_t foff = 0, dioff = 0;
  // the patches in launch order (largest first): edges for edge stars, vertices for vertex stars
  std::vector<int64_t> ids;
  if (h.edge_star) {  // edge stars instead of vertex stars
    std::vector<int64_t> eorder(h.es_ptr.size() - 1);
    for (size_t e = 0; e < eorder.size(); ++e) eorder[e] = (int64_t)e;
    std::stable_sort(eorder.begin(), eorder.end(), [&](int64_t a, int64_t b) {
      return (h.es_ptr[a + 1] - h.es_ptr[a]) > (h.es_ptr[b + 1] - h.es_ptr[b]);
    });
    for (int64_t e : eorder) {
      const int64_t np = h.es_ptr[e + 1] - h.es_ptr[e];
      if (np == 0) continue;
      if (np > 32 * dev::MAXNB) throw Err(RIESZ_ERR_INVALID_ARG, "patch larger than 4096 DOFs");
      ids.push_back(e);
    }
  } else if (!h.apply_only) {
    for (int64_t v : order) {
      const int64_t np = M.patch_ptr[v + 1] - M.patch_ptr[v];
      if (np == 0) continue;
      if (np > 32 * dev::MAXNB) throw Err(RIESZ_ERR_INVALID_ARG, "patch larger than 4096 DOFs");
      ids.push_back(v);
    }
  }
  auto plan_of = [&](int64_t id) {
    if (h.edge_star) {
      const int64_t e = id;
      const int np = (int)(h.es_ptr[e + 1] - h.es_ptr[e]);
      const int32_t a = M.edges[e * 2], b = M.edges[e * 2 + 1];
      std::vector<int32_t> cells;  // cells containing both endpoints
      for (int64_t k = M.star_ptr[a]; k < M.star_ptr[a + 1]; ++k) {
        const int32_t c = M.star_cells[k];
        for (int q = 0; q < 4; ++q)
          if (M.cells[(int64_t)c * 4 + q] == b) {
            cells.push_back(c);
            break;
          }
      }
      double center[3];
      for (int q = 0; q < 3; ++q) center[q] = 0.5 * (h.verts[(size_t)a * 3 + q] + h.verts[(size_t)b * 3 + q]);
      return plan_patch(h, &h.es_dofs[h.es_ptr[e]], np, cells.data(), (int64_t)cells.size(), center);
    }
    const int64_t v = id, b = M.patch_ptr[v];
    const int np = (int)(M.patch_ptr[v + 1] - b);
    return plan_patch(h, &M.patch_dofs[b], np, &M.star_cells[M.star_ptr[v]], M.star_ptr[v + 1] - M.star_ptr[v],
                      &h.verts[(size_t)v * 3]);
  };
  // plans of a chunk of patches on the host threads, then appended in launch order: the same handle
  // as planning them one after the other, with bounded memory for the plans in flight
  constexpr int64_t CHUNK = 4096;
  std::vector<PatchPlan> plans;
  for (int64_t c0 = 0; c0 < (int64_t)ids.size(); c0 += CHUNK) {
    const int cn = (int)std::min<int64_t>(CHUNK, (int64_t)ids.size() - c0);
    plans.assign(cn, PatchPlan());
    parallel_for(cn, [&](int i) { plans[i] = plan_of(ids[c0 + i]); });
    for (const PatchPlan& P : plans) append_patch(h, P, foff, dioff);
  }
  h.factor_entries = foff;
  h.dinv_entries = dioff;
  // interface DOF -> positions in zpatch (patch launch order fixes the sum order)
  h.pz_ptr.assign(nI + 1, 0);
  for (int32_t d : h.p_dofs) h.pz_ptr[d + 1]++;
  for (int64_t d = 0; d < nI; ++d) h.pz_ptr[d + 1] += h.pz_ptr[d];
  h.pz_pos.assign(h.pz_ptr[nI], 0);
  {
    std::vector<int64_t> cur(h.pz_ptr.begin(), h.pz_ptr.end() - 1);
    for (size_t k = 0; k < h.p_dofs.size(); ++k) h.pz_pos[cur[h.p_dofs[k]]++] = (int32_t)k;
  }
}

std::vector<int32_t> transpose_dofs(const std::vector<int32_t>& cd, int64_t C, int n) {
  std::vector<int32_t> t((size_t)C * n);
  for (int64_t c = 0; c < C; ++c)
    for (int j = 0; j < n; ++j) t[(size_t)j * C + c] = cd[(size_t)c * n + j];
  return t;
}

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
// Blocks of 256 threads for the search-direction update: two per SM on large vectors, about four
// entries per thread on short ones.
inline unsigned update_blocks(int64_t n) { return (unsigned)std::min<int64_t>(296, std::max<int64_t>(1, (n + 1023) / 1024)); }

// ---- operator pieces ------------------------------------------------------
// y = A x for nrhs right-hand sides; fp32 selects the FP32 copy of the element
// matrices (inner applies of the mixed-precision solver).
// With scal non-null the interface gather is fused with the PCG reduction (x, y) -> scalar op
// `op` (k_gather_iface_dot: the same values as the gather followed by dot()).
void op_apply(riesz_handle& h, const double* x, double* y, int nrhs, cudaStream_t s, int prec = RIESZ_PREC_FP64,
              double* scal = nullptr, int op = 0) {
  const int n = h.mesh.nref;
  const int64_t C = h.C(), N = h.N();
  const bool fp32 = prec == RIESZ_PREC_FP32;
  if (prec == RIESZ_PREC_BF16X3) {
    const int RT = nrhs >= 8 ? 8 : (nrhs >= 4 ? 4 : (nrhs >= 2 ? 2 : 1));
    const int cells = dev::TC_ROWS / RT;
    dim3 grid((unsigned)((C + cells - 1) / cells), (unsigned)((nrhs + RT - 1) / RT), (unsigned)dev::tc_parts(h.tc_np));
    launch(h, RIESZ_K_APPLY_TC, s, [&] {
      const int npc = dev::tc_part_cols(h.tc_np, 0);
      const int ns = dev::tc_stages(npc);
      const size_t sm = dev::tc_smem_bytes(npc, ns);
      if (h.ref->Q == 12)
        dev::k_apply_tc<12><<<grid, dev::TC_NT, sm, s>>>(C, n, h.nif, h.tc_np, h.tc_kc, RT, ns, h.d_Btc.p, h.d_g.p,
                                                         h.d_cdofs.p, x, y, h.d_Ycell.p, nrhs, N, h.dmask(),
                                                         h.d_flags.p + 2);
      else
        dev::k_apply_tc<7><<<grid, dev::TC_NT, sm, s>>>(C, n, h.nif, h.tc_np, h.tc_kc, RT, ns, h.d_Btc.p, h.d_g.p,
                                                        h.d_cdofs.p, x, y, h.d_Ycell.p, nrhs, N, h.dmask(),
                                                        h.d_flags.p + 2);
    });
  } else if (h.opts.apply_mode == RIESZ_APPLY_ELEMENT && n <= dev::SMALL_ELEM) {
    const unsigned grid = nblk((int64_t)nrhs * C, 256);
    if (fp32)
      launch(h, RIESZ_K_APPLY32, s, [&] {
        dev::k_apply_elem_small<float, dev::SMALL_ELEM><<<grid, 256, 0, s>>>(C, n, h.nif, h.d_Ae32.p, h.d_cdofs.p, x,
                                                                           y, h.d_Ycell.p, nrhs, N, h.dmask());
      });
    else
      launch(h, RIESZ_K_APPLY, s, [&] {
        dev::k_apply_elem_small<double, dev::SMALL_ELEM><<<grid, 256, 0, s>>>(C, n, h.nif, h.d_Ae.p, h.d_cdofs.p, x,
                                                                            y, h.d_Ycell.p, nrhs, N, h.dmask());
      });
  } else if (h.opts.apply_mode == RIESZ_APPLY_ELEMENT) {
    const int rows = (n % 2 == 0) ? n / 2 : n;
    // the rows loop strides by the block size; the multi-RHS variants hold up to 92 registers per
    // thread, so their blocks stay at 512 threads (odd n_ref, e.g. RT_10: 715 rows)
    const int nt = std::min(nrhs == 1 ? 1024 : 512, (rows + 31) / 32 * 32);
    if (fp32) {
      const size_t sm = (size_t)n * nrhs * sizeof(float);
      launch(h, RIESZ_K_APPLY32, s, [&] {
        if (nrhs == 1)
          dev::k_apply_elem<float, 1><<<(unsigned)C, nt, sm, s>>>(C, n, h.nif, h.d_Ae32.p, h.d_cdofs.p, x, y,
                                                                  h.d_Ycell.p, nrhs, N, h.dmask());
        else
          dev::k_apply_elem<float, 8><<<(unsigned)C, nt, sm, s>>>(C, n, h.nif, h.d_Ae32.p, h.d_cdofs.p, x, y,
                                                                  h.d_Ycell.p, nrhs, N, h.dmask());
      });
    } else {
      const size_t sm = (size_t)n * nrhs * sizeof(double);
      launch(h, RIESZ_K_APPLY, s, [&] {
        if (nrhs == 1)
          dev::k_apply_elem<double, 1><<<(unsigned)C, nt, sm, s>>>(C, n, h.nif, h.d_Ae.p, h.d_cdofs.p, x, y,
                                                                   h.d_Ycell.p, nrhs, N, h.dmask());
        else
          dev::k_apply_elem<double, 8><<<(unsigned)C, nt, sm, s>>>(C, n, h.nif, h.d_Ae.p, h.d_cdofs.p, x, y,
                                                                   h.d_Ycell.p, nrhs, N, h.dmask());
      });
    }
  } else {
    const size_t sm = ((size_t)n + h.ref->Q) * dev::TC * sizeof(double);
    dim3 grid(nblk(C, dev::TC), nrhs);
    launch(h, RIESZ_K_APPLY, s, [&] {
      dev::k_apply_mf<<<grid, dev::NT, sm, s>>>(C, n, h.nif, h.ref->Q, h.d_R.p, h.d_g.p, h.d_cdofs.p, x, y, h.d_Ycell.p,
                                               N, h.dmask());
    });
  }
  const int64_t nI = h.mesh.n_interface;
  if (scal) {
    launch(h, RIESZ_K_GATHER, s, [&] {
      dev::k_gather_iface_dot<<<dim3(nrhs, dev::red_blocks(N)), dev::NT, 0, s>>>(
          nI, h.d_sc_ptr.p, h.d_sc_pos.p, h.d_Ycell.p, (int64_t)h.nif * C, y, N, h.dmask(), x, h.d_part.p,
          h.d_ticket.p, op, scal);
    });
    return;
  }
  launch(h, RIESZ_K_GATHER, s, [&] {
    dev::k_gather_iface<<<nblk(nI, 256), 256, 0, s>>>(nI, h.d_sc_ptr.p, h.d_sc_pos.p, h.d_Ycell.p, (int64_t)h.nif * C, y,
                                                     N, nrhs, h.dmask(), x);
  });
}

// Ring slots of the bulk-copy sweep kernel (tiles of 4 KB in FP32, 8 KB in FP64).
constexpr int SWEEP_SLOTS_F32 = 8, SWEEP_SLOTS_F64 = 8;
template <typename T>
size_t sweep_smem(int slots, int nbmax) {
  return (size_t)slots * 1024 * sizeof(T) + (size_t)nbmax * 32 * sizeof(T);
}
size_t sweep8_smem(int nbmax) {  // ring + patch vectors of 8 right-hand sides (FP32)
  return (size_t)SWEEP_SLOTS_F32 * 1024 * sizeof(float) + (size_t)nbmax * 32 * 8 * sizeof(float);
}

// Patch sweeps for nrhs right-hand sides into zpatch.
void op_patch_solves(riesz_handle& h, const double* r, int nrhs, cudaStream_t s) {
  const int64_t N = h.N();
  const int npatch = (int)h.p_n.size();
  if (!npatch) return;
  const int nbmax = (h.p_n[0] + 31) / 32;
  const int64_t zstride = (int64_t)h.p_dofs.size();
  const bool f32 = h.opts.precond_precision == RIESZ_PREC_FP32;
  if (nbmax <= dev::SMALL_NB) {  // small patches: one warp per patch
    const unsigned grid = (unsigned)((npatch + dev::SMALL_WARPS - 1) / dev::SMALL_WARPS);
    for (int r0 = 0; r0 < nrhs; r0 += 8) {
      const int nr = std::min(8, nrhs - r0);
      launch(h, RIESZ_K_PATCH_SOLVE, s, [&] {
        if (f32)
          dev::k_patch_solve_small<float><<<grid, dev::SMALL_WARPS * 32,
                                            dev::SMALL_WARPS * dev::small_warp_smem<float>(), s>>>(
              npatch, h.d_pn.p, h.d_pdoff.p, h.d_pfoff.p, h.d_pdioff.p, h.d_pmoff.p, h.d_meta.p, h.d_pdofs.p,
              h.d_L32.p, h.d_D32.p, r + (int64_t)r0 * N, h.d_zpatch.p + (int64_t)r0 * zstride, N, zstride, nr);
        else
          dev::k_patch_solve_small<double><<<grid, dev::SMALL_WARPS * 32,
                                             dev::SMALL_WARPS * dev::small_warp_smem<double>(), s>>>(
              npatch, h.d_pn.p, h.d_pdoff.p, h.d_pfoff.p, h.d_pdioff.p, h.d_pmoff.p, h.d_meta.p, h.d_pdofs.p,
              h.d_L64.p, h.d_D64.p, r + (int64_t)r0 * N, h.d_zpatch.p + (int64_t)r0 * zstride, N, zstride, nr);
      });
    }
    return;
  }
  if (nrhs == 1) {  // factor tiles streamed through shared memory by bulk copies
    if (f32)
      launch(h, RIESZ_K_PATCH_SOLVE, s, [&] {
        dev::k_patch_sweep<float, SWEEP_SLOTS_F32><<<npatch, dev::SWEEP_NT, sweep_smem<float>(SWEEP_SLOTS_F32, nbmax), s>>>(
            h.d_pn.p, h.d_pdoff.p, h.d_pfoff.p, h.d_pdioff.p, h.d_pmoff.p, h.d_meta.p, h.d_pdofs.p, h.d_L32.p,
            h.d_D32.p, r, h.d_zpatch.p, h.d_flags.p);
      });
    else
      launch(h, RIESZ_K_PATCH_SOLVE, s, [&] {
        dev::k_patch_sweep<double, SWEEP_SLOTS_F64><<<npatch, dev::SWEEP_NT, sweep_smem<double>(SWEEP_SLOTS_F64, nbmax), s>>>(
            h.d_pn.p, h.d_pdoff.p, h.d_pfoff.p, h.d_pdioff.p, h.d_pmoff.p, h.d_meta.p, h.d_pdofs.p, h.d_L64.p,
            h.d_D64.p, r, h.d_zpatch.p, h.d_flags.p);
      });
    return;
  }
  if (f32 && nbmax <= dev::WARP_NB && h.sweep_shape > 0) {  // patches of at most 8 tiles: one warp per patch
    const int wpb = h.sweep_shape;
    const unsigned grid = (unsigned)((npatch + wpb - 1) / wpb);
    for (int r0 = 0; r0 < nrhs; r0 += 8) {
      const int nr = std::min(8, nrhs - r0);
      launch(h, RIESZ_K_PATCH_SOLVE, s, [&] {
        dev::k_patch_sweep_warp8<<<grid, wpb * 32, wpb * dev::warp_sweep_smem(), s>>>(
            npatch, h.d_pn.p, h.d_pdoff.p, h.d_pfoff.p, h.d_pdioff.p, h.d_pmoff.p, h.d_meta.p, h.d_pdofs.p,
            h.d_L32.p, h.d_D32.p, h.d_L32T.p, h.d_D32T.p, r + (int64_t)r0 * N, h.d_zpatch.p + (int64_t)r0 * zstride,
            N, zstride, nr);
      });
    }
    return;
  }
  if (f32) {  // up to 8 right-hand sides per launch on the bulk-copy pipeline
    for (int r0 = 0; r0 < nrhs; r0 += 8) {
      const int nr = std::min(8, nrhs - r0);
      launch(h, RIESZ_K_PATCH_SOLVE, s, [&] {
        dev::k_patch_sweep8<SWEEP_SLOTS_F32><<<npatch, dev::SWEEP_NT, sweep8_smem(nbmax), s>>>(
            h.d_pn.p, h.d_pdoff.p, h.d_pfoff.p, h.d_pdioff.p, h.d_pmoff.p, h.d_meta.p, h.d_pdofs.p, h.d_L32.p,
            h.d_D32.p, h.d_L32T.p, h.d_D32T.p, r + (int64_t)r0 * N, h.d_zpatch.p + (int64_t)r0 * zstride, N, zstride,
            nr, h.d_flags.p);
      });
    }
    return;
  }
  for (int r0 = 0; r0 < nrhs; r0 += h.multi_group) {
    const int nr = std::min(h.multi_group, nrhs - r0);
    const double* rr = r + (int64_t)r0 * N;
    double* zp = h.d_zpatch.p + (int64_t)r0 * zstride;
    launch(h, RIESZ_K_PATCH_SOLVE, s, [&] {
      dev::k_patch_solve_multi<double><<<npatch, dev::NT, (size_t)nr * nbmax * 32 * sizeof(double), s>>>(
          h.d_pn.p, h.d_pdoff.p, h.d_pfoff.p, h.d_pdioff.p, h.d_pmoff.p, h.d_meta.p, h.d_pdofs.p, h.d_L64.p,
          h.d_D64.p, rr, zp, N, zstride, nr);
    });
  }
}

// Coarse corrections zc = A_0^{-1} R_0 r (W^k), when the handle has a coarse space.
template <typename T>
void op_coarse_t(riesz_handle& h, const double* r, int nrhs, cudaStream_t s, T* A0, T* r0, double w) {
  const int64_t N = h.N();
  const unsigned grid = (unsigned)std::min<int64_t>((h.N0 + 7) / 8, 608);
  launch(h, RIESZ_K_COARSE_APPLY, s, [&] {
    dev::k_coarse_gather<T><<<nblk((int64_t)nrhs * h.N0p, 256), 256, 0, s>>>(h.N0, h.N0p, h.d_cw.p, r, N, nrhs, r0);
  });
  for (int k0 = 0; k0 < nrhs; k0 += h.coarse_group) {
    const int nr = std::min(h.coarse_group, nrhs - k0);
    launch(h, RIESZ_K_COARSE_APPLY, s, [&] {
      dev::k_coarse_apply<T><<<grid, 256, (size_t)nr * h.N0p * sizeof(T), s>>>(
          h.N0, h.N0p, A0, r0 + (int64_t)k0 * h.N0p, nr, w, h.d_zc.p + (int64_t)k0 * h.N0);
    });
  }
}

void iter_tail(riesz_handle& h, double* x, int nrhs, cudaStream_t s);
void iter_head(riesz_handle& h, int nrhs, cudaStream_t s);
void op_precond_dot(riesz_handle& h, const double* r, double* z, const double* zold, int op, double* scal, int nrhs,
                    cudaStream_t s);
// Sparse route: zc = w * (opts.coarse_its PCG steps from zero on the p = 1 handle, its vertex-star
// patches as the preconditioner), all on the device with the PCG kernels of the main loop (device-side
// scalars, no host round trip), so it is captured into the loop graphs like any other step.
bool use_flex(const riesz_handle& h);

void op_coarse_sparse(riesz_handle& h, const double* r, int nrhs, cudaStream_t s, double w) {
  riesz_handle& a = *h.caux;
  const int64_t N = h.N(), Na = a.N();
  const size_t vb = (size_t)nrhs * Na * sizeof(double);
  CK(cudaMemsetAsync(a.d_r.p, 0, vb, s));
  CK(cudaMemsetAsync(a.d_xw.p, 0, vb, s));
  CK(cudaMemsetAsync(a.d_scal.p, 0, (size_t)nrhs * dev::SCAL_STRIDE * sizeof(double), s));
  launch(h, RIESZ_K_COARSE_APPLY, s, [&] {
    dev::k_coarse_to_aux<<<nblk((int64_t)nrhs * h.N0, 256), 256, 0, s>>>(h.N0, h.d_cw.p, h.d_caux.p, r, N, nrhs,
                                                                         a.d_r.p, Na);
  });
  // z = P r, p = z (and zold = z for the flexible step), (r, z): every application starts from r alone
  op_precond_dot(a, a.d_r.p, a.d_z.p, nullptr, 5, a.d_scal.p, nrhs, s);
  CK(cudaMemcpyAsync(a.d_p.p, a.d_z.p, vb, cudaMemcpyDeviceToDevice, s));
  if (use_flex(a)) CK(cudaMemcpyAsync(a.d_zold.p, a.d_z.p, vb, cudaMemcpyDeviceToDevice, s));
  for (int k = 0; k < h.opts.coarse_its; ++k) {
    if (k > 0) iter_head(a, nrhs, s);
    iter_tail(a, a.d_xw.p, nrhs, s);
  }
  launch(h, RIESZ_K_COARSE_APPLY, s, [&] {
    dev::k_coarse_from_aux<<<nblk((int64_t)nrhs * h.N0, 256), 256, 0, s>>>(h.N0, h.d_caux.p, a.d_xw.p, Na, nrhs, w,
                                                                           h.d_zc.p);
  });
}

// zc = w A_0^{-1} R_0 r (dense inverse, or the sparse CG's approximation); the additive form uses
// w = COARSE_WEIGHT.
void op_coarse(riesz_handle& h, const double* r, int nrhs, cudaStream_t s, double w = COARSE_WEIGHT) {
  if (!h.coarse_on) return;
  if (h.coarse_sparse)
    op_coarse_sparse(h, r, nrhs, s, w);
  else
    op_coarse_t<double>(h, r, nrhs, s, h.d_X0d.p, h.d_r0d.p, w);
}

// The coarse correction reads only r: it runs on the side stream beside the
// patch sweeps and joins before the gather (a fork/join when captured).
void coarse_fork(riesz_handle& h, const double* r, int nrhs, cudaStream_t s) {
  if (!h.coarse_on) return;
  CK(cudaEventRecord(h.ev_pfork, s));
  CK(cudaStreamWaitEvent(h.side_stream, h.ev_pfork, 0));
  op_coarse(h, r, nrhs, h.side_stream);
  CK(cudaEventRecord(h.ev_pjoin, h.side_stream));
}
void coarse_join(riesz_handle& h, cudaStream_t s) {
  if (h.coarse_on) CK(cudaStreamWaitEvent(s, h.ev_pjoin, 0));
}

// Gradient part of the Hiptmair-Toselli preconditioner: zg = G sum_J R_J^T
// K_J^{-1} R_J G^T r with the potential problems K_J factored in the CG handle.
void ht_potential(riesz_handle& h, const double* r, int nrhs, cudaStream_t s) {
  if (!h.ht) return;
  riesz_handle& a = *h.aux;
  const int64_t ncif = a.mesh.n_interface, nif = h.mesh.n_interface;
  launch(h, RIESZ_K_HT, s, [&] {
    dev::k_ht_map<<<nblk(ncif, 256), 256, 0, s>>>(ncif, h.d_gt_ptr.p, h.d_gt_idx.p, h.d_gt_sgn.p, r, h.N(), a.d_r.p,
                                                 a.N(), nrhs);
  });
  op_patch_solves(a, a.d_r.p, nrhs, s);
  launch(h, RIESZ_K_HT, s, [&] {
    dev::k_ht_gather<<<nblk(ncif, 256), 256, 0, s>>>(ncif, a.d_pz_ptr.p, a.d_pz_pos.p, a.d_zpatch.p,
                                                    (int64_t)a.p_dofs.size(), h.d_zcg.p, ncif, nrhs);
  });
  launch(h, RIESZ_K_HT, s, [&] {
    dev::k_ht_map<<<nblk(nif, 256), 256, 0, s>>>(nif, h.d_gg_ptr.p, h.d_gg_idx.p, h.d_gg_sgn.p, h.d_zcg.p, ncif,
                                                h.d_zg.p, nif, nrhs);
  });
}

// The potential step reads only r: it runs on its own stream beside the
// edge-star sweeps and the coarse correction and joins before the gather.
void ht_fork(riesz_handle& h, const double* r, int nrhs, cudaStream_t s) {
  if (!h.ht) return;
  CK(cudaEventRecord(h.ev_hfork, s));
  CK(cudaStreamWaitEvent(h.ht_stream, h.ev_hfork, 0));
  ht_potential(h, r, nrhs, h.ht_stream);
  CK(cudaEventRecord(h.ev_hjoin, h.ht_stream));
}
void ht_join(riesz_handle& h, cudaStream_t s) {
  if (h.ht) CK(cudaStreamWaitEvent(s, h.ev_hjoin, 0));
}

// The hybrid form (Section 7.1, Eq. (7.2)): the subspace corrections applied one after the other,
// X_1, X_2, X_3, X_2, X_1 (X_3 = W^k only with the coarse space, X_1 only with interior DOFs), each
// divided by its weight rho_m, the residual updated by an operator product after every step but the
// last.  The products use the FP32 element matrices when the patch sweeps are FP32.
bool hyb_fp32(const riesz_handle& h);
int sweep_prec(const riesz_handle& h);
void hybrid_sweep(const riesz_handle& h, std::vector<int>& steps) {
  steps.clear();
  const bool interior = h.mesh.n_interior > 0;
  if (interior) steps.push_back(1);
  steps.push_back(2);
  if (h.coarse_on) {
    steps.push_back(3);
    steps.push_back(2);
  }
  if (interior) steps.push_back(1);
}

void op_precond_hybrid(riesz_handle& h, const double* r, double* z, int nrhs, cudaStream_t s) {
  const int64_t N = h.N(), nI = h.mesh.n_interface;
  std::vector<int> steps;
  hybrid_sweep(h, steps);
  const int sp = sweep_prec(h);
  const double* res = r;
  double* c = h.d_hc.p;
  for (size_t i = 0; i < steps.size(); ++i) {
    const int m = steps[i];
    const int first = i == 0 ? 1 : 0;
    if (m == 1) {
      launch(h, RIESZ_K_PRECOND_GATHER, s, [&] {
        dev::k_hyb_interior<<<nblk(N, 256), 256, 0, s>>>(N, nI, h.d_dinv.p, res, 1.0 / h.rho[1], c, z, nrhs, first);
      });
    } else if (m == 2) {
      ht_fork(h, res, nrhs, s);
      op_patch_solves(h, res, nrhs, s);
      ht_join(h, s);
      launch(h, RIESZ_K_PRECOND_GATHER, s, [&] {
        dev::k_hyb_interface<<<nblk(N, 256), 256, 0, s>>>(N, nI, h.d_pz_ptr.p, h.d_pz_pos.p, h.d_zpatch.p,
                                                         (int64_t)h.p_dofs.size(), h.ht ? h.d_zg.p : nullptr,
                                                         h.dmask(), res, 1.0 / h.rho[2], c, z, nrhs, first);
      });
    } else {
      op_coarse(h, res, nrhs, s, 1.0);
      launch(h, RIESZ_K_PRECOND_GATHER, s, [&] {
        dev::k_hyb_coarse<<<nblk(N, 256), 256, 0, s>>>(N, nI, h.d_cidx.p, h.d_zc.p, h.N0, 1.0 / h.rho[3], c, z,
                                                      nrhs);
      });
    }
    if (i + 1 < steps.size()) {
      op_apply(h, c, h.d_hAc.p, nrhs, s, sp);
      launch(h, RIESZ_K_UPDATE, s, [&] {
        dev::k_hyb_residual<<<1184, 256, 0, s>>>((int64_t)nrhs * N, res, h.d_hAc.p, h.d_hres.p);
      });
      res = h.d_hres.p;
    }
  }
}

void op_precond(riesz_handle& h, const double* r, double* z, int nrhs, cudaStream_t s) {
  const int64_t N = h.N();
  if (h.opts.form == RIESZ_FORM_HYBRID) {
    op_precond_hybrid(h, r, z, nrhs, s);
    return;
  }
  ht_fork(h, r, nrhs, s);
  coarse_fork(h, r, nrhs, s);
  op_patch_solves(h, r, nrhs, s);
  coarse_join(h, s);
  ht_join(h, s);
  launch(h, RIESZ_K_PRECOND_GATHER, s, [&] {
    dev::k_precond_gather<<<nblk(N, 256), 256, 0, s>>>(N, h.mesh.n_interface, h.d_pz_ptr.p, h.d_pz_pos.p, h.d_zpatch.p,
                                                      (int64_t)h.p_dofs.size(), h.d_dinv.p, r, z, nrhs,
                                                      h.coarse_on ? h.d_cidx.p : nullptr, h.d_zc.p, h.N0, h.dmask(),
                                                      h.ht ? h.d_zg.p : nullptr);
  });
}

// z = P^{-1} r followed by (r, z) [and (r, zold)] -> scalar op, per right-hand side.
void dot(riesz_handle& h, const double* a, const double* b, const double* c, int op, double* scal, int nrhs,
         cudaStream_t s);
void op_precond_dot(riesz_handle& h, const double* r, double* z, const double* zold, int op, double* scal, int nrhs,
                    cudaStream_t s) {
  const int64_t N = h.N();
  if (h.opts.form == RIESZ_FORM_HYBRID) {
    op_precond_hybrid(h, r, z, nrhs, s);
    dot(h, r, z, zold, op, scal, nrhs, s);
    return;
  }
  ht_fork(h, r, nrhs, s);
  coarse_fork(h, r, nrhs, s);
  op_patch_solves(h, r, nrhs, s);
  coarse_join(h, s);
  ht_join(h, s);
  launch(h, RIESZ_K_PRECOND_GATHER, s, [&] {
    dev::k_precond_gather_dot<<<dim3(nrhs, dev::red_blocks(h.N())), dev::NT, 0, s>>>(
        N, h.mesh.n_interface, h.d_pz_ptr.p, h.d_pz_pos.p, h.d_zpatch.p, h.d_dinv.p, r, z, zold, h.d_part.p,
        h.d_ticket.p, op, scal, (int64_t)h.p_dofs.size(), h.coarse_on ? h.d_cidx.p : nullptr, h.d_zc.p, h.N0,
        h.dmask(), h.ht ? h.d_zg.p : nullptr);
  });
}

void dot(riesz_handle& h, const double* a, const double* b, const double* c, int op, double* scal, int nrhs,
         cudaStream_t s) {
  launch(h, RIESZ_K_DOT, s, [&] {
    dev::k_dot2<<<dim3(dev::red_blocks(h.N()), nrhs), dev::NT, 0, s>>>(h.N(), a, b, c, h.d_part.p, h.d_ticket.p, op, scal);
  });
}

void read_scal(riesz_handle& h, const double* scal, int nrhs, cudaStream_t s) {
  CK(cudaMemcpyAsync(h.h_scal, scal, (size_t)nrhs * dev::SCAL_STRIDE * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
}

// The FP32 copy of the element matrices serves the search-direction products (apply_precision FP32)
// and the residual updates inside the hybrid sweep (precond_precision FP32).
bool hyb_fp32(const riesz_handle& h) {
  return h.opts.form == RIESZ_FORM_HYBRID && h.opts.precond_precision == RIESZ_PREC_FP32 &&
         h.opts.apply_mode == RIESZ_APPLY_ELEMENT;
}

// Precision of the search-direction products inside riesz_solve: FP64, the FP32 element matrices, or
// the BF16x3 tensor-core contraction (matrix-free).
int inner_prec(const riesz_handle& h) {
  if (h.opts.apply_precision == RIESZ_PREC_BF16X3) return RIESZ_PREC_BF16X3;
  if (h.opts.apply_precision == RIESZ_PREC_FP32 && h.opts.apply_mode == RIESZ_APPLY_ELEMENT) return RIESZ_PREC_FP32;
  return RIESZ_PREC_FP64;
}
bool use_a32(const riesz_handle& h) { return inner_prec(h) != RIESZ_PREC_FP64; }
// Residual replacement (reliable updates) once (r, r) has fallen by this factor since the last true
// residual: four digits of the residual norm with FP32 products, two with BF16x3 products (their
// ~1e-5 relative error would otherwise build up a larger gap between the recursive and true residuals).
double reliable_gain(const riesz_handle& h) {
  const int ip = inner_prec(h);
  if (ip == RIESZ_PREC_FP64) return 0.0;
  const int d = h.opts.replace_digits > 0 ? h.opts.replace_digits : (ip == RIESZ_PREC_BF16X3 ? 2 : 4);
  return std::pow(10.0, -2.0 * d);  // (r, r) falls by the square of the norm's factor
}
// Precision of the residual updates inside the hybrid sweep.
int sweep_prec(const riesz_handle& h) {
  if (h.opts.apply_precision == RIESZ_PREC_BF16X3) return RIESZ_PREC_BF16X3;
  return hyb_fp32(h) ? RIESZ_PREC_FP32 : RIESZ_PREC_FP64;
}
bool needs_ae32(const riesz_handle& h) {
  return inner_prec(h) == RIESZ_PREC_FP32 || (h.opts.form == RIESZ_FORM_HYBRID && sweep_prec(h) == RIESZ_PREC_FP32);
}
bool needs_tc(const riesz_handle& h) { return h.opts.apply_precision == RIESZ_PREC_BF16X3; }
// Flexible (Polak-Ribiere) beta whenever an FP32 piece enters the preconditioner
// or the search-direction product.
bool use_flex(const riesz_handle& h) {
  return h.opts.precond_precision == RIESZ_PREC_FP32 || use_a32(h) || h.coarse_on;
}

// Weights of the hybrid form (Section 7.1, Eq. (7.3)): rho_m = (lambda_min + 3 lambda_max) / 4 of the
// generalized eigenproblem a(u, v) = lambda a~_m(u, v) on X_m, the extremes estimated by `iters` steps
// of CG on X_m preconditioned by the subspace solver (the Lanczos tridiagonal from the CG coefficients,
// its eigenvalues by Jacobi rotations), from a fixed pseudo-random start vector.  X_1 (interior,
// point-Jacobi) and X_2 (interface, the patch solves); the W^k solve is exact (dense inverse) or
// a few PCG steps on the lowest-order problem (sparse route), so rho_3 = 1.
uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

double lanczos_weight(riesz_handle& h, int m, int iters, cudaStream_t s) {
  const int64_t N = h.N(), nI = h.mesh.n_interface;
  double *r = h.d_r.p, *z = h.d_z.p, *p = h.d_p.p, *Ap = h.d_Ap.p;
  std::vector<double> r0(N);
  uint64_t st = 0x5eed0000ull + (uint64_t)m;
  for (int64_t i = 0; i < N; ++i) r0[i] = (double)(splitmix64(st) >> 11) * 0x1.0p-52 - 1.0;
  CK(cudaMemcpyAsync(r, r0.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
  const int keep = m == 1 ? 2 : 1;
  auto restrict_ = [&](double* v) {
    dev::k_restrict<<<nblk(N, 256), 256, 0, s>>>(N, nI, h.dmask(), keep, v);
    KCHECK();
  };
  auto solver = [&]() {  // z = B_m r
    if (m == 1) {
      dev::k_hyb_interior<<<nblk(N, 256), 256, 0, s>>>(N, nI, h.d_dinv.p, r, 1.0, z, z, 1, 1);
      KCHECK();
    } else {
      ht_fork(h, r, 1, s);
      op_patch_solves(h, r, 1, s);
      ht_join(h, s);
      dev::k_hyb_interface<<<nblk(N, 256), 256, 0, s>>>(N, nI, h.d_pz_ptr.p, h.d_pz_pos.p, h.d_zpatch.p,
                                                       (int64_t)h.p_dofs.size(), h.ht ? h.d_zg.p : nullptr,
                                                       h.dmask(), r, 1.0, z, z, 1, 1);
      KCHECK();
    }
    restrict_(z);
  };
  auto dotv = [&](const double* a, const double* b) {
    dot(h, a, b, nullptr, 6, h.d_scal.p, 1, s);
    read_scal(h, h.d_scal.p, 1, s);
    return h.h_scal[dev::S_XX];
  };
  restrict_(r);
  solver();
  CK(cudaMemcpyAsync(p, z, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double rz = dotv(r, z);
  std::vector<double> al, be;
  for (int j = 0; j < iters && rz > 0.0 && std::isfinite(rz); ++j) {
    op_apply(h, p, Ap, 1, s, sweep_prec(h));
    restrict_(Ap);
    const double pap = dotv(p, Ap);
    if (!(pap > 0.0)) break;
    const double a = rz / pap;
    dev::k_axpby<<<1184, 256, 0, s>>>(N, -a, Ap, 1.0, r);
    KCHECK();
    solver();
    const double rzn = dotv(r, z);
    al.push_back(a);
    be.push_back(rzn / rz);
    if (!(rzn > 0.0) || !std::isfinite(rzn)) break;
    dev::k_axpby<<<1184, 256, 0, s>>>(N, 1.0, z, be.back(), p);
    KCHECK();
    rz = rzn;
  }
  const int k = (int)al.size();
  if (k == 0) return 1.0;
  Mat T(k, k);
  for (int j = 0; j < k; ++j) {
    T(j, j) = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j + 1 < k) T(j, j + 1) = T(j + 1, j) = std::sqrt(be[j]) / al[j];
  }
  std::vector<double> w;
  Mat V;
  sym_eig(T, w, V);
  return (w.front() + 3.0 * w.back()) / 4.0;
}

void hybrid_weights(riesz_handle& h, cudaStream_t s) {
  if (h.opts.form != RIESZ_FORM_HYBRID || h.rho_fixed) return;
  const double r1 = h.mesh.n_interior > 0 ? lanczos_weight(h, 1, 10, s) : 1.0;
  const double r2 = lanczos_weight(h, 2, 10, s);
  if (r1 != h.rho[1] || r2 != h.rho[2]) h.drop_graphs();  // the loop graphs hold the weights as arguments
  h.rho[1] = r1;
  h.rho[2] = r2;
  h.rho[3] = 1.0;
}

// PCG for nrhs right-hand sides in lockstep (Section 7.1): one apply and one
// preconditioner launch serve all of them.  With apply_precision FP32 the
// search-direction products use the FP32 element matrices and the residual is
// replaced by the FP64 true residual whenever a right-hand side has gained
// four more digits (reliable updates: the FP32 product error, ~1e-7 relative
// per step, stays well below the recursive residual) and when the recursive
// residual claims convergence; the search direction is kept across a
// replacement.
int pcg_batch(riesz_handle& h, const double* b, double* x, int nrhs, cudaStream_t s, int* iters_out,
              double* relres_out) {
  const int64_t N = h.N();
  double* scal = h.d_scal.p;
  const int SS = dev::SCAL_STRIDE;
  const bool a32 = use_a32(h);
  const bool flex = use_flex(h);
  double* r = h.d_r.p;
  double* z = h.d_z.p;
  double* zold = h.d_zold.p;
  double* p = h.d_p.p;
  double* Ap = h.d_Ap.p;
  CK(cudaMemsetAsync(scal, 0, (size_t)nrhs * SS * sizeof(double), s));
  auto residual = [&](bool x_is_zero = false) {  // r = b - A x (FP64), RR
    if (!x_is_zero) op_apply(h, x, Ap, nrhs, s);
    launch(h, RIESZ_K_UPDATE, s, [&] {
      dev::k_residual<<<dim3(dev::red_blocks(N), nrhs), dev::NT, 0, s>>>(N, b, x_is_zero ? nullptr : Ap, r, h.d_part.p,
                                                                      h.d_ticket.p, scal);
    });
  };
  auto restart = [&]() {  // z = P r, p = z, RZ
    op_precond_dot(h, r, z, nullptr, 5, scal, nrhs, s);
    CK(cudaMemcpyAsync(p, z, (size_t)nrhs * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (flex) CK(cudaMemcpyAsync(zold, z, (size_t)nrhs * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  };
  auto nonfinite = [&]() {
    for (int k = 0; k < nrhs; ++k)
      if (h.h_scal[k * SS + dev::S_NONFINITE] != 0.0 || !std::isfinite(h.h_scal[k * SS + dev::S_RR])) return true;
    return false;
  };
  dot(h, b, b, nullptr, 4, scal, nrhs, s);
  dot(h, x, x, nullptr, 6, scal, nrhs, s);
  read_scal(h, scal, nrhs, s);
  bool x_zero = true;  // a zero initial guess needs no operator product for r = b
  for (int k = 0; k < nrhs; ++k) x_zero = x_zero && h.h_scal[k * SS + dev::S_XX] == 0.0;
  residual(x_zero);
  read_scal(h, scal, nrhs, s);
  std::vector<double> bb(nrhs), tol2(nrhs), rr_last(nrhs);
  for (int k = 0; k < nrhs; ++k) {
    bb[k] = h.h_scal[k * SS + dev::S_BB];
    tol2[k] = h.opts.rtol * h.opts.rtol * bb[k];
    rr_last[k] = h.h_scal[k * SS + dev::S_RR];
  }
  if (nonfinite()) {
    g_err = "non-finite right-hand side or initial guess";
    return RIESZ_ERR_NONFINITE;
  }
  auto all_below = [&]() {
    for (int k = 0; k < nrhs; ++k)
      if (!(h.h_scal[k * SS + dev::S_RR] <= tol2[k])) return false;
    return true;
  };
  int it = 0;
  int status = RIESZ_ERR_NOT_CONVERGED;
  if (all_below()) {
    status = RIESZ_OK;
  } else {
    restart();
    while (it < h.opts.maxit) {
      op_apply(h, p, Ap, nrhs, s, inner_prec(h), scal, 0);  // and (p, Ap) -> alpha
      launch(h, RIESZ_K_UPDATE, s, [&] {
        dev::k_update_xr<<<dim3(dev::red_blocks(N), nrhs), dev::NT, 0, s>>>(N, scal, x, r, p, Ap, h.d_part.p,
                                                                          h.d_ticket.p);
      });
      ++it;
      // Copy the scalars back, then enqueue the next preconditioner step before
      // waiting for them, so the GPU is busy while the host checks convergence.
      CK(cudaMemcpyAsync(h.h_scal, scal, (size_t)nrhs * SS * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(h.ev_scal, s));
      op_precond_dot(h, r, z, flex ? zold : nullptr, flex ? 3 : 2, scal, nrhs, s);
      CK(cudaEventSynchronize(h.ev_scal));
      if (nonfinite()) {
        status = RIESZ_ERR_NONFINITE;
        g_err = "non-finite value in the PCG recurrence";
        break;
      }
      bool replace = false;
      if (all_below()) {
        residual();  // verify on the true residual
        read_scal(h, scal, nrhs, s);
        if (all_below()) {
          status = RIESZ_OK;
          break;
        }
        if (!a32) {  // FP64 operator: the recurrence drifted; start afresh from the true residual
          for (int k = 0; k < nrhs; ++k) rr_last[k] = h.h_scal[k * SS + dev::S_RR];
          restart();
          continue;
        }
        replace = true;  // FP32 products: keep the search direction, continue from the true residual
      } else if (a32) {  // reliable update: four more digits on some right-hand side
        for (int k = 0; k < nrhs; ++k) {
          const double rrk = h.h_scal[k * SS + dev::S_RR];
          if (rrk > tol2[k] && rrk <= reliable_gain(h) * rr_last[k]) replace = true;
        }
        if (replace) {
          residual();
          read_scal(h, scal, nrhs, s);
        }
      }
      if (replace) {
        for (int k = 0; k < nrhs; ++k) rr_last[k] = h.h_scal[k * SS + dev::S_RR];
        op_precond_dot(h, r, z, zold, 3, scal, nrhs, s);  // redo the step on the replaced residual
      }
      launch(h, RIESZ_K_UPDATE, s, [&] {
        dev::k_update_p<<<dim3(update_blocks(N), nrhs), 256, 0, s>>>(N, scal, z, p, flex ? zold : nullptr);
      });
    }
    if (status == RIESZ_ERR_NOT_CONVERGED) {
      residual();
      read_scal(h, scal, nrhs, s);
      g_err = "PCG did not reach rtol within maxit";
    }
  }
  for (int k = 0; k < nrhs; ++k) {
    if (iters_out) iters_out[k] = it;
    if (relres_out) relres_out[k] = bb[k] > 0 ? std::sqrt(h.h_scal[k * SS + dev::S_RR] / bb[k]) : 0.0;
  }
  h.last_iters = it;
  return status;
}

// ---- device-driven PCG loop (CUDA graph with a WHILE node) ------------------
// One pass of the loop body is one PCG iteration in the order
//   z = P^{-1} r with (r, z) -> beta;  p = z + beta p;  Ap = A p;  (p, Ap) -> alpha;
//   x += alpha p, r -= alpha Ap with (r, r);  control
// which is the host-driven loop's order rotated so that the control kernel,
// which decides whether another pass runs, comes last.  The entry graph runs
// the second half once (after a restart) before the WHILE node; the resume
// graph starts with the body (after a residual replacement).  Both use only
// handle-owned buffers (x is the handle's working copy d_xw), so they are
// built once per handle and nrhs and relaunched.

constexpr unsigned LOOP_KINDS = (1u << RIESZ_K_APPLY) | (1u << RIESZ_K_APPLY32) | (1u << RIESZ_K_APPLY_TC) |
                                (1u << RIESZ_K_GATHER) |
                                (1u << RIESZ_K_PATCH_SOLVE) | (1u << RIESZ_K_PRECOND_GATHER) | (1u << RIESZ_K_DOT) |
                                (1u << RIESZ_K_SCALAR) | (1u << RIESZ_K_UPDATE) | (1u << RIESZ_K_COARSE_APPLY) |
                                (1u << RIESZ_K_HT);

bool profiling_loop(const riesz_handle& h) { return h.prof && (h.prof_mask & LOOP_KINDS) != 0u; }

// Ap = A p; (p, Ap) -> alpha; x += alpha p, r -= alpha Ap; (r, r) -> RR
void iter_tail(riesz_handle& h, double* x, int nrhs, cudaStream_t s) {
  const int64_t N = h.N();
  op_apply(h, h.d_p.p, h.d_Ap.p, nrhs, s, inner_prec(h), h.d_scal.p, 0);  // and (p, Ap) -> alpha
  launch(h, RIESZ_K_UPDATE, s, [&] {
    dev::k_update_xr<<<dim3(dev::red_blocks(N), nrhs), dev::NT, 0, s>>>(N, h.d_scal.p, x, h.d_r.p, h.d_p.p, h.d_Ap.p,
                                                                      h.d_part.p, h.d_ticket.p);
  });
}

// z = P^{-1} r with (r, z) [and (r, zold)] -> beta; p = z + beta p [zold = z]
void iter_head(riesz_handle& h, int nrhs, cudaStream_t s) {
  const bool flex = use_flex(h);
  op_precond_dot(h, h.d_r.p, h.d_z.p, flex ? h.d_zold.p : nullptr, flex ? 3 : 2, h.d_scal.p, nrhs, s);
  launch(h, RIESZ_K_UPDATE, s, [&] {
    dev::k_update_p<<<dim3(update_blocks(h.N()), nrhs), 256, 0, s>>>(h.N(), h.d_scal.p, h.d_z.p, h.d_p.p, flex ? h.d_zold.p : nullptr);
  });
}

// Add handle h's loop to graph G as a new root branch: [tail, control] then
// WHILE { head, tail, control } (entry), or the WHILE node alone with its
// condition starting at 1 (resume).  Returns the launches of the prologue and
// of one body pass.
std::pair<int64_t, int64_t> add_loop(riesz_handle& h, cudaGraph_t G, int nrhs, bool entry) {
  cudaStream_t cs = h.cap_stream;
  const int64_t l0 = h.launches;
  const int64_t la0 = h.aux ? h.aux->launches : 0;  // launches of the potential problems count here too
  const int64_t lc0 = h.caux ? h.caux->launches : 0;  // and those of the lowest-order coarse handle
  int64_t pro = 0, body = 0;
  cudaGraphConditionalHandle hc;
  CK(cudaGraphConditionalHandleCreate(&hc, G, entry ? 0u : 1u, cudaGraphCondAssignDefault));
  const double rtol2 = h.opts.rtol * h.opts.rtol;
  const double reliable = reliable_gain(h);
  auto control = [&] {
    launch(h, RIESZ_K_SCALAR, cs, [&] {
      dev::k_pcg_control<<<1, 32, 0, cs>>>(hc, h.d_scal.p, nrhs, rtol2, reliable, h.d_ctl.p);
    });
  };
  auto captured = [&](cudaGraph_t target, auto&& body_fn, std::vector<cudaGraphNode_t>* leaves) {
    CK(cudaStreamBeginCaptureToGraph(cs, target, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
      body_fn();
      if (leaves) {
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t* d = nullptr;
        size_t nd = 0;
        CK(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &d, nullptr, &nd));
        leaves->assign(d, d + nd);
      }
    } catch (...) {
      cudaGraph_t g;
      cudaStreamEndCapture(cs, &g);
      cudaGetLastError();
      throw;
    }
    cudaGraph_t g;
    CK(cudaStreamEndCapture(cs, &g));
  };
  std::vector<cudaGraphNode_t> deps;
  if (entry) {
    captured(G, [&] { iter_tail(h, h.d_xw.p, nrhs, cs); control(); }, &deps);
    pro = h.launches - l0;
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wn;
  CK(cudaGraphAddNode(&wn, G, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &cp));
  const int64_t l1 = h.launches;
  captured(cp.conditional.phGraph_out[0], [&] { iter_head(h, nrhs, cs); iter_tail(h, h.d_xw.p, nrhs, cs); control(); },
           nullptr);
  body = h.launches - l1;
  if (h.caux) {  // the coarse steps run in the body (and in the entry graph's prologue only via the head)
    body += h.caux->launches - lc0;
    h.caux->launches = lc0;
  }
  if (h.aux) {
    const int64_t la = h.aux->launches - la0;  // prologue has none: the potential step is in the body only
    body += la;
    h.aux->launches = la0;
  }
  h.launches = l0;  // captured, not launched: counted per executed pass instead
  return {pro, body};
}

cudaGraphExec_t instantiate(cudaGraph_t G) {
  cudaGraphExec_t e = nullptr;
  // kernel nodes keep the priority of the stream they were captured from (the coarse side stream's)
  const cudaError_t rc = cudaGraphInstantiate(&e, G, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(G);
  CK(rc);
  return e;
}

// The handle's cached entry and resume graphs for nrhs right-hand sides.
void ensure_graphs(riesz_handle& h, int nrhs) {
  if (h.g_entry && h.g_nrhs == nrhs) return;
  h.drop_graphs();
  cudaGraph_t G;
  CK(cudaGraphCreate(&G, 0));
  auto pb = add_loop(h, G, nrhs, true);
  h.g_entry = instantiate(G);
  CK(cudaGraphCreate(&G, 0));
  add_loop(h, G, nrhs, false);
  h.g_resume = instantiate(G);
  h.g_nrhs = nrhs;
  h.g_pro_launches = pb.first;
  h.g_body_launches = pb.second;
}

// Host-side state of one system solved with the device-driven loop.
struct LoopSolve {
  riesz_handle* h = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  int nrhs = 1;
  std::vector<double> bb, tol2;
  int status = RIESZ_ERR_NOT_CONVERGED;
  bool done = false;
  int next = 0;     // graph to launch: 1 entry, 2 resume
  int pending = 0;  // host step waiting for scalars: 1 convergence check, 2 replacement, 3 final residual
  int it_before = 0;  // iterations done before the current launch
  int64_t pro = 0, body = 0;  // launches of the current graph's prologue and of one body pass
  std::string err;
};

void ls_read(LoopSolve& L, cudaStream_t s, bool ctl) {
  riesz_handle& h = *L.h;
  CK(cudaMemcpyAsync(h.h_scal, h.d_scal.p, (size_t)L.nrhs * dev::SCAL_STRIDE * sizeof(double),
                     cudaMemcpyDeviceToHost, s));
  if (ctl) CK(cudaMemcpyAsync(h.h_ctl, h.d_ctl.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
}

double ls_scal(const LoopSolve& L, int k, int slot) { return L.h->h_scal[k * dev::SCAL_STRIDE + slot]; }

bool ls_all_below(const LoopSolve& L) {
  for (int k = 0; k < L.nrhs; ++k)
    if (!(ls_scal(L, k, dev::S_RR) <= L.tol2[k])) return false;
  return true;
}

bool ls_nonfinite(const LoopSolve& L) {
  for (int k = 0; k < L.nrhs; ++k)
    if (ls_scal(L, k, dev::S_NONFINITE) != 0.0 || !std::isfinite(ls_scal(L, k, dev::S_RR))) return true;
  return false;
}

// r = b - A x on the working copy (FP64), RR and RRLAST
void ls_residual(LoopSolve& L, cudaStream_t s, bool x_is_zero) {
  riesz_handle& h = *L.h;
  const int64_t N = h.N();
  if (!x_is_zero) op_apply(h, h.d_xw.p, h.d_Ap.p, L.nrhs, s);
  launch(h, RIESZ_K_UPDATE, s, [&] {
    dev::k_residual<<<dim3(dev::red_blocks(N), L.nrhs), dev::NT, 0, s>>>(
        N, L.b, x_is_zero ? nullptr : h.d_Ap.p, h.d_r.p, h.d_part.p, h.d_ticket.p, h.d_scal.p);
  });
}

// z = P r, p = z (and zold = z), RZ
void ls_restart(LoopSolve& L, cudaStream_t s) {
  riesz_handle& h = *L.h;
  const size_t bytes = (size_t)L.nrhs * h.N() * sizeof(double);
  op_precond_dot(h, h.d_r.p, h.d_z.p, nullptr, 5, h.d_scal.p, L.nrhs, s);
  CK(cudaMemcpyAsync(h.d_p.p, h.d_z.p, bytes, cudaMemcpyDeviceToDevice, s));
  if (use_flex(h)) CK(cudaMemcpyAsync(h.d_zold.p, h.d_z.p, bytes, cudaMemcpyDeviceToDevice, s));
}

void ls_finish(LoopSolve& L, int status, const char* msg) {
  L.status = status;
  L.done = true;
  L.next = 0;
  if (msg) L.err = msg;
}

// Solve the systems with the device-driven loop; every phase enqueues the
// work of all systems before one synchronisation.
void solve_graph(std::vector<LoopSolve>& Ls, cudaStream_t s) {
  auto sync = [&] { CK(cudaStreamSynchronize(s)); };
  // phase 1: working copy of x, (b, b) and (x, x)
  for (auto& L : Ls) {
    riesz_handle& h = *L.h;
    const size_t bytes = (size_t)L.nrhs * h.N() * sizeof(double);
    CK(cudaMemcpyAsync(h.d_xw.p, L.x, bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(h.d_scal.p, 0, (size_t)L.nrhs * dev::SCAL_STRIDE * sizeof(double), s));
    dot(h, L.b, L.b, nullptr, 4, h.d_scal.p, L.nrhs, s);
    dot(h, h.d_xw.p, h.d_xw.p, nullptr, 6, h.d_scal.p, L.nrhs, s);
    ls_read(L, s, false);
  }
  sync();
  // phase 2: initial residual (no product for a zero initial guess)
  for (auto& L : Ls) {
    bool x_zero = true;
    for (int k = 0; k < L.nrhs; ++k) x_zero = x_zero && ls_scal(L, k, dev::S_XX) == 0.0;
    ls_residual(L, s, x_zero);
    ls_read(L, s, false);
  }
  sync();
  // phase 3: tolerances, early exits, first restart
  for (auto& L : Ls) {
    riesz_handle& h = *L.h;
    L.bb.resize(L.nrhs);
    L.tol2.resize(L.nrhs);
    for (int k = 0; k < L.nrhs; ++k) {
      L.bb[k] = ls_scal(L, k, dev::S_BB);
      L.tol2[k] = h.opts.rtol * h.opts.rtol * L.bb[k];
    }
    if (ls_nonfinite(L)) {
      ls_finish(L, RIESZ_ERR_NONFINITE, "non-finite right-hand side or initial guess");
      continue;
    }
    if (ls_all_below(L)) {
      ls_finish(L, RIESZ_OK, nullptr);
      continue;
    }
    h.h_ctl[0] = 0;
    h.h_ctl[1] = h.opts.maxit;
    h.h_ctl[2] = 0;
    h.h_ctl[3] = 0;
    CK(cudaMemcpyAsync(h.d_ctl.p, h.h_ctl, 4 * sizeof(int), cudaMemcpyHostToDevice, s));
    if (h.opts.maxit <= 0) {
      L.pending = 3;  // no iteration allowed: report the initial residual
      L.status = RIESZ_ERR_NOT_CONVERGED;
      continue;
    }
    ls_restart(L, s);
    L.next = 1;
  }
  // the copies of h_ctl above must land before the pinned words are reused
  sync();
  for (auto& L : Ls)
    if (L.pending == 3) ls_finish(L, RIESZ_ERR_NOT_CONVERGED, "PCG did not reach rtol within maxit");
  // loop launches until every system is done
  for (int round = 0;; ++round) {
    std::vector<LoopSolve*> act;
    for (auto& L : Ls)
      if (!L.done && L.next) act.push_back(&L);
    if (act.empty()) break;
    if (act.size() == 1) {  // the handle's cached graphs
      LoopSolve& L = *act[0];
      ensure_graphs(*L.h, L.nrhs);
      L.pro = L.next == 1 ? L.h->g_pro_launches : 0;
      L.body = L.h->g_body_launches;
      CK(cudaGraphLaunch(L.next == 1 ? L.h->g_entry : L.h->g_resume, s));
    } else {  // one graph with a branch per system
      cudaGraph_t G;
      CK(cudaGraphCreate(&G, 0));
      try {
        for (LoopSolve* L : act) {
          const auto pb = add_loop(*L->h, G, L->nrhs, L->next == 1);
          L->pro = pb.first;
          L->body = pb.second;
        }
      } catch (...) {
        cudaGraphDestroy(G);
        throw;
      }
      cudaGraphExec_t e = instantiate(G);
      const cudaError_t rc = cudaGraphLaunch(e, s);
      cudaGraphExecDestroy(e);  // freed once the launch completes
      CK(rc);
    }
    for (LoopSolve* L : act) ls_read(*L, s, true);
    sync();
    // launches that ran: the prologue once (entry) and the body once per further pass
    for (LoopSolve* L : act) {
      riesz_handle& h = *L->h;
      const int it = h.h_ctl[0];
      const int64_t passes = it - L->it_before - (L->next == 1 ? 1 : 0);
      h.launches += L->pro + std::max<int64_t>(0, passes) * L->body;
      L->it_before = it;
    }
    bool any_pending = false;
    for (LoopSolve* L : act) {
      const int reason = L->h->h_ctl[2];
      L->next = 0;
      if (reason == 1) {
        ls_finish(*L, RIESZ_ERR_NONFINITE, "non-finite value in the PCG recurrence");
      } else if (reason == 2 || reason == 3 || reason == 4) {
        ls_residual(*L, s, false);
        ls_read(*L, s, false);
        L->pending = reason == 2 ? 1 : reason == 3 ? 2 : 3;
        any_pending = true;
      } else {
        ls_finish(*L, RIESZ_ERR_INTERNAL, "device loop stopped without a reason");
      }
    }
    if (any_pending) sync();
    for (LoopSolve* L : act) {
      if (!L->pending) continue;
      const int p = L->pending;
      L->pending = 0;
      riesz_handle& h = *L->h;
      if (p == 1 && ls_all_below(*L)) {
        ls_finish(*L, RIESZ_OK, nullptr);
      } else if (p == 3 || h.h_ctl[0] >= h.opts.maxit) {
        ls_finish(*L, RIESZ_ERR_NOT_CONVERGED, "PCG did not reach rtol within maxit");
      } else if (p == 1 && !use_a32(h)) {
        ls_restart(*L, s);  // FP64 operator: the recurrence drifted; start afresh from the true residual
        L->next = 1;
      } else {
        L->next = 2;  // FP32 products: keep the search direction, continue from the true residual
      }
    }
  }
  for (auto& L : Ls) L.h->last_iters = L.it_before;
  // results back to the caller's x
  for (auto& L : Ls) {
    riesz_handle& h = *L.h;
    CK(cudaMemcpyAsync(L.x, h.d_xw.p, (size_t)L.nrhs * h.N() * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  sync();
}

// One system: the device-driven loop unless the handle asks for the host loop
// or the profiler times loop kernels.
int solve_one(riesz_handle& h, const double* b, double* x, int nrhs, cudaStream_t s, int* iters, double* relres) {
  if (h.opts.loop != RIESZ_LOOP_GRAPH || profiling_loop(h)) return pcg_batch(h, b, x, nrhs, s, iters, relres);
  std::vector<LoopSolve> Ls(1);
  Ls[0].h = &h;
  Ls[0].b = b;
  Ls[0].x = x;
  Ls[0].nrhs = nrhs;
  solve_graph(Ls, s);
  const LoopSolve& L = Ls[0];
  for (int k = 0; k < nrhs; ++k) {
    if (iters) iters[k] = L.it_before;
    if (relres) relres[k] = L.bb[k] > 0 ? std::sqrt(ls_scal(L, k, dev::S_RR) / L.bb[k]) : 0.0;
  }
  if (L.status != RIESZ_OK) g_err = L.err;
  return L.status;
}

// The dynamic shared-memory limit of a kernel is a property of the function
// in the device's context, shared by every handle: only ever raise it, so a
// handle with smaller needs cannot lower it below another live handle's.
template <typename K>
void raise_smem_limit(K* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[{dev, (const void*)kernel}];
  if (bytes <= cur) return;
  CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
}

// Dynamic shared memory that limits k_cholesky to `ctas` resident CTAs per SM
// (0: no limit beyond registers and its static shared memory).  With fewer
// resident CTAs than patches, the patches left over start as CTAs finish, in
// launch order (largest first), which balances the SMs' work when a few large
// patches would otherwise pile up on some SMs.
size_t chol_pad(int ctas) {
  if (ctas <= 0) return 0;
  static std::mutex mu;
  static std::map<int, std::array<long, 3>> dev_info;  // smem per SM, reserved per CTA, static smem
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::array<long, 3> di;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = dev_info.find(dev);
    if (it == dev_info.end()) {
      int smem_sm = 0, reserved = 0;
      CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
      CK(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
      cudaFuncAttributes fa;
      CK(cudaFuncGetAttributes(&fa, dev::k_cholesky<1>));
      it = dev_info.emplace(dev, std::array<long, 3>{smem_sm, reserved, (long)fa.sharedSizeBytes}).first;
    }
    di = it->second;
  }
  const long per_cta = (di[0] / ctas) / 1024 * 1024;  // ctas fit, ctas + 1 do not
  const long pad = per_cta - di[2] - di[1];
  if (pad <= 0) return 0;
  raise_smem_limit(dev::k_cholesky<1>, (size_t)pad);
  raise_smem_limit(dev::k_cholesky<2>, (size_t)pad);
  return (size_t)pad;
}

// The patch factorisation with `split` CTAs per patch (1, or a 2-CTA cluster)
// and `ctas` resident CTAs per SM (0: no limit).
void launch_cholesky(riesz_handle& h, int split, int ctas, cudaStream_t s) {
  const int npatch = (int)h.p_n.size();
  const size_t pad = chol_pad(ctas);
  if (split == 1) {
    dev::k_cholesky<1><<<npatch, dev::NT, pad, s>>>(h.d_pn.p, h.d_pfoff.p, h.d_pdioff.p, h.d_pmoff.p, h.d_meta.p,
                                                    h.d_L64.p, h.d_D64.p, h.d_info.p);
    KCHECK();
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * npatch));
  cfg.blockDim = dim3(dev::NT);
  cfg.dynamicSmemBytes = pad;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CK(cudaLaunchKernelEx(&cfg, dev::k_cholesky<2>, (const int32_t*)h.d_pn.p, (const int64_t*)h.d_pfoff.p,
                        (const int64_t*)h.d_pdioff.p, (const int64_t*)h.d_pmoff.p, (const int32_t*)h.d_meta.p,
                        h.d_L64.p, h.d_D64.p, h.d_info.p));
}

// FP64: positive definite inverse X = L^{-T} L^{-1} from the blocked Cholesky factor
// (stored negated in d_X0d, the convention of the swept Gauss-Jordan matrix).
void coarse_setup_chol(riesz_handle& h, cudaStream_t s) {
  const int nb = h.N0p / dev::CB;
  const RefElement& R = *h.ref;
  const size_t sm = dev::gj_smem<double>();
  double* A = h.d_A0d.p;
  CK(cudaMemsetAsync(A, 0, h.d_A0d.bytes(), s));
  CK(cudaMemsetAsync(h.d_cbad.p, 0, sizeof(int), s));
  launch(h, RIESZ_K_COARSE, s, [&] {
    dev::k_coarse_assemble<double><<<nblk(h.N0p, 128), 128, 0, s>>>(h.N0, h.N0p, h.d_cptr.p, h.d_cJ.p, h.d_ccell.p,
                                                                    h.d_cab.p, h.C(), h.mesh.nref, R.Q, h.d_g.p,
                                                                    h.d_R.p, A);
  });
  for (int k = 0; k < nb; ++k) {
    launch(h, RIESZ_K_COARSE, s, [&] { dev::k_cc_pivot<<<1, 256, 0, s>>>(h.N0p, k, A, h.d_Dinv0d.p, h.d_cbad.p); });
    const int m = nb - 1 - k;
    if (m > 0) {
      launch(h, RIESZ_K_COARSE, s, [&] { dev::k_cc_panel<<<m, 256, sm, s>>>(h.N0p, k, A, h.d_Dinv0d.p); });
      launch(h, RIESZ_K_COARSE, s, [&] { dev::k_cc_update<<<m * (m + 1) / 2, 256, sm, s>>>(h.N0p, k, A); });
    }
  }
  for (int k = 0; k < nb; ++k) {
    if (k > 0)
      launch(h, RIESZ_K_COARSE, s,
             [&] { dev::k_ct_row<<<k, 256, sm, s>>>(h.N0p, k, A, h.d_Dinv0d.p, h.d_Rb0d.p); });
    if (k > 0 && nb - 1 - k > 0)
      launch(h, RIESZ_K_COARSE, s,
             [&] { dev::k_ct_update<<<(nb - 1 - k) * k, 256, sm, s>>>(h.N0p, k, A, h.d_Rb0d.p); });
    launch(h, RIESZ_K_COARSE, s,
           [&] { dev::k_ct_finish<<<nb, 256, sm, s>>>(h.N0p, k, A, h.d_Dinv0d.p, h.d_Rb0d.p); });
  }
  launch(h, RIESZ_K_COARSE, s,
         [&] { dev::k_ct_lauum<<<nb * (nb + 1) / 2, 256, sm, s>>>(h.N0p, nb, A, h.d_X0d.p); });
  if (nb > 1)
    launch(h, RIESZ_K_COARSE, s,
           [&] { dev::k_coarse_mirror<double><<<nb * (nb - 1) / 2, 256, 0, s>>>(h.N0p, h.d_X0d.p); });
}

void device_compute(riesz_handle& h, cudaStream_t s, bool with_aux, bool sync);
// Sparse route: the p = 1 handle's geometry, element matrices and patch factors for the same vertices.
void coarse_setup_sparse(riesz_handle& h, cudaStream_t s) {
  riesz_handle& a = *h.caux;
  CK(cudaMemcpyAsync(a.d_verts.p, h.d_verts.p, h.d_verts.bytes(), cudaMemcpyDeviceToDevice, s));
  device_compute(a, s, false, false);
}

void coarse_setup(riesz_handle& h, cudaStream_t s) {
  if (h.coarse_sparse)
    coarse_setup_sparse(h, s);
  else
    coarse_setup_chol(h, s);
}

// Patch factorisations that met a non-positive pivot (after the stream is synchronised).
void check_factor_info(riesz_handle& h, cudaStream_t s) {
  if (h.coarse_on && !h.coarse_sparse) {
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, h.d_cbad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (bad) throw Err(RIESZ_ERR_INTERNAL, "coarse matrix not positive definite");
  }
  const int npatch = (int)h.p_n.size();
  if (!npatch) return;
  std::vector<int> info(npatch);
  CK(cudaMemcpyAsync(info.data(), h.d_info.p, sizeof(int) * npatch, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int P = 0; P < npatch; ++P)
    if (info[P]) throw Err(RIESZ_ERR_INTERNAL, "patch matrix not positive definite");
}

// Device setup from resident maps and vertex coordinates: a1 geometry,
// element matrices, a6 interior diagonal, a8 patch assembly + Cholesky.
// with_aux: also recompute the potential problems of a Hiptmair-Toselli
// handle (on their own stream, beside this handle's factorisation).  sync:
// wait for the result, record the device setup time and check the pivots.
// Device setup, first part: everything up to the assembled patch matrices (the potential problems and
// the coarse setup forked onto their streams).
void device_compute_pre(riesz_handle& h, cudaStream_t s, bool aux_now) {
  const RefElement& R = *h.ref;
  const MeshMaps& M = h.mesh;
  const int n = M.nref;
  const int64_t C = M.ncells;
  const int npatch = (int)h.p_n.size();
  if (aux_now) {  // the potential problems follow the same vertices
    CK(cudaEventRecord(h.ev_hfork, s));
    CK(cudaStreamWaitEvent(h.ht_stream, h.ev_hfork, 0));
    CK(cudaMemcpyAsync(h.aux->d_verts.p, h.d_verts.p, h.d_verts.bytes(), cudaMemcpyDeviceToDevice, h.ht_stream));
    device_compute(*h.aux, h.ht_stream, false, false);
    CK(cudaEventRecord(h.ev_hjoin, h.ht_stream));
  }
  launch(h, RIESZ_K_GEOM, s, [&] {
    dev::k_geom<<<nblk(C, 128), 128, 0, s>>>(h.space, C, h.d_verts.p, h.d_cells.p, ref_edge_inverse(),
                                              h.opts.alpha, h.opts.beta, h.d_g.p, h.d_jac.p);
  });
  if (h.coarse_on) {  // the coarse setup (FP32) needs only g: run it beside the FP64 patch factorisation
    CK(cudaEventRecord(h.ev_fork, s));
    CK(cudaStreamWaitEvent(h.side_stream, h.ev_fork, 0));
    coarse_setup(h, h.side_stream);
    CK(cudaEventRecord(h.ev_join, h.side_stream));
  }
  if (h.opts.apply_mode == RIESZ_APPLY_ELEMENT) {
    launch(h, RIESZ_K_ELEM, s, [&] {
      const unsigned grid = (unsigned)((C + dev::ELEM_CELLS - 1) / dev::ELEM_CELLS);
      if (R.Q == 12)
        dev::k_elem_matrices<12><<<grid, 256, 0, s>>>(C, n, h.d_g.p, h.d_R.p, h.d_Ae.p);
      else
        dev::k_elem_matrices<7><<<grid, 256, 0, s>>>(C, n, h.d_g.p, h.d_R.p, h.d_Ae.p);
    });
    if (h.d_Ae32.p)
      launch(h, RIESZ_K_TO_F32, s, [&] {
        dev::k_to_f32<<<1184, 256, 0, s>>>((int64_t)h.d_Ae.n, h.d_Ae.p, h.d_Ae32.p);
      });
  }
  if (M.n_interior > 0) {
    const int64_t cnt = C * (int64_t)(n - h.nif);
    launch(h, RIESZ_K_DIAG, s, [&] {
      dev::k_interior_diag<<<nblk(cnt, 256), 256, 0, s>>>(C, n, h.nif, R.Q, h.d_g.p, h.d_R.p, h.d_cdofs.p,
                                                         M.n_interface, h.d_dinv.p);
    });
  }
  CK(cudaMemsetAsync(h.d_info.p, 0, sizeof(int) * std::max(1, npatch), s));
  if (npatch) {
    launch(h, RIESZ_K_ASSEMBLE, s, [&] {
      dev::k_patch_assemble<<<npatch, 256, 0, s>>>(h.d_pn.p, h.d_pfoff.p, h.d_pmoff.p, h.d_meta.p, h.d_pb_ptr.p,
                                                   h.d_pb_cell.p, h.d_pb_off.p, h.d_pb_ent.p, C, n, R.Q, h.d_g.p,
                                                   h.d_R.p, h.d_Ae.p, h.d_L64.p);
    });
  }
}

// Device setup, last part (after the patch factorisation): the FP32 copies of the factors, then the
// joins of the side streams.
void device_compute_post(riesz_handle& h, cudaStream_t s, bool aux_now) {
  const int npatch = (int)h.p_n.size();
  if (npatch) {
    if (h.opts.precond_precision == RIESZ_PREC_FP32 && h.factor_entries % 1024 == 0 &&
        h.dinv_entries % 1024 == 0) {  // whole tiles: one pass per factor array
      launch(h, RIESZ_K_TO_F32, s, [&] {
        dev::k_to_f32_tiles<<<1184, 256, 0, s>>>(h.factor_entries >> 10, h.d_L64.p, h.d_L32.p, h.d_L32T.p);
      });
      launch(h, RIESZ_K_TO_F32, s, [&] {
        dev::k_to_f32_tiles<<<296, 256, 0, s>>>(h.dinv_entries >> 10, h.d_D64.p, h.d_D32.p, h.d_D32T.p);
      });
    } else if (h.opts.precond_precision == RIESZ_PREC_FP32) {
      launch(h, RIESZ_K_TO_F32, s, [&] {
        dev::k_to_f32<<<1184, 256, 0, s>>>(h.factor_entries, h.d_L64.p, h.d_L32.p);
      });
      if (h.d_L32T.p) {
        launch(h, RIESZ_K_TO_F32, s, [&] {
          dev::k_to_f32_tiles_t<<<1184, 256, 0, s>>>(h.factor_entries, h.d_L64.p, h.d_L32T.p);
        });
        launch(h, RIESZ_K_TO_F32, s, [&] {
          dev::k_to_f32_tiles_t<<<296, 256, 0, s>>>(h.dinv_entries, h.d_D64.p, h.d_D32T.p);
        });
      }
      launch(h, RIESZ_K_TO_F32, s, [&] {
        dev::k_to_f32<<<296, 256, 0, s>>>(h.dinv_entries, h.d_D64.p, h.d_D32.p);
      });
    }
  }
  if (h.coarse_on) CK(cudaStreamWaitEvent(s, h.ev_join, 0));
  if (aux_now) CK(cudaStreamWaitEvent(s, h.ev_hjoin, 0));
}

void device_compute(riesz_handle& h, cudaStream_t s, bool with_aux = true, bool sync = true) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (sync) {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
  }
  const bool aux_now = h.aux && with_aux;
  device_compute_pre(h, s, aux_now);
  if (!h.p_n.empty())
    launch(h, RIESZ_K_CHOLESKY, s, [&] {
      launch_cholesky(h, h.chol_split, h.chol_ctas, s);
    });
  device_compute_post(h, s, aux_now);
  if (!sync) return;
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  h.setup_dev_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check_factor_info(h, s);
  if (aux_now) check_factor_info(*h.aux, s);
  if (h.caux && h.coarse_on) check_factor_info(*h.caux, s);
  hybrid_weights(h, s);
}

// Autotuner of the patch factorisation's residency: with between one and 24
// patches per SM the balance of work over the SMs depends on how many CTAs
// are resident at once (all at once: fixed round-robin placement; fewer:
// later patches go to whichever SM frees a slot first).  Each candidate is
// timed on the handle's own patches (assembly untimed, then the Cholesky
// launch between CUDA events) and the fastest is kept; the factors are then
// recomputed with it.  Every candidate computes bitwise the same factors.
void tune_cholesky(riesz_handle& h, cudaStream_t s) {
  const int npatch = (int)h.p_n.size();
  int nsm = 0;
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h.device));
  h.chol_ctas = 0;
  h.chol_split = h.opts.autotune == 2 ? 2 : 1;
  h.chol_tuned = 0;
  if (h.opts.autotune == 2) {  // fixed: 2-CTA clusters, maximum residency
    device_compute(h, s, false);
    return;
  }
  if (!h.opts.autotune || npatch <= nsm || npatch > 24 * nsm) return;
  // a decision taken for the same space, degree and patch structure on this device is reused
  static std::mutex mu;
  static std::map<std::array<int64_t, 6>, std::array<int, 3>> done;  // split, ctas, candidates timed
  const std::array<int64_t, 6> key{h.device, h.space, h.p, npatch, (int64_t)h.factor_entries, h.C()};
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(key);
    if (it != done.end()) {
      h.chol_split = it->second[0];
      h.chol_ctas = it->second[1];
      h.chol_tuned = it->second[2];
      if (h.chol_split != 1 || h.chol_ctas != 0) device_compute(h, s, false);
      return;
    }
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 0.f;
  int best_c = 0, best_split = 1;
  for (int split : {1, 2})
    for (int c : {0, 4, 3, 2}) {
      CK(cudaMemsetAsync(h.d_info.p, 0, sizeof(int) * npatch, s));
      dev::k_patch_assemble<<<npatch, 256, 0, s>>>(h.d_pn.p, h.d_pfoff.p, h.d_pmoff.p, h.d_meta.p, h.d_pb_ptr.p,
                                                   h.d_pb_cell.p, h.d_pb_off.p, h.d_pb_ent.p, h.C(), h.mesh.nref,
                                                   h.ref->Q, h.d_g.p, h.d_R.p, h.d_Ae.p, h.d_L64.p);
      KCHECK();
      CK(cudaEventRecord(e0, s));
      launch_cholesky(h, split, c, s);
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      h.launches += 2;
      ++h.chol_tuned;
      if (h.chol_tuned == 1 || ms < best) {
        best = ms;
        best_c = c;
        best_split = split;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h.chol_ctas = best_c;
  h.chol_split = best_split;
  {
    std::lock_guard<std::mutex> lk(mu);
    done[key] = {best_split, best_c, h.chol_tuned};
  }
  device_compute(h, s, false);  // factors (and their FP32 copies) with the chosen residency
}

// Autotuner of the multi-RHS FP32 sweep shape for patches of at most 8 tiles (the edge stars of
// PAFW_1 and Hiptmair-Toselli): one CTA per patch with the bulk-copy ring (k_patch_sweep8), or one
// warp per patch with 4 or 8 warps per block (k_patch_sweep_warp8).  Each candidate sweeps 8
// right-hand sides (the residual workspace, zeroed) over the handle's own factors, once untimed and
// twice between CUDA events; the fastest is kept per device and patch structure.  Every candidate
// computes the same patch solutions up to the FP32 summation order within a tile row.
void tune_sweeps(riesz_handle& h, cudaStream_t s) {
  const int npatch = (int)h.p_n.size();
  h.sweep_tuned = 0;
  h.sweep_shape = 8;
  const int nr = std::min(8, h.opts.nrhs_max);
  if (h.opts.autotune != 1 || !npatch || nr < 2 || h.opts.precond_precision != RIESZ_PREC_FP32 ||
      (h.p_n[0] + 31) / 32 > dev::WARP_NB || (h.p_n[0] + 31) / 32 <= dev::SMALL_NB)
    return;
  static std::mutex mu;
  static std::map<std::array<int64_t, 5>, std::array<int, 2>> done;  // shape, candidates timed
  const std::array<int64_t, 5> key{h.device, npatch, (int64_t)h.factor_entries, (int64_t)h.p_dofs.size(), nr};
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(key);
    if (it != done.end()) {
      h.sweep_shape = it->second[0];
      h.sweep_tuned = it->second[1];
      return;
    }
  }
  CK(cudaMemsetAsync(h.d_r.p, 0, (size_t)nr * h.N() * sizeof(double), s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 0.f;
  int best_shape = 8;
  for (int shape : {8, 4, 0}) {
    h.sweep_shape = shape;
    op_patch_solves(h, h.d_r.p, nr, s);
    CK(cudaEventRecord(e0, s));
    for (int rep = 0; rep < 2; ++rep) op_patch_solves(h, h.d_r.p, nr, s);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ++h.sweep_tuned;
    if (h.sweep_tuned == 1 || ms < best) {
      best = ms;
      best_shape = shape;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h.sweep_shape = best_shape;
  std::lock_guard<std::mutex> lk(mu);
  done[key] = {best_shape, h.sweep_tuned};
}

// Round-to-nearest-even BF16 bits of an FP32 value (finite inputs).
uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
float bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// The B operand of k_apply_tc: for each stage (TC_KC-wide chunk jc of j, then q) the split
// R_q[i][jc*TC_KC + kk] = hi + lo (hi = bf16(R), lo = bf16(R - hi)), hi block then lo block, each
// [NP/8 row groups][TC_KCORE K core matrices][8 rows][8 values] (the K-major layout without swizzle).
void build_tc_table(riesz_handle& h, std::vector<uint16_t>& t) {
  const int n = h.mesh.nref, Q = h.ref->Q, NP = h.tc_np, KC = h.tc_kc;
  const std::vector<double>& R = h.ref->R;
  const size_t blk = (size_t)NP * dev::TC_KC;
  t.assign((size_t)KC * Q * 2 * blk, 0);
  for (int jc = 0; jc < KC; ++jc)
    for (int q = 0; q < Q; ++q) {
      const size_t base = ((size_t)jc * Q + q) * 2 * blk;
      for (int i = 0; i < n; ++i)
        for (int kk = 0; kk < dev::TC_KC; ++kk) {
          const int k = jc * dev::TC_KC + kk;
          if (k >= n) break;
          const double v = R[(size_t)q * n * n + (size_t)i * n + k];
          const uint16_t hi = bf16_bits((float)v);
          const uint16_t lo = bf16_bits((float)(v - (double)bf16_value(hi)));
          const size_t idx = ((size_t)(i / 8) * dev::TC_KCORE + kk / 8) * 64 + (size_t)(i % 8) * 8 + kk % 8;
          t[base + idx] = hi;
          t[base + blk + idx] = lo;
        }
    }
}

void setup_device_impl(riesz_handle& h, cudaStream_t s) {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) throw Err(RIESZ_ERR_CUDA, "no CUDA device");
  CK(cudaGetDevice(&h.device));
  h.free_device();
  const RefElement& R = *h.ref;
  const MeshMaps& M = h.mesh;
  const int n = M.nref;
  const int64_t C = M.ncells, N = M.ndofs;
  const int nrhs = std::max(1, h.opts.nrhs_max);
  h.d_verts.upload(h.verts, s);
  h.d_cells.upload(M.cells, s);
  h.d_cdofs.upload(transpose_dofs(M.cell_dofs, C, n), s);
  h.d_R.upload(R.R, s);
  h.d_g.alloc((size_t)R.Q * C);
  h.d_jac.alloc((size_t)C * 10);
  h.d_Ycell.alloc((size_t)nrhs * h.nif * C);
  h.d_dinv.alloc(std::max<int64_t>(1, M.n_interior));
  h.d_sc_ptr.upload(h.sc_ptr, s);
  h.d_sc_pos.upload(h.sc_pos, s);
  h.d_pn.upload(h.p_n, s);
  h.d_pdoff.upload(h.p_doff, s);
  h.d_pfoff.upload(h.p_foff, s);
  h.d_pdofs.upload(h.p_dofs, s);
  h.d_pz_ptr.upload(h.pz_ptr, s);
  h.d_pz_pos.upload(h.pz_pos, s);
  h.d_pb_ptr.upload(h.pb_ptr, s);
  h.d_pb_off.upload(h.pb_off, s);
  h.d_pb_cell.upload(h.pb_cell, s);
  h.d_pb_ent.upload(h.pb_ent, s);
  h.d_zpatch.alloc(std::max<size_t>(1, h.p_dofs.size() * nrhs));
  h.d_X.upload(R.Xcross, s);
  h.d_cgdofs.upload(transpose_dofs(h.meshcg.cell_dofs, C, h.refcg->nref), s);
  for (auto* b : {&h.d_r, &h.d_z, &h.d_zold, &h.d_p, &h.d_Ap, &h.d_tmp, &h.d_xh, &h.d_xw}) b->alloc((size_t)N * nrhs);
  h.d_ctl.alloc(4);
  h.d_flags.alloc(4);
  CK(cudaMemsetAsync(h.d_flags.p, 0, 4 * sizeof(int), s));
  CK(cudaMallocHost((void**)&h.h_ctl, 4 * sizeof(int)));
  if (!h.cap_stream) CK(cudaStreamCreateWithFlags(&h.cap_stream, cudaStreamNonBlocking));
  if (!h.side_stream) {
    // the coarse correction's small kernels run beside the patch sweeps; at the highest priority their
    // blocks are scheduled as soon as SMs free up instead of queueing behind the sweep's blocks
    int prio_low = 0, prio_high = 0;
    CK(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    CK(cudaStreamCreateWithPriority(&h.side_stream, cudaStreamNonBlocking, prio_high));
  }
  if (!h.ev_fork) CK(cudaEventCreateWithFlags(&h.ev_fork, cudaEventDisableTiming));
  if (!h.ev_join) CK(cudaEventCreateWithFlags(&h.ev_join, cudaEventDisableTiming));
  if (!h.ev_pfork) CK(cudaEventCreateWithFlags(&h.ev_pfork, cudaEventDisableTiming));
  if (!h.ev_pjoin) CK(cudaEventCreateWithFlags(&h.ev_pjoin, cudaEventDisableTiming));
  h.d_part.alloc((size_t)2 * dev::RED_BLOCKS * nrhs);
  h.d_scal.alloc(16 * (size_t)nrhs);
  CK(cudaMallocHost((void**)&h.h_scal, (size_t)16 * nrhs * sizeof(double)));
  if (!h.ev_scal) CK(cudaEventCreateWithFlags(&h.ev_scal, cudaEventDisableTiming));
  const int npatch = (int)h.p_n.size();
  h.d_info.alloc(std::max(1, npatch));
  if (h.opts.apply_mode == RIESZ_APPLY_ELEMENT) {
    h.d_Ae.alloc((size_t)C * n * n);
    if (needs_ae32(h)) h.d_Ae32.alloc((size_t)C * n * n);
  } else {
    const size_t sm = ((size_t)n + R.Q) * dev::TC * sizeof(double);
    raise_smem_limit(dev::k_apply_mf, (size_t)sm);
  }
  {
    const size_t sm = (size_t)n * nrhs * sizeof(double);
    if (sm > 48 * 1024) {
      raise_smem_limit(dev::k_apply_elem<double, 8>, (size_t)sm);
      raise_smem_limit(dev::k_apply_elem<float, 8>, (size_t)sm);
    }
  }
  {  // right-hand sides per multi-RHS sweep launch: as many as fit in shared memory (<= 8)
    const size_t per = (size_t)(h.p_n.empty() ? 32 : (h.p_n[0] + 31) / 32 * 32) *
                       (h.opts.precond_precision == RIESZ_PREC_FP32 ? sizeof(float) : sizeof(double));
    const size_t budget = 160 * 1024;  // dynamic share, leaves room for the static reduction buffers
    h.multi_group = (int)std::max<size_t>(1, std::min<size_t>(8, budget / per));
    const int smm = (int)(per * h.multi_group);
    raise_smem_limit(dev::k_patch_solve_multi<double>, (size_t)smm);
    const int nbm = h.p_n.empty() ? 1 : (h.p_n[0] + 31) / 32;
    raise_smem_limit(dev::k_patch_sweep8<SWEEP_SLOTS_F32>, sweep8_smem(nbm));
    raise_smem_limit(dev::k_patch_solve_small<double>, dev::SMALL_WARPS * dev::small_warp_smem<double>());
    raise_smem_limit(dev::k_patch_sweep_warp8, dev::WARP_SWEEP_WARPS * dev::warp_sweep_smem());
    raise_smem_limit(dev::k_patch_solve_small<float>, dev::SMALL_WARPS * dev::small_warp_smem<float>());
  }
  h.d_pdioff.upload(h.p_dioff, s);
  h.d_pmoff.upload(h.p_moff, s);
  h.d_meta.upload(h.p_meta, s);
  if (h.opts.dirichlet) h.d_dmask.upload(h.dir_mask, s);
  if (h.ht) {
    if (!h.ht_stream) CK(cudaStreamCreateWithFlags(&h.ht_stream, cudaStreamNonBlocking));
    if (!h.ev_hfork) CK(cudaEventCreateWithFlags(&h.ev_hfork, cudaEventDisableTiming));
    if (!h.ev_hjoin) CK(cudaEventCreateWithFlags(&h.ev_hjoin, cudaEventDisableTiming));
    setup_device_impl(*h.aux, s);
    h.d_gt_ptr.upload(h.gt_ptr, s);
    h.d_gt_idx.upload(h.gt_idx, s);
    h.d_gt_sgn.upload(h.gt_sgn, s);
    h.d_gg_ptr.upload(h.gg_ptr, s);
    h.d_gg_idx.upload(h.gg_idx, s);
    h.d_gg_sgn.upload(h.gg_sgn, s);
    h.d_zcg.alloc((size_t)nrhs * h.aux->mesh.n_interface);
    h.d_zg.alloc((size_t)nrhs * M.n_interface);
  }
  if (h.coarse_on && h.coarse_sparse) {
    h.d_cw.upload(h.c_w, s);
    h.d_cidx.upload(h.c_idx, s);
    h.d_caux.upload(h.c_aux, s);
    h.d_zc.alloc((size_t)nrhs * h.N0);
    setup_device_impl(*h.caux, s);
  } else if (h.coarse_on) {
    h.d_cw.upload(h.c_w, s);
    h.d_cidx.upload(h.c_idx, s);
    h.d_cptr.upload(h.c_ptr, s);
    h.d_cJ.upload(h.c_J, s);
    h.d_ccell.upload(h.c_cell, s);
    h.d_cab.upload(h.c_ab, s);
    {  // FP64 Cholesky-route inverse (positive definite by construction)
      h.d_A0d.alloc((size_t)h.N0p * h.N0p);
      h.d_X0d.alloc((size_t)h.N0p * h.N0p);
      h.d_Dinv0d.alloc((size_t)h.N0p * dev::CB);  // the inverse of every diagonal tile of L
      h.d_Rb0d.alloc((size_t)dev::CB * h.N0p);
      h.d_r0d.alloc((size_t)nrhs * h.N0p);
      h.d_cbad.alloc(1);
      CK(cudaMemsetAsync(h.d_cbad.p, 0, sizeof(int), s));
      raise_smem_limit(dev::k_cc_panel, dev::gj_smem<double>());
      raise_smem_limit(dev::k_cc_update, dev::gj_smem<double>());
      raise_smem_limit(dev::k_ct_row, dev::gj_smem<double>());
      raise_smem_limit(dev::k_ct_update, dev::gj_smem<double>());
      raise_smem_limit(dev::k_ct_finish, dev::gj_smem<double>());
      raise_smem_limit(dev::k_ct_lauum, dev::gj_smem<double>());
    }
    h.d_zc.alloc((size_t)nrhs * h.N0);
    const size_t per = (size_t)h.N0p * sizeof(double);
    h.coarse_group = (int)std::max<size_t>(1, std::min<size_t>(8, (160 * 1024) / per));
    raise_smem_limit(dev::k_coarse_apply<double>, per * h.coarse_group);
  }
  if (npatch) {
    h.d_L64.alloc((size_t)h.factor_entries);
    h.d_D64.alloc((size_t)h.dinv_entries);
    if (h.opts.precond_precision == RIESZ_PREC_FP32) {
      h.d_L32.alloc((size_t)h.factor_entries);
      if (nrhs > 1) {
        h.d_L32T.alloc((size_t)h.factor_entries);
        h.d_D32T.alloc((size_t)h.dinv_entries);
      }
      h.d_D32.alloc((size_t)h.dinv_entries);
    }
  }
  {
    const int nbm = h.p_n.empty() ? 1 : (h.p_n[0] + 31) / 32;
    raise_smem_limit(dev::k_patch_sweep<float, SWEEP_SLOTS_F32>, sweep_smem<float>(SWEEP_SLOTS_F32, nbm));
    raise_smem_limit(dev::k_patch_sweep<double, SWEEP_SLOTS_F64>, sweep_smem<double>(SWEEP_SLOTS_F64, nbm));
  }
  if (h.opts.form == RIESZ_FORM_HYBRID)
    for (auto* b : {&h.d_hres, &h.d_hc, &h.d_hAc}) b->alloc((size_t)N * nrhs);
  if (needs_tc(h)) {
    h.tc_np = (n + 15) / 16 * 16;
    h.tc_kc = (n + dev::TC_KC - 1) / dev::TC_KC;
    std::vector<uint16_t> t;
    build_tc_table(h, t);
    h.d_Btc.upload(t, s);
    if (h.ref->Q != 7 && h.ref->Q != 12) throw Err(RIESZ_ERR_INTERNAL, "tensor-core products: Q must be 7 or 12");
    for (int c = 0; c < C; ++c)  // interior DOFs of a cell are contiguous (the kernel writes them from the first)
      for (int t = h.nif + 1; t < n; ++t)
        if (M.cell_dofs[(size_t)c * n + t] != M.cell_dofs[(size_t)c * n + h.nif] + (t - h.nif))
          throw Err(RIESZ_ERR_INTERNAL, "interior DOFs of a cell are not contiguous");
    const int npc = dev::tc_part_cols(h.tc_np, 0);
    raise_smem_limit(dev::k_apply_tc<7>, dev::tc_smem_bytes(npc, dev::tc_stages(npc)));
    raise_smem_limit(dev::k_apply_tc<12>, dev::tc_smem_bytes(npc, dev::tc_stages(npc)));
  }
  h.d_ticket.alloc(nrhs);
  CK(cudaMemsetAsync(h.d_ticket.p, 0, sizeof(unsigned) * nrhs, s));
  CK(cudaFuncSetAttribute(dev::k_cholesky<1>, cudaFuncAttributePreferredSharedMemoryCarveout,
                          (int)cudaSharedmemCarveoutMaxShared));
  CK(cudaFuncSetAttribute(dev::k_cholesky<2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                          (int)cudaSharedmemCarveoutMaxShared));
  device_compute(h, s, false);  // the potential problems were factored by their own setup above
  tune_cholesky(h, s);
  tune_sweeps(h, s);
  h.on_device = true;
}

// Device bytes riesz_setup_device will allocate for this handle (the sum of
// its device buffers, the internal potential-problem handle included), from
// the host plans alone: the same sizes as setup_device_impl, buffer by buffer,
// so that admission control can budget a request before it touches the GPU.
// *nalloc receives the number of device allocations (for the allocator's
// per-allocation rounding).
double plan_device_bytes(const riesz_handle& h, int64_t* nalloc) {
  const RefElement& R = *h.ref;
  const MeshMaps& M = h.mesh;
  const double n = M.nref, C = (double)M.ncells, N = (double)M.ndofs;
  const double nrhs = std::max(1, h.opts.nrhs_max);
  const double npatch = (double)h.p_n.size();
  double b = 0.0;
  int64_t na = 0;
  auto add = [&](double count, double size) {
    if (count > 0) {
      b += count * size;
      ++na;
    }
  };
  add((double)h.verts.size(), 8);
  add((double)M.cells.size(), 4);
  add(C * n, 4);                                   // cell_dofs
  add((double)R.R.size(), 8);
  add((double)R.Q * C, 8);                         // g
  add(C * 10, 8);                                  // jac
  add(nrhs * h.nif * C, 8);                        // Ycell
  add(std::max<double>(1, (double)M.n_interior), 8);
  add((double)h.sc_ptr.size(), 8);
  add((double)h.sc_pos.size(), 4);
  add((double)h.p_n.size(), 4);
  add((double)h.p_doff.size(), 8);
  add((double)h.p_foff.size(), 8);
  add((double)h.p_dofs.size(), 4);
  add((double)h.pz_ptr.size(), 8);
  add((double)h.pz_pos.size(), 4);
  add((double)h.pb_ptr.size(), 8);
  add((double)h.pb_off.size(), 8);
  add((double)h.pb_cell.size(), 4);
  add((double)h.pb_ent.size(), 4);
  add(std::max<double>(1, (double)h.p_dofs.size() * nrhs), 8);  // zpatch
  add((double)R.Xcross.size(), 8);
  add(C * h.refcg->nref, 4);                       // CG cell_dofs (load)
  for (int k = 0; k < 8; ++k) add(N * nrhs, 8);    // r, z, zold, p, Ap, tmp, xh, xw
  add(4, 4);                                       // ctl
  add(4, 4);                                       // flags
  add(2.0 * dev::RED_BLOCKS * nrhs, 8);            // part
  add(16 * nrhs, 8);                               // scal
  add(std::max<double>(1, npatch), 4);             // info
  if (h.opts.apply_mode == RIESZ_APPLY_ELEMENT) {
    add(C * n * n, 8);
    if (needs_ae32(h)) add(C * n * n, 4);
  }
  add((double)h.p_dioff.size(), 8);
  add((double)h.p_moff.size(), 8);
  add((double)h.p_meta.size(), 4);
  if (h.opts.dirichlet) add((double)h.dir_mask.size(), 1);
  if (h.ht) {
    int64_t na_aux = 0;
    b += plan_device_bytes(*h.aux, &na_aux);
    na += na_aux;
    add((double)h.gt_ptr.size(), 8);
    add((double)h.gt_idx.size(), 4);
    add((double)h.gt_sgn.size(), 4);
    add((double)h.gg_ptr.size(), 8);
    add((double)h.gg_idx.size(), 4);
    add((double)h.gg_sgn.size(), 4);
    add(nrhs * (double)h.aux->mesh.n_interface, 8);
    add(nrhs * (double)M.n_interface, 8);
  }
  if (h.coarse_on && h.coarse_sparse) {
    add((double)h.c_w.size(), 4);
    add((double)h.c_idx.size(), 4);
    add((double)h.c_aux.size(), 4);
    add(nrhs * h.N0, 8);  // zc
    int64_t na_c = 0;
    b += plan_device_bytes(*h.caux, &na_c);
    na += na_c;
  } else if (h.coarse_on) {
    const double N0p = h.N0p, CB = dev::CB;
    add((double)h.c_w.size(), 4);
    add((double)h.c_idx.size(), 4);
    add((double)h.c_ptr.size(), 8);
    add((double)h.c_J.size(), 4);
    add((double)h.c_cell.size(), 4);
    add((double)h.c_ab.size(), 4);
    {
      add(N0p * N0p, 8);
      add(N0p * N0p, 8);
      add(N0p * CB, 8);
      add(CB * N0p, 8);
      add(nrhs * N0p, 8);
      add(1, 4);
    }
    add(nrhs * h.N0, 8);
  }
  if (npatch > 0) {
    const double fe = (double)h.factor_entries, de = (double)h.dinv_entries;
    add(fe, 8);
    add(de, 8);
    if (h.opts.precond_precision == RIESZ_PREC_FP32) {
      add(fe, 4);
      if (nrhs > 1) {
        add(fe, 4);
        add(de, 4);
      }
      add(de, 4);
    }
  }
  if (h.opts.form == RIESZ_FORM_HYBRID)
    for (int k = 0; k < 3; ++k) add(N * nrhs, 8);  // sweep residual, correction, product
  if (needs_tc(h)) {  // split reference matrices in the tensor-core stage layout
    const double NP = (M.nref + 15) / 16 * 16, KC = (M.nref + dev::TC_KC - 1) / dev::TC_KC;
    add(KC * R.Q * 2 * NP * dev::TC_KC, 2);
  }
  add(nrhs, 4);  // ticket
  if (nalloc) *nalloc = na;
  return b;
}

void check_dev(const riesz_handle* h) {
  need(h != nullptr, "null handle");
  need(h->on_device, "handle has no device state (call riesz_setup_device)", RIESZ_ERR_NO_DEVICE);
}

// Host part of a handle: reference element, mesh maps and plans.  `internal`
// handles (the potential problems of the Hiptmair-Toselli decomposition) may
// have beta = 0.
riesz_handle* create_handle(int space, int p, int64_t nverts, const double* verts, int64_t ncells,
                            const int64_t* cells, const riesz_opts& opts, bool internal, bool apply_only = false) {
  need(space >= RIESZ_H1 && space <= RIESZ_HDIV2 && space != RIESZ_L2,
       "space must be RIESZ_H1, RIESZ_HCURL, RIESZ_HDIV, RIESZ_HCURL2 or RIESZ_HDIV2");
  const int kind = space >= RIESZ_HCURL2 ? 2 : 1;
  if (kind == 2) space -= RIESZ_HCURL2 - RIESZ_HCURL;  // k of the second-kind space
  // internal handles: the CG_{p+1} potentials of NedTwo_p reach degree 11
  need(p >= 1 && p <= (internal ? 11 : 10), "degree p must be in 1..10");
  need(verts && cells && nverts > 0 && ncells > 0, "empty mesh", RIESZ_ERR_BAD_MESH);
  auto t0 = std::chrono::steady_clock::now();
  auto h = std::make_unique<riesz_handle>();
  h->space = space;
  h->kind = kind;
  h->p = p;
  h->opts = opts;
  need(h->opts.rtol > 0 && h->opts.maxit >= 0 && h->opts.nrhs_max >= 1 && h->opts.nrhs_max <= 64, "bad options");
  need(h->opts.precond_precision == 0 || h->opts.precond_precision == 1, "bad precond_precision");
  need(h->opts.apply_mode == 0 || h->opts.apply_mode == 1, "bad apply_mode");
  h->apply_only = internal && apply_only;
  need((h->opts.alpha > 0 || (h->apply_only && h->opts.alpha == 0)) &&
           (h->opts.beta > 0 || (internal && h->opts.beta == 0)) && (h->opts.alpha > 0 || h->opts.beta > 0) &&
           std::isfinite(h->opts.alpha) && std::isfinite(h->opts.beta),
       "alpha and beta must be positive and finite");
  if (h->apply_only) h->opts.coarse = 0;
  need(h->opts.apply_precision >= RIESZ_PREC_FP64 && h->opts.apply_precision <= RIESZ_PREC_BF16X3,
       "bad apply_precision");
  need(h->opts.loop == RIESZ_LOOP_HOST || h->opts.loop == RIESZ_LOOP_GRAPH, "bad loop");
  need(h->opts.autotune >= 0 && h->opts.autotune <= 2, "bad autotune");
  need(h->opts.coarse >= 0 && h->opts.coarse <= 2, "bad coarse");
  need(h->opts.coarse_its >= 1 && h->opts.coarse_its <= 1000, "coarse_its must be in 1..1000");
  need(!h->opts.dirichlet_vertices || h->opts.dirichlet, "dirichlet_vertices needs dirichlet = 1");
  need(h->opts.replace_digits >= 0 && h->opts.replace_digits <= 12, "replace_digits must be in 0..12");
  need(h->opts.form == RIESZ_FORM_ADDITIVE || h->opts.form == RIESZ_FORM_HYBRID, "bad form");
  need(h->opts.dirichlet == 0 || h->opts.dirichlet == 1, "bad dirichlet");
  need(h->opts.decomposition >= RIESZ_DECOMP_VERTEX_STAR && h->opts.decomposition <= RIESZ_DECOMP_EDGE_STAR,
       "bad decomposition");
  need(h->opts.decomposition != RIESZ_DECOMP_HT || (space == RIESZ_HCURL && !h->opts.dirichlet),
       "the Hiptmair-Toselli decomposition is for H(curl) without Dirichlet conditions");
  need(h->opts.decomposition != RIESZ_DECOMP_EDGE_STAR || space == RIESZ_HDIV,
       "the edge-star decomposition (PAFW_1) is for H(div)");
  for (int64_t i = 0; i < nverts * 3; ++i)
    need(std::isfinite(verts[i]), "non-finite vertex coordinate", RIESZ_ERR_BAD_MESH);
  h->verts.assign(verts, verts + nverts * 3);
  try {
    h->ref = &reference_element(space, p, kind);
    h->refcg = &reference_element(RIESZ_H1, p);
    h->mesh = build_mesh(*h->ref, nverts, ncells, cells);
    h->meshcg = (space == RIESZ_H1) ? h->mesh : build_mesh(*h->refcg, nverts, ncells, cells);
    if (kind == 2 && h->opts.decomposition == RIESZ_DECOMP_HT)
      h->meshpot = build_mesh(reference_element(RIESZ_H1, p + 1), nverts, ncells, cells);
  } catch (const Err&) {
    throw;
  } catch (const std::exception& e) {
    throw Err(RIESZ_ERR_BAD_MESH, e.what());
  }
  need(h->opts.apply_precision != RIESZ_PREC_BF16X3 || h->mesh.nref <= dev::TC_MAXN,
       "the BF16x3 tensor-core products hold n_ref <= 1024 accumulators per row (degree too high)");
  if (h->opts.dirichlet) plan_dirichlet(*h);
  if (h->opts.decomposition == RIESZ_DECOMP_HT) plan_ht(*h);
  if (h->opts.decomposition == RIESZ_DECOMP_EDGE_STAR) plan_edge_stars(*h, 0, h->mesh.per_entity[2]);
  build_plans(*h);
  plan_coarse(*h, internal);  // the internal handles with a coarse space are the Hodge-Laplace blocks
  if (h->coarse_on && h->coarse_sparse) {  // W^k = the lowest-order space (Whitney forms, Lemma 4.1, for either kind): its own p = 1 handle
    riesz_opts co = h->opts;
    co.coarse = 0;
    co.form = RIESZ_FORM_ADDITIVE;
    co.decomposition = RIESZ_DECOMP_VERTEX_STAR;
    // FP32 patch sweeps (the coarse steps are approximate anyway, and FP64 arithmetic runs at ~1/40 of
    // the FP32 rate on GB300), FP64 products, residuals and inner products
    co.precond_precision = RIESZ_PREC_FP32;
    co.apply_precision = RIESZ_PREC_FP64;
    co.apply_mode = RIESZ_APPLY_ELEMENT;
    co.autotune = 0;
    h->caux = create_handle(space, 1, nverts, verts, ncells, cells, co, true);
    if (h->caux->N() < (int64_t)h->c_w.size()) throw Err(RIESZ_ERR_INTERNAL, "lowest-order handle too small");
  }
  if (h->ht) {  // potential problems: CG_p (CG_{p+1} for NedTwo_p) on the same mesh, a = beta (grad, grad), vertex stars
    riesz_opts ao = h->opts;
    ao.alpha = h->opts.beta;
    ao.beta = 0.0;
    ao.coarse = 0;
    ao.dirichlet = 0;
    ao.decomposition = RIESZ_DECOMP_VERTEX_STAR;
    ao.apply_precision = RIESZ_PREC_FP64;
    ao.apply_mode = RIESZ_APPLY_ELEMENT;
    h->aux = create_handle(RIESZ_H1, kind == 2 ? p + 1 : p, nverts, verts, ncells, cells, ao, true);
  }
  h->opts.dirichlet_vertices = nullptr;  // the caller's array is read during creation only
  h->setup_host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return h.release();
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch for riesz_apply_noalloc: a file-scope device array, so that entry
// point never allocates.  Every device that loads this library reserves it
// until the process exits.  Its host-side name is not a device address: the
// address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
#define RIESZ_NOALLOC_SCRATCH_DOUBLES (1 << 21)
static __device__ __align__(256) double g_noalloc_scratch[RIESZ_NOALLOC_SCRATCH_DOUBLES];

namespace {
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (looked up on first use).
double* noalloc_scratch(int device) {
  if (device < 0 || device >= kMaxDevices) throw Err(RIESZ_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* ptr = nullptr;
    CK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_noalloc_ptr[device] = static_cast<double*>(ptr);
  }
  return g_noalloc_ptr[device];
}
}  // namespace

extern "C" {

void riesz_default_opts(riesz_opts* o) {
  if (!o) return;
  o->precond_precision = RIESZ_PREC_FP64;
  o->apply_mode = RIESZ_APPLY_ELEMENT;
  o->rtol = 1e-8;
  o->maxit = 1000;
  o->nrhs_max = 1;
  o->alpha = 1.0;
  o->beta = 1.0;
  o->apply_precision = RIESZ_PREC_FP64;
  o->loop = RIESZ_LOOP_GRAPH;
  o->autotune = 1;
  o->coarse = 1;
  o->dirichlet = 0;
  o->decomposition = RIESZ_DECOMP_VERTEX_STAR;
  o->form = RIESZ_FORM_ADDITIVE;
  o->coarse_its = 4;
  o->dirichlet_vertices = nullptr;
  o->replace_digits = 0;
}

const char* riesz_last_error(void) { return g_err.c_str(); }

int riesz_create(int space, int p, int64_t nverts, const double* verts, int64_t ncells, const int64_t* cells,
                 const riesz_opts* opts, riesz_handle** out) {
  return guarded([&] {
    need(out != nullptr, "out is NULL");
    *out = nullptr;
    riesz_opts o;
    riesz_default_opts(&o);
    if (opts) o = *opts;
    *out = create_handle(space, p, nverts, verts, ncells, cells, o, false);
  });
}

int riesz_num_dofs(const riesz_handle* h, int64_t* n, int64_t* n_interior) {
  return guarded([&] {
    need(h != nullptr, "null handle");
    if (n) *n = h->mesh.ndofs;
    if (n_interior) *n_interior = h->mesh.n_interior;
  });
}

int riesz_num_cg_dofs(const riesz_handle* h, int64_t* n_cg) {
  return guarded([&] {
    need(h != nullptr && n_cg != nullptr, "null argument");
    *n_cg = h->meshcg.ndofs;
  });
}

int riesz_ref_info(const riesz_handle* h, int* info) {
  return guarded([&] {
    need(h != nullptr && info != nullptr, "null argument");
    const RefElement& R = *h->ref;
    info[0] = R.nref;
    info[1] = R.ninterior;
    info[2] = R.ncomp;
    info[3] = R.dcomp;
    for (int d = 0; d < 4; ++d) info[4 + d] = R.per_entity[d];
  });
}

int riesz_dof_map(const riesz_handle* h, int32_t* cell_dofs) {
  return guarded([&] {
    need(h != nullptr && cell_dofs != nullptr, "null argument");
    std::memcpy(cell_dofs, h->mesh.cell_dofs.data(), h->mesh.cell_dofs.size() * sizeof(int32_t));
  });
}

int riesz_patch_count(const riesz_handle* h, int64_t* npatches) {
  return guarded([&] {
    need(h != nullptr && npatches != nullptr, "null argument");
    *npatches = h->edge_star ? (int64_t)h->es_ptr.size() - 1 : (int64_t)h->mesh.patch_ptr.size() - 1;
  });
}

int riesz_patch_map(const riesz_handle* h, int64_t* offsets, int32_t* dofs) {
  return guarded([&] {
    need(h != nullptr && offsets != nullptr, "null argument");
    const std::vector<int64_t>& ptr = h->edge_star ? h->es_ptr : h->mesh.patch_ptr;
    const std::vector<int32_t>& d = h->edge_star ? h->es_dofs : h->mesh.patch_dofs;
    std::memcpy(offsets, ptr.data(), ptr.size() * sizeof(int64_t));
    if (dofs) std::memcpy(dofs, d.data(), d.size() * sizeof(int32_t));
  });
}

int riesz_ht_gradient_map(const riesz_handle* h, int64_t* ptr, int32_t* idx, float* sgn) {
  return guarded([&] {
    need(h != nullptr && ptr != nullptr, "null argument");
    need(h->ht, "not a Hiptmair-Toselli handle");
    std::copy(h->gg_ptr.begin(), h->gg_ptr.end(), ptr);
    if (idx) std::copy(h->gg_idx.begin(), h->gg_idx.end(), idx);
    if (sgn) std::copy(h->gg_sgn.begin(), h->gg_sgn.end(), sgn);
  });
}

int riesz_ref_tabulate(int space, int p, int64_t npts, const double* pts, double* vals, double* dvals) {
  return guarded([&] {
    need(space >= 0 && space <= RIESZ_HDIV2 && p >= 1 && p <= 10, "bad space or degree");
    need(npts >= 0 && (npts == 0 || pts != nullptr), "bad points");
    if (space == RIESZ_L2) {  // DG_{p-1}: values only, d = 0
      const int n = dg_dim(p);
      if (vals) dg_tabulate(p, (int)npts, pts, vals);
      if (dvals) std::fill(dvals, dvals + (size_t)npts * n, 0.0);
      return;
    }
    if (space >= RIESZ_HCURL2)
      reference_element(space - (RIESZ_HCURL2 - RIESZ_HCURL), p, 2).tabulate((int)npts, pts, vals, dvals);
    else
      reference_element(space, p).tabulate((int)npts, pts, vals, dvals);
  });
}

int riesz_ref_mixed_tables(int k, int p, double* out) {
  return guarded([&] {
    need(k >= 1 && k <= 3, "k must be 1, 2 or 3");
    need(p >= 1 && p <= 10, "degree p must be in 1..10");
    need(out != nullptr, "null output");
    const std::vector<double>& R = mixed_reference_tables(k, p);
    std::copy(R.begin(), R.end(), out);
  });
}

int riesz_setup_device(riesz_handle* h, void* stream) {
  return guarded([&] {
    need(h != nullptr, "null handle");
    setup_device_impl(*h, S(stream));
  });
}

int riesz_setup(int space, int p, int64_t nverts, const double* verts, int64_t ncells, const int64_t* cells,
                const riesz_opts* opts, void* stream, riesz_handle** out) {
  int rc = riesz_create(space, p, nverts, verts, ncells, cells, opts, out);
  if (rc != RIESZ_OK) return rc;
  rc = riesz_setup_device(*out, stream);
  if (rc != RIESZ_OK) {
    delete *out;
    *out = nullptr;
  }
  return rc;
}

int riesz_apply(riesz_handle* h, const double* x, double* y, int nrhs, void* stream) {
  return guarded([&] {
    check_dev(h);
    need(x && y && nrhs >= 1 && nrhs <= h->opts.nrhs_max, "bad apply arguments");
    op_apply(*h, x, y, nrhs, S(stream));
  });
}

int riesz_apply_noalloc(riesz_handle* h, const double* x, double* y, void* stream) {
  return guarded([&] {
    check_dev(h);
    need(x && y, "null argument");
    int device = -1;
    CK(cudaGetDevice(&device));
    need(device == h->device, "the current CUDA device is not the handle's device");
    const int64_t C = h->C(), N = h->N();
    const int n = h->mesh.nref;
    const int64_t need_doubles = (int64_t)h->nif * C;
    if (need_doubles > RIESZ_NOALLOC_SCRATCH_DOUBLES)
      throw Err(RIESZ_ERR_INVALID_ARG,
                "riesz_apply_noalloc: interface DOFs per cell x cells = " + std::to_string(need_doubles) +
                    " exceeds the fixed scratch of " + std::to_string(RIESZ_NOALLOC_SCRATCH_DOUBLES) + " doubles");
    double* ycell = noalloc_scratch(device);
    cudaStream_t s = S(stream);
    // same kernels as riesz_apply with nrhs = 1; every scratch slot read by the
    // gather is written by the contraction of the same call, so no clearing
    if (h->opts.apply_mode == RIESZ_APPLY_ELEMENT) {
      const int rows = (n % 2 == 0) ? n / 2 : n;
      const int nt = std::min(1024, (rows + 31) / 32 * 32);
      launch(*h, RIESZ_K_APPLY, s, [&] {
        dev::k_apply_elem<double, 1><<<(unsigned)C, nt, (size_t)n * sizeof(double), s>>>(C, n, h->nif, h->d_Ae.p, h->d_cdofs.p,
                                                                              x, y, ycell, 1, N, h->dmask());
      });
    } else {
      const size_t sm = ((size_t)n + h->ref->Q) * dev::TC * sizeof(double);
      dim3 grid(nblk(C, dev::TC), 1);
      launch(*h, RIESZ_K_APPLY, s, [&] {
        dev::k_apply_mf<<<grid, dev::NT, sm, s>>>(C, n, h->nif, h->ref->Q, h->d_R.p, h->d_g.p, h->d_cdofs.p, x, y,
                                                 ycell, N, h->dmask());
      });
    }
    const int64_t nI = h->mesh.n_interface;
    launch(*h, RIESZ_K_GATHER, s, [&] {
      dev::k_gather_iface<<<nblk(nI, 256), 256, 0, s>>>(nI, h->d_sc_ptr.p, h->d_sc_pos.p, ycell, (int64_t)h->nif * C,
                                                       y, N, 1, h->dmask(), x);
    });
  });
}

int riesz_precond(riesz_handle* h, const double* r, double* z, int nrhs, void* stream) {
  return guarded([&] {
    check_dev(h);
    need(r && z && nrhs >= 1 && nrhs <= h->opts.nrhs_max, "bad precond arguments");
    op_precond(*h, r, z, nrhs, S(stream));
  });
}

int riesz_solve(riesz_handle* h, const double* b, double* x, int nrhs, void* stream, int* iters, double* relres) {
  int status = RIESZ_OK;
  int rc = guarded([&] {
    check_dev(h);
    need(b && x && nrhs >= 1, "bad solve arguments");
    need(nrhs <= h->opts.nrhs_max, "nrhs exceeds opts.nrhs_max");
    status = solve_one(*h, b, x, nrhs, S(stream), iters, relres);
  });
  return rc != RIESZ_OK ? rc : status;
}

int riesz_solve_batch(riesz_handle* const* hs, int count, const double* const* b, double* const* x,
                      const int* nrhs, void* stream, int* iters, double* relres, int* status) {
  int first = RIESZ_OK;
  int rc = guarded([&] {
    need(count >= 0 && (count == 0 || (hs && b && x)), "bad batch arguments");
    int dev_now = 0;
    CK(cudaGetDevice(&dev_now));
    std::vector<LoopSolve> Ls(count);
    for (int i = 0; i < count; ++i) {
      check_dev(hs[i]);
      need(hs[i]->device == dev_now, "a handle of the batch is not on the current CUDA device");
      for (int j = 0; j < i; ++j) need(hs[j] != hs[i], "a handle appears twice in the batch");
      const int nr = nrhs ? nrhs[i] : 1;
      need(b[i] && x[i] && nr >= 1 && nr <= hs[i]->opts.nrhs_max, "bad solve arguments in the batch");
      need(!profiling_loop(*hs[i]), "the profiler records loop kernels on a handle of the batch");
      Ls[i].h = hs[i];
      Ls[i].b = b[i];
      Ls[i].x = x[i];
      Ls[i].nrhs = nr;
    }
    if (count == 0) return;
    solve_graph(Ls, S(stream));
    int off = 0;
    for (int i = 0; i < count; ++i) {
      const LoopSolve& L = Ls[i];
      for (int k = 0; k < L.nrhs; ++k, ++off) {
        if (iters) iters[off] = L.it_before;
        if (relres) relres[off] = L.bb[k] > 0 ? std::sqrt(ls_scal(L, k, dev::S_RR) / L.bb[k]) : 0.0;
      }
      if (status) status[i] = L.status;
      if (L.status != RIESZ_OK && first == RIESZ_OK) {
        first = L.status;
        g_err = "system " + std::to_string(i) + ": " + L.err;
      }
    }
  });
  return rc != RIESZ_OK ? rc : first;
}

int riesz_solve_host(riesz_handle* h, const double* b_host, double* x_host, int nrhs, void* stream, int* iters,
                     double* relres) {
  int status = RIESZ_OK;
  int rc = guarded([&] {
    check_dev(h);
    need(b_host && x_host && nrhs >= 1 && nrhs <= h->opts.nrhs_max, "bad solve arguments");
    const int64_t N = h->N();
    cudaStream_t s = S(stream);
    double* db = h->d_tmp.p;  // staging of b
    double* dx = h->d_xh.p;   // staging of x
    CK(cudaMemcpyAsync(db, b_host, (size_t)N * nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dx, x_host, (size_t)N * nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    status = solve_one(*h, db, dx, nrhs, s, iters, relres);
    CK(cudaMemcpyAsync(x_host, dx, (size_t)N * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  });
  return rc != RIESZ_OK ? rc : status;
}

int riesz_load(riesz_handle* h, const double* fcg, double* b, void* stream) {
  return guarded([&] {
    check_dev(h);
    need(fcg && b, "null argument");
    const int64_t C = h->C(), N = h->N();
    const int n = h->mesh.nref;
    const int ncomp = (h->space == RIESZ_H1) ? 1 : 3;
    const size_t sm = (size_t)ncomp * h->refcg->nref * sizeof(double);
    cudaStream_t s = S(stream);
    launch(*h, RIESZ_K_LOAD, s, [&] {
      dev::k_load<<<(unsigned)C, 256, sm, s>>>(h->space, C, n, h->nif, h->refcg->nref, h->d_jac.p, h->d_cgdofs.p, fcg,
                                             h->meshcg.ndofs, h->d_X.p, h->d_cdofs.p, b, h->d_Ycell.p);
    });
    const int64_t nI = h->mesh.n_interface;
    launch(*h, RIESZ_K_GATHER, s, [&] {
      dev::k_gather_iface<<<nblk(nI, 256), 256, 0, s>>>(nI, h->d_sc_ptr.p, h->d_sc_pos.p, h->d_Ycell.p,
                                                       (int64_t)h->nif * C, b, N, 1, h->dmask(), nullptr);
    });
  });
}

int riesz_update_geometry(riesz_handle* h, const double* verts, void* stream) {
  return guarded([&] {
    check_dev(h);
    need(verts != nullptr, "null vertex array");
    cudaStream_t s = S(stream);
    CK(cudaMemcpyAsync(h->d_verts.p, verts, h->d_verts.bytes(), cudaMemcpyDeviceToDevice, s));
    device_compute(*h, s);
  });
}

int riesz_update_geometry_batch(riesz_handle* const* hs, int count, const double* const* verts, void* stream) {
  return guarded([&] {
    need(count >= 0 && (count == 0 || (hs && verts)), "bad batch arguments");
    int dev_now = 0;
    CK(cudaGetDevice(&dev_now));
    for (int i = 0; i < count; ++i) {
      check_dev(hs[i]);
      need(hs[i]->device == dev_now, "a handle of the batch is not on the current CUDA device");
      need(verts[i] != nullptr, "null vertex array in the batch");
      for (int j = 0; j < i; ++j) need(hs[j] != hs[i], "a handle appears twice in the batch");
    }
    if (count == 0) return;
    cudaStream_t s = S(stream);
    cudaEvent_t fork;
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    CK(cudaEventRecord(fork, s));
    // 1. every system's setup up to its assembled patch matrices, on a stream of its own
    for (int i = 0; i < count; ++i) {
      riesz_handle& h = *hs[i];
      if (!h.batch_stream) CK(cudaStreamCreateWithFlags(&h.batch_stream, cudaStreamNonBlocking));
      if (!h.ev_batch) CK(cudaEventCreateWithFlags(&h.ev_batch, cudaEventDisableTiming));
      CK(cudaStreamWaitEvent(h.batch_stream, fork, 0));
      CK(cudaMemcpyAsync(h.d_verts.p, verts[i], h.d_verts.bytes(), cudaMemcpyDeviceToDevice, h.batch_stream));
      device_compute_pre(h, h.batch_stream, h.aux != nullptr);
      CK(cudaEventRecord(h.ev_batch, h.batch_stream));
      CK(cudaStreamWaitEvent(s, h.ev_batch, 0));
    }
    // 2. all systems' patch factorisations in one persistent launch, largest patches first
    std::vector<dev::CholJob> jobs;
    for (int i = 0; i < count; ++i) {
      const riesz_handle& h = *hs[i];
      for (size_t P = 0; P < h.p_n.size(); ++P)
        jobs.push_back({h.d_meta.p + h.p_moff[P], h.d_L64.p + h.p_foff[P], h.d_D64.p + h.p_dioff[P],
                        h.d_info.p + P, h.p_n[P], 0});
    }
    std::stable_sort(jobs.begin(), jobs.end(), [](const dev::CholJob& a, const dev::CholJob& b) { return a.n > b.n; });
    struct JobBuf {  // the work list; freed on every exit (after the synchronisation below on success)
      unsigned char* p = nullptr;
      ~JobBuf() {
        if (p) cudaFree(p);
      }
    } jbuf;
    if (!jobs.empty()) {
      const size_t jb = jobs.size() * sizeof(dev::CholJob);
      CK(cudaMalloc((void**)&jbuf.p, jb + sizeof(int)));
      int* next = reinterpret_cast<int*>(jbuf.p + jb);
      CK(cudaMemcpyAsync(jbuf.p, jobs.data(), jb, cudaMemcpyHostToDevice, s));
      CK(cudaMemsetAsync(next, 0, sizeof(int), s));
      int occ = 0, nsm = 0;
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dev::k_cholesky_many, dev::NT, 0));
      CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev_now));
      const int grid = (int)std::min<size_t>(jobs.size(), (size_t)std::max(1, occ) * nsm);
      dev::k_cholesky_many<<<grid, dev::NT, 0, s>>>(reinterpret_cast<const dev::CholJob*>(jbuf.p), (int)jobs.size(),
                                                     next);
      KCHECK();
      ++hs[0]->launches;
    }
    CK(cudaEventRecord(fork, s));
    // 3. each system's FP32 factor copies and joins, on its own stream again
    for (int i = 0; i < count; ++i) {
      riesz_handle& h = *hs[i];
      CK(cudaStreamWaitEvent(h.batch_stream, fork, 0));
      device_compute_post(h, h.batch_stream, h.aux != nullptr);
      CK(cudaEventRecord(h.ev_batch, h.batch_stream));
      CK(cudaStreamWaitEvent(s, h.ev_batch, 0));
    }
    cudaEventDestroy(fork);
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i) {  // the host checks of a single setup, system by system
      riesz_handle& h = *hs[i];
      check_factor_info(h, s);
      if (h.aux) check_factor_info(*h.aux, s);
      if (h.caux && h.coarse_on) check_factor_info(*h.caux, s);
      hybrid_weights(h, s);
    }
  });
}

int riesz_dirichlet_map(const riesz_handle* h, uint8_t* mask) {
  return guarded([&] {
    need(h != nullptr && mask != nullptr, "null argument");
    const int64_t N = h->mesh.ndofs;
    std::fill(mask, mask + N, (uint8_t)0);
    if (h->opts.dirichlet) std::copy(h->dir_mask.begin(), h->dir_mask.end(), mask);
  });
}

int riesz_tuning(const riesz_handle* h, int* out) {
  return guarded([&] {
    check_dev(h);
    need(out != nullptr, "null argument");
    out[0] = h->chol_ctas;
    out[1] = h->chol_tuned;
    out[2] = h->coarse_on ? h->N0 : 0;
    out[3] = h->chol_split;
    out[4] = !h->coarse_on ? 0 : (h->coarse_sparse ? 2 : 1);
  });
}

int riesz_sweep_shape(const riesz_handle* h, int* shape, int* timed) {
  return guarded([&] {
    check_dev(h);
    need(shape != nullptr, "null argument");
    const bool applies = h->opts.precond_precision == RIESZ_PREC_FP32 && h->opts.nrhs_max > 1 && !h->p_n.empty() &&
                         (h->p_n[0] + 31) / 32 <= dev::WARP_NB && (h->p_n[0] + 31) / 32 > dev::SMALL_NB;
    *shape = applies ? h->sweep_shape : -1;
    if (timed) *timed = h->sweep_tuned;
  });
}

int riesz_profile(riesz_handle* h, int enable) {
  return guarded([&] {
    need(h != nullptr, "null handle");
    // the potential problems' kernels are reported with the handle's own kinds; the kernels of the
    // lowest-order coarse handle as RIESZ_K_COARSE (its setup) and RIESZ_K_COARSE_APPLY (its PCG steps)
    const unsigned mask = (unsigned)enable;
    unsigned cmask = 0;
    if (mask & (1u << RIESZ_K_COARSE)) cmask |= ~LOOP_KINDS;
    if (mask & (1u << RIESZ_K_COARSE_APPLY)) cmask |= LOOP_KINDS;
    for (riesz_handle* x : {h, h->aux, h->caux}) {
      if (!x) continue;
      if (!x->prof_pending.empty()) prof_collect(*x);
      const unsigned m = x == h->caux ? cmask : mask;
      x->prof = m != 0;
      x->prof_mask = m;
      for (int k = 0; k < RIESZ_NKIND; ++k) {
        x->prof_ms[k] = 0.0;
        x->prof_cnt[k] = 0;
      }
    }
  });
}

int riesz_profile_read(riesz_handle* h, double* ms, int64_t* counts) {
  return guarded([&] {
    need(h != nullptr, "null handle");
    prof_collect(*h);
    if (h->aux) prof_collect(*h->aux);
    if (h->caux) prof_collect(*h->caux);
    for (int k = 0; k < RIESZ_NKIND; ++k) {
      if (ms) ms[k] = h->prof_ms[k] + (h->aux ? h->aux->prof_ms[k] : 0.0);
      if (counts) counts[k] = h->prof_cnt[k] + (h->aux ? h->aux->prof_cnt[k] : 0);
    }
    if (h->caux) {
      for (int k = 0; k < RIESZ_NKIND; ++k) {
        const int to = ((LOOP_KINDS >> k) & 1u) ? RIESZ_K_COARSE_APPLY : RIESZ_K_COARSE;
        if (ms) ms[to] += h->caux->prof_ms[k];
        if (counts) counts[to] += h->caux->prof_cnt[k];
      }
    }
  });
}

int riesz_stats(const riesz_handle* h, double* out) {
  return guarded([&] {
    need(h != nullptr && out != nullptr, "null argument");
    out[0] = h->setup_host_ms;
    out[1] = h->setup_dev_ms;
    out[2] = (double)h->device_bytes();
    out[3] = (double)(h->factor_entries + h->dinv_entries) * (h->opts.precond_precision == RIESZ_PREC_FP32 ? 4.0 : 8.0);
    out[4] = h->last_iters;
    out[5] = (double)(h->launches + (h->aux ? h->aux->launches : 0) + (h->caux ? h->caux->launches : 0));
    out[6] = h->chol_flops + (h->aux ? h->aux->chol_flops : 0.0);
    const double fb = h->opts.precond_precision == RIESZ_PREC_FP32 ? 4.0 : 8.0;
    out[7] = 2.0 * (double)(h->factor_entries + h->dinv_entries) * fb + (double)h->p_dofs.size() * 20.0;
  });
}

int riesz_probe_fp64(int iters, void* stream, double* tflops) {
  return guarded([&] {
    need(tflops != nullptr && iters >= 1 && iters <= (1 << 24), "iters must be in 1..2^24");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 4 * nsm, threads = 256;
    DBuf<double> out;
    out.alloc((size_t)blocks * threads);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float ms = 0.f;
    cudaError_t rc = cudaSuccess;
    dev::k_fp64_probe<<<blocks, threads, 0, s>>>(std::min(iters, 1024), 0.999999, 1e-7, out.p);  // warm-up
    rc = cudaEventRecord(e0, s);
    if (rc == cudaSuccess) {
      dev::k_fp64_probe<<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7, out.p);
      rc = cudaGetLastError();
    }
    if (rc == cudaSuccess) rc = cudaEventRecord(e1, s);
    if (rc == cudaSuccess) rc = cudaEventSynchronize(e1);
    if (rc == cudaSuccess) rc = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(rc);
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
  });
}

int riesz_apply_prec(riesz_handle* h, const double* x, double* y, int nrhs, int prec, void* stream) {
  return guarded([&] {
    check_dev(h);
    need(x && y && x != y, "x and y must be distinct device arrays");
    need(nrhs >= 1 && nrhs <= h->opts.nrhs_max, "nrhs out of range");
    need(prec == RIESZ_PREC_FP64 || (prec == RIESZ_PREC_FP32 && h->d_Ae32.p) || (prec == RIESZ_PREC_BF16X3 && h->d_Btc.p),
         "precision not held by this handle (FP32: FP32 element matrices; BF16X3: apply_precision BF16X3)");
    op_apply(*h, x, y, nrhs, S(stream), prec);
    KCHECK();
  });
}

int riesz_hybrid_weights(riesz_handle* h, double* rho, int set) {
  return guarded([&] {
    need(h != nullptr && rho != nullptr, "null argument");
    need(h->opts.form == RIESZ_FORM_HYBRID, "the handle does not use the hybrid form");
    if (set) {
      for (int m = 0; m < 3; ++m) need(rho[m] > 0.0 && std::isfinite(rho[m]), "weights must be positive");
      for (int m = 0; m < 3; ++m) h->rho[m + 1] = rho[m];
      h->rho_fixed = true;
      h->drop_graphs();
    } else {
      for (int m = 0; m < 3; ++m) rho[m] = h->rho[m + 1];
    }
  });
}

int riesz_plan_bytes(const riesz_handle* h, double* bytes, int64_t* nalloc) {
  return guarded([&] {
    need(h != nullptr && bytes != nullptr, "null argument");
    *bytes = plan_device_bytes(*h, nalloc);
  });
}

int riesz_destroy(riesz_handle* h) {
  return guarded([&] { delete h; });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Hodge-Laplace problems of Section 7.2 (Eq. (7.5)) for k = 1 (CG_p x Ned1_p)
// and k = 2 (Ned1_p x RT_p): block vectors [sigma (n0) | u (n1)], the block
// operator [-M_{k-1} B^T; B K_k], the block-diagonal augmented-Lagrangian
// preconditioner of Eq. (7.6) with each weighted Riesz map replaced by its
// Schwarz preconditioner, and preconditioned MINRES on the device.
// ---------------------------------------------------------------------------
struct riesz_hodge {
  int k = 0, p = 0;
  double gamma = 1.0, rtol = 1e-8;
  int maxit = 1000;
  riesz_handle* P0 = nullptr;  // X^{k-1}: (sigma, tau) + gamma (d sigma, d tau), preconditioner block
  riesz_handle* P1 = nullptr;  // X^k: gamma^{-1} (u, v) + (d u, d v), preconditioner block
  riesz_handle* Mh = nullptr;  // X^{k-1} mass (operator only)
  riesz_handle* Kh = nullptr;  // X^k d-stiffness (operator only; none for k = 3, where d^3 = 0)
  int64_t n0 = 0, n1 = 0;
  // k = 3: X^3 = DG_{p-1}, cell-major DOFs; no handle: its cell map, reference mass diagonal, load
  // cross table (CG_p -> DG) and the exact inverse of the block gamma^{-1} M_DG
  int n_dg = 0;
  DBuf<int32_t> d_dg_cd;
  DBuf<double> d_dg_mhat, d_dg_X, d_dg_dinv;
  int64_t launches = 0;
  int last_iters = 0;
  double last_relres = 0.0, last_phi = 0.0;
  DBuf<double> d_R, d_gB, d_jacB, d_Be;                   // coupling tables, factors, element matrices
  DBuf<double> v, vp, u, w, z, d1, d2, d_m, d_part;       // MINRES vectors and scalars
  DBuf<double> xw;                                          // working copy of x (device-driven loop)
  DBuf<unsigned> d_ticket;
  DBuf<int> d_ctl;                                          // loop control: iterations, limit, reason
  double* h_m = nullptr;
  int* h_ctl = nullptr;
  int loop = RIESZ_LOOP_GRAPH;
  // device-driven loop: a CUDA graph WHILE { iteration, control, IF { iteration, control } } (two
  // iterations per pass so that the Lanczos and direction buffers return to their roles), its
  // capture stream, and the kernels one iteration launches
  cudaGraphExec_t g_loop = nullptr;
  cudaStream_t cap = nullptr;
  int64_t g_iter_launches = 0;
  // the second block preconditioner runs on its own stream beside the first
  cudaStream_t s1 = nullptr;
  cudaEvent_t ev_f = nullptr, ev_j = nullptr;
  ~riesz_hodge() {
    if (g_loop) cudaGraphExecDestroy(g_loop);
    if (cap) cudaStreamDestroy(cap);
    if (h_ctl) cudaFreeHost(h_ctl);
    if (h_m) cudaFreeHost(h_m);
    if (s1) cudaStreamDestroy(s1);
    if (ev_f) cudaEventDestroy(ev_f);
    if (ev_j) cudaEventDestroy(ev_j);
    for (auto* b : {&d_R, &d_gB, &d_jacB, &d_Be, &v, &vp, &u, &w, &z, &d1, &d2, &d_m, &d_part, &d_dg_mhat, &d_dg_X,
                    &d_dg_dinv, &xw})
      b->free();
    d_ticket.free();
    d_ctl.free();
    d_dg_cd.free();
    delete P0;
    delete P1;
    delete Mh;
    delete Kh;
  }
  int64_t N() const { return n0 + n1; }
  int64_t sub_launches() const {
    int64_t l = 0;
    for (riesz_handle* x : {P0, P1, Mh, Kh})
      if (x) l += x->launches + (x->aux ? x->aux->launches : 0);
    return l;
  }
};

namespace {

void hodge_geometry(riesz_hodge& H, cudaStream_t s) {
  riesz_handle& M = *H.Mh;
  const int64_t C = M.C();
  if (H.k == 3) {
    // RT_p factors with alpha = 1, beta = 0: g[6] = 1 / |det J|, the single coupling factor
    dev::k_geom<<<nblk(C, 128), 128, 0, s>>>(2, C, M.d_verts.p, M.d_cells.p, ref_edge_inverse(), 1.0, 0.0,
                                            H.d_gB.p, H.d_jacB.p);
    CK(cudaGetLastError());
    dev::k_mixed_elem<<<(unsigned)C, 256, 0, s>>>(C, M.mesh.nref, H.n_dg, 1, H.d_gB.p + 6 * C, H.d_R.p, H.d_Be.p);
    CK(cudaGetLastError());
    dev::k_dg_diag<<<nblk(C * H.n_dg, 256), 256, 0, s>>>(C, H.n_dg, H.d_jacB.p, H.d_dg_mhat.p, H.gamma,
                                                        H.d_dg_dinv.p);
    CK(cudaGetLastError());
    H.launches += 3;
    return;
  }
  // the X^k mass factors (beta = 1, alpha = 0) are the metric of the coupling
  dev::k_geom<<<nblk(C, 128), 128, 0, s>>>(H.k, C, M.d_verts.p, M.d_cells.p, ref_edge_inverse(), 0.0, 1.0, H.d_gB.p,
                                          H.d_jacB.p);
  CK(cudaGetLastError());
  dev::k_mixed_elem<<<(unsigned)C, 256, 0, s>>>(C, M.mesh.nref, H.Kh->mesh.nref, 6, H.d_gB.p, H.d_R.p, H.d_Be.p);
  CK(cudaGetLastError());
  H.launches += 2;
}

void hodge_apply(riesz_hodge& H, const double* x, double* y, cudaStream_t s) {
  riesz_handle& M = *H.Mh;
  riesz_handle* K = H.Kh;  // null for k = 3
  const int64_t C = M.C();
  const int n0 = M.mesh.nref, n1 = K ? K->mesh.nref : H.n_dg;
  const size_t sm = dev::hodge_apply_smem(dev::NT, n0, n1);
  dev::k_hodge_apply<<<(unsigned)C, dev::NT, sm, s>>>(
      C, n0, n1, M.nif, K ? K->nif : 0, M.d_Ae.p, K ? K->d_Ae.p : nullptr, H.d_Be.p, M.d_cdofs.p,
      K ? K->d_cdofs.p : H.d_dg_cd.p, x, x + H.n0, y, y + H.n0, M.d_Ycell.p, K ? K->d_Ycell.p : nullptr);
  CK(cudaGetLastError());
  const int64_t nI0 = M.mesh.n_interface;
  dev::k_gather_iface<<<nblk(nI0, 256), 256, 0, s>>>(nI0, M.d_sc_ptr.p, M.d_sc_pos.p, M.d_Ycell.p,
                                                     (int64_t)M.nif * C, y, H.n0, 1, nullptr, nullptr);
  CK(cudaGetLastError());
  H.launches += 2;
  if (K && K->mesh.n_interface > 0) {
    const int64_t nI1 = K->mesh.n_interface;
    dev::k_gather_iface<<<nblk(nI1, 256), 256, 0, s>>>(nI1, K->d_sc_ptr.p, K->d_sc_pos.p, K->d_Ycell.p,
                                                       (int64_t)K->nif * C, y + H.n0, H.n1, 1, nullptr, nullptr);
    CK(cudaGetLastError());
    ++H.launches;
  }
}

// The two blocks of Eq. (7.6) are independent: the X^k block runs on the handle's second stream
// beside the X^{k-1} block and joins before the caller's next step.
void hodge_precond(riesz_hodge& H, const double* r, double* z, cudaStream_t s) {
  CK(cudaEventRecord(H.ev_f, s));
  CK(cudaStreamWaitEvent(H.s1, H.ev_f, 0));
  if (H.P1) {
    op_precond(*H.P1, r + H.n0, z + H.n0, 1, H.s1);
  } else {  // k = 3: the diagonal DG block, inverted exactly
    dev::k_dg_scale<<<nblk(H.n1, 256), 256, 0, H.s1>>>(H.n1, H.d_dg_dinv.p, r + H.n0, z + H.n0);
    CK(cudaGetLastError());
    ++H.launches;
  }
  op_precond(*H.P0, r, z, 1, s);
  CK(cudaEventRecord(H.ev_j, H.s1));
  CK(cudaStreamWaitEvent(s, H.ev_j, 0));
}

void hodge_dot(riesz_hodge& H, const double* a, const double* b, int op, cudaStream_t s) {
  dev::k_mr_dot<<<dev::red_blocks(H.N()), dev::NT, 0, s>>>(H.N(), a, b, H.d_part.p, H.d_ticket.p, op, H.d_m.p);
  CK(cudaGetLastError());
  ++H.launches;
}

void hodge_read(riesz_hodge& H, cudaStream_t s) {
  CK(cudaMemcpyAsync(H.h_m, H.d_m.p, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
}

// One MINRES iteration k: w = A u_k - beta_k v_{k-1} - alpha_k v_k (v_0 = 0), z = P^{-1} w,
// beta_{k+1} and the Givens step, then d_k, x and the next Lanczos vectors (v_{k+1} written over
// v_{k-1}, d_k over d_{k-2}).
void hodge_iteration(riesz_hodge& H, double* x, double* vcur, double* vprev, double* dd1, double* dd2,
                     cudaStream_t s) {
  const int64_t N = H.N();
  const unsigned nb = nblk(N, 256);
  hodge_apply(H, H.u.p, H.w.p, s);
  dev::k_mr_sub_beta<<<nb, 256, 0, s>>>(N, H.d_m.p, H.w.p, vprev);
  ++H.launches;
  hodge_dot(H, H.u.p, H.w.p, 1, s);
  dev::k_mr_sub_alpha<<<nb, 256, 0, s>>>(N, H.d_m.p, H.w.p, vcur);
  hodge_precond(H, H.w.p, H.z.p, s);
  hodge_dot(H, H.w.p, H.z.p, 2, s);
  dev::k_mr_update<<<nb, 256, 0, s>>>(N, H.d_m.p, x, H.u.p, dd1, dd2, vprev, H.w.p, H.z.p);
  CK(cudaGetLastError());
  H.launches += 2;
}

// launch counters of the Hodge handle and of every block handle (captured work is counted per pass)
struct HodgeCounters {
  std::vector<std::pair<int64_t*, int64_t>> c;
  explicit HodgeCounters(riesz_hodge& H) {
    c.push_back({&H.launches, H.launches});
    for (riesz_handle* x : {H.P0, H.P1, H.Mh, H.Kh})
      if (x)
        for (riesz_handle* y : {x, x->aux, x->caux})
          if (y) c.push_back({&y->launches, y->launches});
  }
  int64_t delta() const {
    int64_t d = 0;
    for (auto& e : c) d += *e.first - e.second;
    return d;
  }
  void restore() {
    for (auto& e : c) *e.first = e.second;
  }
};

bool hodge_profiling(const riesz_hodge& H) {
  for (riesz_handle* x : {H.P0, H.P1, H.Mh, H.Kh})
    if (x && (x->prof || (x->aux && x->aux->prof))) return true;
  return false;
}

// The device-driven loop's graph, built once per handle (every buffer it touches is handle-owned).
void hodge_ensure_graph(riesz_hodge& H) {
  if (H.g_loop) return;
  if (!H.cap) CK(cudaStreamCreateWithFlags(&H.cap, cudaStreamNonBlocking));
  cudaStream_t cs = H.cap;
  HodgeCounters cnt(H);
  cudaGraph_t G;
  CK(cudaGraphCreate(&G, 0));
  auto captured = [&](cudaGraph_t target, auto&& fn, std::vector<cudaGraphNode_t>* leaves) {
    CK(cudaStreamBeginCaptureToGraph(cs, target, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
      fn();
      if (leaves) {
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t* d = nullptr;
        size_t nd = 0;
        CK(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &d, nullptr, &nd));
        leaves->assign(d, d + nd);
      }
    } catch (...) {
      cudaGraph_t g;
      cudaStreamEndCapture(cs, &g);
      cudaGetLastError();
      throw;
    }
    cudaGraph_t g;
    CK(cudaStreamEndCapture(cs, &g));
  };
  try {
    cudaGraphConditionalHandle hw;
    CK(cudaGraphConditionalHandleCreate(&hw, G, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wn;
    CK(cudaGraphAddNode(&wn, G, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    cudaGraphConditionalHandle hi;
    CK(cudaGraphConditionalHandleCreate(&hi, body, 0u, cudaGraphCondAssignDefault));
    std::vector<cudaGraphNode_t> deps;
    captured(body, [&] {
      hodge_iteration(H, H.xw.p, H.v.p, H.vp.p, H.d1.p, H.d2.p, cs);
      dev::k_mr_control<<<1, 32, 0, cs>>>(hw, hi, 1, H.d_m.p, H.rtol, H.d_ctl.p);
      CK(cudaGetLastError());
      ++H.launches;
    }, &deps);
    H.g_iter_launches = cnt.delta();
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hi;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t in;
    CK(cudaGraphAddNode(&in, body, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &ip));
    captured(ip.conditional.phGraph_out[0], [&] {
      hodge_iteration(H, H.xw.p, H.vp.p, H.v.p, H.d2.p, H.d1.p, cs);
      dev::k_mr_control<<<1, 32, 0, cs>>>(hw, hi, 0, H.d_m.p, H.rtol, H.d_ctl.p);
      CK(cudaGetLastError());
      ++H.launches;
    }, nullptr);
  } catch (...) {
    cnt.restore();
    cudaGraphDestroy(G);
    throw;
  }
  cnt.restore();  // captured, not launched
  H.g_loop = instantiate(G);
}

// Preconditioned MINRES (Paige-Saunders): Lanczos on P^{-1} A in the P-inner
// product, the tridiagonal reduced by Givens rotations as it grows; stops when
// the P^{-1}-norm of the residual, |phibar|, drops below rtol times its initial
// value, then reports the true relative residual ||b - A x|| / ||b||.  The
// iterations run either from the host (one synchronisation per iteration) or
// in the device-driven graph loop; both enqueue the same kernels in the same
// order and give bitwise the same iterates.
int hodge_minres(riesz_hodge& H, const double* b, double* x, cudaStream_t s, int* iters, double* relres) {
  const int64_t N = H.N();
  const unsigned nb = nblk(N, 256);
  const bool graph = H.loop == RIESZ_LOOP_GRAPH && !hodge_profiling(H);
  double* xs = x;  // the iterate: the caller's x, or the handle's working copy for the graph loop
  if (graph) {
    if (!H.xw.p) H.xw.alloc((size_t)N);
    CK(cudaMemcpyAsync(H.xw.p, x, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    xs = H.xw.p;
  }
  hodge_apply(H, xs, H.w.p, s);
  dev::k_mr_residual<<<nb, 256, 0, s>>>(N, b, H.w.p);
  hodge_precond(H, H.w.p, H.z.p, s);
  hodge_dot(H, H.w.p, H.z.p, 0, s);
  dev::k_mr_scale<<<nb, 256, 0, s>>>(N, H.d_m.p, H.w.p, H.z.p, H.v.p, H.u.p);
  CK(cudaMemsetAsync(H.d1.p, 0, N * sizeof(double), s));
  CK(cudaMemsetAsync(H.d2.p, 0, N * sizeof(double), s));
  CK(cudaMemsetAsync(H.vp.p, 0, N * sizeof(double), s));  // v_0 = 0
  H.launches += 2;
  hodge_read(H, s);
  if (H.h_m[6] != 0.0) throw Err(RIESZ_ERR_NONFINITE, "non-finite right-hand side or preconditioner");
  if (H.h_m[dev::M_RAW] < 0.0) throw Err(RIESZ_ERR_INTERNAL, "block preconditioner is not positive definite");
  const double beta1 = H.h_m[dev::M_BETA1];
  int it = 0;
  int rc = RIESZ_OK;
  double phi = beta1;
  if (graph && beta1 > 0.0) {
    if (H.maxit == 0) {
      rc = RIESZ_ERR_NOT_CONVERGED;
    } else {
      hodge_ensure_graph(H);
      H.h_ctl[0] = 0;
      H.h_ctl[1] = H.maxit;
      H.h_ctl[2] = 0;
      CK(cudaMemcpyAsync(H.d_ctl.p, H.h_ctl, 4 * sizeof(int), cudaMemcpyHostToDevice, s));
      CK(cudaGraphLaunch(H.g_loop, s));
      CK(cudaMemcpyAsync(H.h_ctl, H.d_ctl.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
      hodge_read(H, s);
      it = H.h_ctl[0];
      H.launches += (int64_t)it * H.g_iter_launches;
      const int reason = H.h_ctl[2];
      if (reason == 1) throw Err(RIESZ_ERR_NONFINITE, "non-finite value in the MINRES recurrence");
      if (reason == 5) throw Err(RIESZ_ERR_INTERNAL, "block preconditioner is not positive definite");
      if (reason == 4) rc = RIESZ_ERR_NOT_CONVERGED;
      phi = std::fabs(H.h_m[dev::M_PHIBAR]);
    }
    // an odd number of iterations leaves the roles of the two buffer pairs swapped; x is unaffected
    CK(cudaMemcpyAsync(x, H.xw.p, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    double* vcur = H.v.p;
    double* vprev = H.vp.p;
    double* dd1 = H.d1.p;
    double* dd2 = H.d2.p;
    while (beta1 > 0.0) {
      if (it >= H.maxit) {
        rc = RIESZ_ERR_NOT_CONVERGED;
        break;
      }
      ++it;
      hodge_iteration(H, x, vcur, vprev, dd1, dd2, s);
      std::swap(dd1, dd2);      // d_k is now in dd1, d_{k-1} in dd2
      std::swap(vprev, vcur);   // v_{k+1} was written over v_{k-1}
      hodge_read(H, s);
      if (H.h_m[6] != 0.0) throw Err(RIESZ_ERR_NONFINITE, "non-finite value in the MINRES recurrence");
      if (H.h_m[dev::M_RAW] < 0.0) throw Err(RIESZ_ERR_INTERNAL, "block preconditioner is not positive definite");
      phi = std::fabs(H.h_m[dev::M_PHIBAR]);
      if (phi <= H.rtol * beta1 || H.h_m[dev::M_BNEXT] == 0.0) break;
    }
  }
  // true residual
  hodge_apply(H, x, H.w.p, s);
  dev::k_mr_residual<<<nb, 256, 0, s>>>(N, b, H.w.p);
  ++H.launches;
  hodge_dot(H, H.w.p, H.w.p, 1, s);
  hodge_read(H, s);
  const double rr = H.h_m[dev::M_ALPHA];
  hodge_dot(H, b, b, 1, s);
  hodge_read(H, s);
  const double bb = H.h_m[dev::M_ALPHA];
  H.last_iters = it;
  H.last_relres = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
  H.last_phi = beta1 > 0.0 ? phi / beta1 : 0.0;
  if (iters) *iters = it;
  if (relres) *relres = H.last_relres;
  return rc;
}

}  // namespace

extern "C" {

int riesz_hodge_setup(int k, int p, int64_t nverts, const double* verts, int64_t ncells, const int64_t* cells,
                      double gamma, const riesz_opts* opts, void* stream, riesz_hodge** out) {
  return guarded([&] {
    need(out != nullptr, "null output");
    *out = nullptr;
    need(k >= 1 && k <= 3, "k must be 1 (CG_p x Ned1_p), 2 (Ned1_p x RT_p) or 3 (RT_p x DG_{p-1})");
    need(gamma > 0 && std::isfinite(gamma), "gamma must be positive and finite");
    riesz_opts o;
    riesz_default_opts(&o);
    if (opts) o = *opts;
    need(!o.dirichlet, "the Hodge-Laplace problems are pure Neumann");
    need(o.rtol > 0 && o.maxit >= 0, "bad rtol or maxit");
    const bool paper = o.decomposition != RIESZ_DECOMP_VERTEX_STAR;
    auto H = std::make_unique<riesz_hodge>();
    H->k = k;
    H->p = p;
    H->gamma = gamma;
    H->rtol = o.rtol;
    H->maxit = o.maxit;
    need(o.loop == RIESZ_LOOP_HOST || o.loop == RIESZ_LOOP_GRAPH, "bad loop");
    H->loop = o.loop;
    riesz_opts b = o;
    b.nrhs_max = 1;
    b.loop = RIESZ_LOOP_HOST;
    b.apply_mode = RIESZ_APPLY_ELEMENT;
    b.apply_precision = RIESZ_PREC_FP64;
    // preconditioner blocks: the weighted Riesz maps of Eq. (7.6), with the paper's decomposition of
    // each space (vertex stars for CG_p, Hiptmair-Toselli for Ned1_p, edge stars for RT_p) or vertex stars
    auto decomp = [&](int space) {
      if (!paper) return (int)RIESZ_DECOMP_VERTEX_STAR;
      return space == RIESZ_HCURL ? (int)RIESZ_DECOMP_HT
                                  : (space == RIESZ_HDIV ? (int)RIESZ_DECOMP_EDGE_STAR : (int)RIESZ_DECOMP_VERTEX_STAR);
    };
    riesz_opts o0 = b, o1 = b;
    o0.alpha = gamma;
    o0.beta = 1.0;
    o0.decomposition = decomp(k - 1);
    H->P0 = create_handle(k - 1, p, nverts, verts, ncells, cells, o0, true);
    // MINRES needs a positive definite preconditioner: the W^k inverses of the blocks by the FP64
    // Cholesky route (A_0 = R_0 (M + gamma K) R_0^T and gamma^{-1} M + K reach kappa ~ 1e7 for gamma
    // far from 1, where an explicit Gauss-Jordan inverse, even in FP64, is no longer definite).  It also
    // needs a fixed (linear) preconditioner, which the few lowest-order PCG steps of the coarse route
    // above the dense limit are not: such blocks stay one-level.
    auto dense_coarse_only = [](riesz_handle* P) {
      if (P->coarse_sparse) P->coarse_on = P->coarse_sparse = false;
    };
    dense_coarse_only(H->P0);
    if (k < 3) {
      o1.alpha = 1.0;
      o1.beta = 1.0 / gamma;
      o1.decomposition = decomp(k);
      H->P1 = create_handle(k, p, nverts, verts, ncells, cells, o1, true);
      dense_coarse_only(H->P1);
    }
    // operator blocks
    riesz_opts om = b, ok = b;
    om.alpha = 0.0;
    om.beta = 1.0;
    om.decomposition = RIESZ_DECOMP_VERTEX_STAR;
    ok.alpha = 1.0;
    ok.beta = 0.0;
    ok.decomposition = RIESZ_DECOMP_VERTEX_STAR;
    H->Mh = create_handle(k - 1, p, nverts, verts, ncells, cells, om, true, true);
    if (k < 3) H->Kh = create_handle(k, p, nverts, verts, ncells, cells, ok, true, true);
    const int64_t C = H->Mh->C();
    H->n0 = H->Mh->N();
    if (k < 3) {
      H->n1 = H->Kh->N();
    } else {
      H->n_dg = dg_dim(p);
      H->n1 = C * H->n_dg;
      need(H->n1 < ((int64_t)1 << 31), "too many DG DOFs for 32-bit indices");
    }
    cudaStream_t s = S(stream);
    CK(cudaStreamCreateWithFlags(&H->s1, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&H->ev_f, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&H->ev_j, cudaEventDisableTiming));
    for (riesz_handle* x : {H->P0, H->P1, H->Mh, H->Kh})
      if (x) setup_device_impl(*x, s);
    const int n0 = H->Mh->mesh.nref, n1 = H->Kh ? H->Kh->mesh.nref : H->n_dg;
    std::vector<double> R;
    try {
      R = mixed_reference_tables(k, p);
    } catch (const std::exception& e) {
      throw Err(RIESZ_ERR_INTERNAL, e.what());
    }
    H->d_R.upload(R, s);
    H->d_gB.alloc((size_t)12 * C);  // k_geom writes all Q factors of its space (12 for Ned1_p)
    H->d_jacB.alloc((size_t)C * 10);
    H->d_Be.alloc((size_t)C * n0 * n1);
    if (k == 3) {  // DG_{p-1}: cell-major map, reference mass diagonal, load cross table
      const int nd = H->n_dg;
      std::vector<int32_t> cd((size_t)nd * C);
      for (int i = 0; i < nd; ++i)
        for (int64_t c = 0; c < C; ++c) cd[(size_t)i * C + c] = (int32_t)(c * nd + i);
      H->d_dg_cd.upload(cd, s);
      Rule Q = simplex_rule(3, p + 2);
      const int np = Q.npt();
      const RefElement& cg = *H->Mh->refcg;
      std::vector<double> v((size_t)np * nd), vc((size_t)np * cg.nref);
      dg_tabulate(p, np, Q.x.data(), v.data());
      cg.tabulate(np, Q.x.data(), vc.data(), nullptr);
      std::vector<double> mhat(nd, 0.0), X((size_t)cg.nref * nd, 0.0);
      for (int q = 0; q < np; ++q)
        for (int i = 0; i < nd; ++i) {
          const double wv = Q.w[q] * v[(size_t)q * nd + i];
          mhat[i] += wv * v[(size_t)q * nd + i];
          for (int a = 0; a < cg.nref; ++a) X[(size_t)a * nd + i] += wv * vc[(size_t)q * cg.nref + a];
        }
      H->d_dg_mhat.upload(mhat, s);
      H->d_dg_X.upload(X, s);
      H->d_dg_dinv.alloc((size_t)H->n1);
    }
    const size_t sm = dev::hodge_apply_smem(dev::NT, n0, n1);
    if (sm > 48 * 1024) raise_smem_limit(dev::k_hodge_apply, sm);
    for (auto* v : {&H->v, &H->vp, &H->u, &H->w, &H->z, &H->d1, &H->d2}) v->alloc((size_t)H->N());
    H->d_m.alloc(16);
    CK(cudaMemsetAsync(H->d_m.p, 0, 16 * sizeof(double), s));
    H->d_part.alloc(dev::RED_BLOCKS);
    H->d_ticket.alloc(1);
    CK(cudaMemsetAsync(H->d_ticket.p, 0, sizeof(unsigned), s));
    H->d_ctl.alloc(4);
    CK(cudaMallocHost((void**)&H->h_m, 16 * sizeof(double)));
    CK(cudaMallocHost((void**)&H->h_ctl, 4 * sizeof(int)));
    hodge_geometry(*H, s);
    CK(cudaStreamSynchronize(s));
    *out = H.release();
  });
}

int riesz_hodge_sizes(const riesz_hodge* h, int64_t* n0, int64_t* n1, int64_t* ncg) {
  return guarded([&] {
    need(h && n0 && n1, "null argument");
    *n0 = h->n0;
    *n1 = h->n1;
    if (ncg) *ncg = h->Mh->meshcg.ndofs;
  });
}

int riesz_hodge_apply(riesz_hodge* h, const double* x, double* y, void* stream) {
  return guarded([&] {
    need(h && x && y, "null argument");
    hodge_apply(*h, x, y, S(stream));
  });
}

int riesz_hodge_precond(riesz_hodge* h, const double* r, double* z, void* stream) {
  return guarded([&] {
    need(h && r && z, "null argument");
    hodge_precond(*h, r, z, S(stream));
  });
}

int riesz_hodge_load(riesz_hodge* h, const double* fcg, double* b, void* stream) {
  return guarded([&] {
    need(h && fcg && b, "null argument");
    cudaStream_t s = S(stream);
    CK(cudaMemsetAsync(b, 0, h->n0 * sizeof(double), s));
    if (h->k == 3) {  // scalar source f in CG_p against the DG functions
      riesz_handle& M = *h->Mh;
      dev::k_dg_load<<<(unsigned)M.C(), 128, 0, s>>>(M.C(), h->n_dg, M.refcg->nref, M.d_jac.p, M.d_cgdofs.p, fcg,
                                                     h->d_dg_X.p, b + h->n0);
      CK(cudaGetLastError());
      ++h->launches;
      return;
    }
    const int rc = riesz_load(h->Kh, fcg, b + h->n0, stream);
    if (rc != RIESZ_OK) throw Err(rc, "load on X^k failed");
  });
}

int riesz_hodge_update_geometry(riesz_hodge* h, const double* verts, void* stream) {
  return guarded([&] {
    need(h && verts, "null argument");
    cudaStream_t s = S(stream);
    for (riesz_handle* x : {h->P0, h->P1, h->Mh, h->Kh}) {
      if (!x) continue;
      CK(cudaMemcpyAsync(x->d_verts.p, verts, x->d_verts.bytes(), cudaMemcpyDeviceToDevice, s));
      device_compute(*x, s);
    }
    hodge_geometry(*h, s);
  });
}

int riesz_hodge_solve(riesz_hodge* h, const double* b, double* x, void* stream, int* iters, double* relres) {
  int rc = RIESZ_OK;
  const int g = guarded([&] {
    need(h && b && x, "null argument");
    rc = hodge_minres(*h, b, x, S(stream), iters, relres);
  });
  if (g != RIESZ_OK) return g;
  if (rc != RIESZ_OK) g_err = "MINRES did not reach rtol within maxit";
  return rc;
}

int riesz_hodge_stats(const riesz_hodge* h, double* out) {
  return guarded([&] {
    need(h && out, "null argument");
    out[0] = (double)(h->launches + h->sub_launches());
    out[1] = h->last_iters;
    out[2] = h->last_relres;
    out[3] = h->last_phi;
    out[4] = (double)h->n0;
    out[5] = (double)h->n1;
  });
}

int riesz_hodge_destroy(riesz_hodge* h) {
  return guarded([&] { delete h; });
}

}  // extern "C"
