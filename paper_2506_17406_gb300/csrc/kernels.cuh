// Device kernels of the Riesz-map solver (sm_103a).
//
// Data layout in HBM (C = cells, N = global DOFs, n = n_ref):
//   cell_dofs  int32 [n][C]      local DOF j of cell c at [j*C + c] (coalesced over cells)
//   g          f64   [Q][C]      per-cell geometric factors of the affine pullbacks
//   R          f64   [Q][n][n]   reference matrices (L2-resident)
//   Ae         f64   [C][n][n]   optional stored element matrices
//   Ycell      f64   [nrhs][n_if][C]  per-cell interface results before the scatter
//   patches    packed lower-triangular row-major factors, one CTA per patch
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace riesz {
namespace dev {

constexpr int NT = 256;   // threads per CTA for the per-patch / per-cell kernels
constexpr int NB = 32;    // Cholesky / triangular-sweep block size

__device__ __forceinline__ int64_t tri(int64_t i, int64_t j) { return i * (i + 1) / 2 + j; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// a1: geometry.  J = [x1-x0, x2-x0, x3-x0] * Er^{-1}; factors per space:
//   H1   : |det|, G = |det| J^{-1} J^{-T} (6)
//   HCURL: G (6), H = J^T J / |det| (6)
//   HDIV : H (6), 1/|det|
// pair order (00, 11, 22, 01, 02, 12).  Also stores J, det for the load.
// ---------------------------------------------------------------------------
struct Mat3 {
  double a[9];
};

__global__ void k_geom(int space, int64_t C, const double* __restrict__ verts, const int32_t* __restrict__ cells,
                       Mat3 Erinv, double* __restrict__ g, double* __restrict__ jac) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= C) return;
  double X[4][3];
  for (int k = 0; k < 4; ++k)
    for (int d = 0; d < 3; ++d) X[k][d] = verts[(int64_t)cells[c * 4 + k] * 3 + d];
  double Ep[3][3];
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < 3; ++k) Ep[d][k] = X[k + 1][d] - X[0][d];
  double J[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += Ep[i][k] * Erinv.a[k * 3 + j];
      J[i][j] = s;
    }
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double Ji[3][3];
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  const double ad = fabs(det);
  const int P[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  double G[6], H[6];
  for (int q = 0; q < 6; ++q) {
    const int a = P[q][0], b = P[q][1];
    double s = 0.0, t = 0.0;
    for (int k = 0; k < 3; ++k) {
      s += Ji[a][k] * Ji[b][k];  // (J^{-1} J^{-T})_ab
      t += J[k][a] * J[k][b];    // (J^T J)_ab
    }
    G[q] = ad * s;
    H[q] = t / ad;
  }
  if (space == 0) {
    g[c] = ad;
    for (int q = 0; q < 6; ++q) g[(1 + q) * C + c] = G[q];
  } else if (space == 1) {
    for (int q = 0; q < 6; ++q) g[q * C + c] = G[q];
    for (int q = 0; q < 6; ++q) g[(6 + q) * C + c] = H[q];
  } else {
    for (int q = 0; q < 6; ++q) g[q * C + c] = H[q];
    g[6 * C + c] = 1.0 / ad;
  }
  for (int k = 0; k < 9; ++k) jac[c * 10 + k] = J[k / 3][k % 3];
  jac[c * 10 + 9] = det;
}

// A_T = sum_q g_q(T) R_q, stored [C][n][n] (setup of the element-matrix apply).
__global__ void k_elem_matrices(int64_t C, int n, int Q, const double* __restrict__ g, const double* __restrict__ R,
                                double* __restrict__ Ae) {
  const int64_t c = blockIdx.x;
  const int64_t nn = (int64_t)n * n;
  double gq[16];
  for (int q = 0; q < Q; ++q) gq[q] = g[q * C + c];
  for (int64_t t = threadIdx.x; t < nn; t += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < Q; ++q) s += gq[q] * R[q * nn + t];
    Ae[c * nn + t] = s;
  }
}

// ---------------------------------------------------------------------------
// a3-a5: apply.  Gather x on the cell, y_T = A_T x_T, interior rows written
// directly (each interior DOF belongs to one cell), interface rows to Ycell.
// ---------------------------------------------------------------------------
// Element-matrix variant: one CTA per cell, one warp per row (lanes over j).
__global__ void k_apply_elem(int64_t C, int n, int nif, const double* __restrict__ Ae,
                             const int32_t* __restrict__ cdofs, const double* __restrict__ x, double* __restrict__ y,
                             double* __restrict__ Ycell, int nrhs, int64_t N) {
  extern __shared__ double xs[];  // [nrhs][n]
  const int64_t c = blockIdx.x;
  for (int t = threadIdx.x; t < n * nrhs; t += blockDim.x) {
    const int r = t / n, j = t % n;
    xs[t] = x[r * N + cdofs[(int64_t)j * C + c]];
  }
  __syncthreads();
  const double* A = Ae + c * (int64_t)n * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < n; i += nw) {
    const double* Ai = A + (int64_t)i * n;
    for (int r = 0; r < nrhs; ++r) {
      double s = 0.0;
      const double* xr = xs + r * n;
      for (int j = lane; j < n; j += 32) s += Ai[j] * xr[j];
      s = warp_sum(s);
      if (lane == 0) {
        if (i >= nif)
          y[r * N + cdofs[(int64_t)i * C + c]] = s;
        else
          Ycell[((int64_t)r * nif + i) * C + c] = s;
      }
    }
  }
}

// Matrix-free variant: y_T = sum_q g_q(T) R_q x_T for a tile of TC cells.
// lane = cell of the tile, warps split the rows; R entries are warp-uniform
// (broadcast loads), x_T and g_T live in shared memory.
constexpr int TC = 32;
constexpr int RB = 8;  // rows per thread per pass
__global__ void k_apply_mf(int64_t C, int n, int nif, int Q, const double* __restrict__ R,
                           const double* __restrict__ g, const int32_t* __restrict__ cdofs,
                           const double* __restrict__ x, double* __restrict__ y, double* __restrict__ Ycell, int64_t N) {
  extern __shared__ double sm[];
  double* Xs = sm;               // [n][TC]
  double* Gs = sm + n * TC;      // [Q][TC]
  const int64_t c0 = (int64_t)blockIdx.x * TC;
  const int r = blockIdx.y;      // right-hand side
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = threadIdx.x; t < n * TC; t += blockDim.x) {
    const int j = t / TC, cc = t % TC;
    const int64_t c = c0 + cc;
    Xs[t] = (c < C) ? x[r * N + cdofs[(int64_t)j * C + c]] : 0.0;
  }
  for (int t = threadIdx.x; t < Q * TC; t += blockDim.x) {
    const int q = t / TC, cc = t % TC;
    const int64_t c = c0 + cc;
    Gs[t] = (c < C) ? g[q * C + c] : 0.0;
  }
  __syncthreads();
  const int64_t c = c0 + lane;
  const int64_t nn = (int64_t)n * n;
  for (int i0 = warp * RB; i0 < n; i0 += nw * RB) {
    double acc[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) acc[k] = 0.0;
    for (int q = 0; q < Q; ++q) {
      double t[RB];
#pragma unroll
      for (int k = 0; k < RB; ++k) t[k] = 0.0;
      const double* Rq = R + q * nn;
      for (int j = 0; j < n; ++j) {
        const double xv = Xs[j * TC + lane];
#pragma unroll
        for (int k = 0; k < RB; ++k) {
          const int i = i0 + k;
          const double rv = (i < n) ? __ldg(Rq + (int64_t)i * n + j) : 0.0;
          t[k] = fma(rv, xv, t[k]);
        }
      }
      const double gv = Gs[q * TC + lane];
#pragma unroll
      for (int k = 0; k < RB; ++k) acc[k] = fma(gv, t[k], acc[k]);
    }
    if (c < C) {
#pragma unroll
      for (int k = 0; k < RB; ++k) {
        const int i = i0 + k;
        if (i >= n) break;
        if (i >= nif)
          y[r * N + cdofs[(int64_t)i * C + c]] = acc[k];
        else
          Ycell[((int64_t)r * nif + i) * C + c] = acc[k];
      }
    }
  }
}

// Deterministic scatter of the interface rows: y[d] = sum over the cells that
// share DOF d, in a fixed order (CSR built on the host).
__global__ void k_gather_iface(int64_t nifd, const int64_t* __restrict__ ptr, const int32_t* __restrict__ pos,
                               const double* __restrict__ Ycell, int64_t ystride, double* __restrict__ y,
                               int64_t N, int nrhs) {
  const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (d >= nifd) return;
  const int64_t b = ptr[d], e = ptr[d + 1];
  for (int r = 0; r < nrhs; ++r) {
    double s = 0.0;
    for (int64_t k = b; k < e; ++k) s += Ycell[r * ystride + pos[k]];
    y[r * N + d] = s;
  }
}

// ---------------------------------------------------------------------------
// a6: interior diagonal (point-Jacobi of Eq. (6.11)).
// ---------------------------------------------------------------------------
__global__ void k_interior_diag(int64_t C, int n, int nif, int Q, const double* __restrict__ g,
                                const double* __restrict__ R, const int32_t* __restrict__ cdofs,
                                int64_t n_interface, double* __restrict__ dinv) {
  const int nI = n - nif;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= C * nI) return;
  const int64_t c = t % C;
  const int j = nif + (int)(t / C);
  const int64_t nn = (int64_t)n * n;
  double s = 0.0;
  for (int q = 0; q < Q; ++q) s += g[q * C + c] * R[q * nn + (int64_t)j * n + j];
  dinv[cdofs[(int64_t)j * C + c] - n_interface] = 1.0 / s;
}

// ---------------------------------------------------------------------------
// a8: patch assembly.  A_V = sum over star cells of the restriction of A_T.
// Cells are processed one after the other (no two threads write the same
// entry within a cell), so the sum order is fixed.
// blocks of patch P: [pb_ptr[P], pb_ptr[P+1]); block b: cell pb_cell[b],
// entries pb_ent[pb_off[b] .. pb_off[b+1]) = local j + 1024 * patch index.
// ---------------------------------------------------------------------------
__global__ void k_patch_assemble(const int32_t* __restrict__ pn, const int64_t* __restrict__ pfoff,
                                 const int64_t* __restrict__ pb_ptr, const int32_t* __restrict__ pb_cell,
                                 const int64_t* __restrict__ pb_off, const int32_t* __restrict__ pb_ent,
                                 int64_t C, int n, int Q, const double* __restrict__ g, const double* __restrict__ R,
                                 const double* __restrict__ Ae, double* __restrict__ Lall) {
  const int P = blockIdx.x;
  const int64_t np = pn[P];
  double* A = Lall + pfoff[P];
  const int64_t ntri = np * (np + 1) / 2;
  for (int64_t t = threadIdx.x; t < ntri; t += blockDim.x) A[t] = 0.0;
  __syncthreads();
  const int64_t nn = (int64_t)n * n;
  for (int64_t b = pb_ptr[P]; b < pb_ptr[P + 1]; ++b) {
    const int64_t c = pb_cell[b];
    const int32_t* ent = pb_ent + pb_off[b];
    const int m = (int)(pb_off[b + 1] - pb_off[b]);
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int s = t / m, u = t % m;
      const int js = ent[s] & 1023, ps = ent[s] >> 10;
      const int ju = ent[u] & 1023, pu = ent[u] >> 10;
      if (ps < pu) continue;
      double v;
      if (Ae) {
        v = Ae[c * nn + (int64_t)js * n + ju];
      } else {
        v = 0.0;
        for (int q = 0; q < Q; ++q) v += g[q * C + c] * R[q * nn + (int64_t)js * n + ju];
      }
      A[tri(ps, pu)] += v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// a8: batched FP64 Cholesky, one CTA per patch, in place on the packed lower
// triangle (row-major).  Right-looking, NB-wide panels: factor the diagonal
// block in shared memory, solve the panel below, update the trailing matrix
// tile by tile.  A non-positive pivot sets info[P] and is replaced by 1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_cholesky(const int32_t* __restrict__ pn, const int64_t* __restrict__ pfoff,
                                                 double* __restrict__ Lall, int* __restrict__ info) {
  const int P = blockIdx.x;
  const int n = pn[P];
  double* A = Lall + pfoff[P];
  __shared__ double D[NB][NB + 1];
  __shared__ double Ti[NB][NB + 1], Tj[NB][NB + 1];
  const int tid = threadIdx.x;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    for (int t = tid; t < NB * NB; t += NT) {
      const int i = t / NB, j = t % NB;
      D[i][j] = (i < kb && j <= i) ? A[tri(k0 + i, k0 + j)] : 0.0;
    }
    __syncthreads();
    if (tid < 32) {
      const int lane = tid;
      for (int j = 0; j < kb; ++j) {
        if (lane == 0) {
          double d = D[j][j];
          if (!(d > 0.0)) {
            if (info[P] == 0) info[P] = k0 + j + 1;
            d = 1.0;
          }
          D[j][j] = sqrt(d);
        }
        __syncwarp();
        const double djj = D[j][j];
        if (lane > j && lane < kb) D[lane][j] /= djj;
        __syncwarp();
        for (int k = j + 1; k < kb; ++k)
          if (lane >= k && lane < kb) D[lane][k] -= D[lane][j] * D[k][j];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int t = tid; t < kb * kb; t += NT) {
      const int i = t / kb, j = t % kb;
      if (j <= i) A[tri(k0 + i, k0 + j)] = D[i][j];
    }
    // panel: rows below solve x L11^T = a
    for (int i = k0 + kb + tid; i < n; i += NT) {
      double xr[NB];
      double* Ai = A + tri(i, k0);
#pragma unroll
      for (int j = 0; j < NB; ++j) xr[j] = (j < kb) ? Ai[j] : 0.0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j < kb) {
          double s = xr[j];
          for (int k = 0; k < j; ++k) s -= xr[k] * D[j][k];
          xr[j] = s / D[j][j];
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (j < kb) Ai[j] = xr[j];
    }
    __syncthreads();
    // trailing update A22 -= L21 L21^T on tiles (I >= J)
    const int m0 = k0 + kb;
    const int nt = (n - m0 + NB - 1) / NB;
    const int ntiles = nt * (nt + 1) / 2;
    for (int tile = 0; tile < ntiles; ++tile) {
      int I = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
      while ((I + 1) * (I + 2) / 2 <= tile) ++I;
      while (I * (I + 1) / 2 > tile) --I;
      const int J = tile - I * (I + 1) / 2;
      const int i0 = m0 + I * NB, j0 = m0 + J * NB;
      for (int t = tid; t < NB * NB; t += NT) {
        const int r = t / NB, k = t % NB;
        Ti[r][k] = (i0 + r < n && k < kb) ? A[tri(i0 + r, k0 + k)] : 0.0;
        Tj[r][k] = (j0 + r < n && k < kb) ? A[tri(j0 + r, k0 + k)] : 0.0;
      }
      __syncthreads();
      for (int t = tid; t < NB * NB; t += NT) {
        const int r = t / NB, s = t % NB;
        const int gi = i0 + r, gj = j0 + s;
        if (gi < n && gj < n && gj <= gi) {
          double acc = 0.0;
#pragma unroll 8
          for (int k = 0; k < NB; ++k) acc += Ti[r][k] * Tj[s][k];
          A[tri(gi, gj)] -= acc;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// ---------------------------------------------------------------------------
// a7: patch solves z_V = L_V^{-T} L_V^{-1} R_V r, one CTA per patch.
// Forward sweep: block rows [i0, i0+32): dot products with the solved prefix
// (warp per row, coalesced row reads), then a 32x32 triangular solve by one
// warp.  Backward sweep: block columns from the bottom, each row below
// contributes its 32-wide segment (coalesced), then the 32x32 solve.
// Every factor entry is read once per sweep.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NT) k_patch_solve(const int32_t* __restrict__ pn, const int64_t* __restrict__ pdoff,
                                                    const int64_t* __restrict__ pfoff, const int32_t* __restrict__ pdofs,
                                                    const T* __restrict__ Lall, const double* __restrict__ r,
                                                    double* __restrict__ zpatch, int64_t N, int64_t zstride) {
  extern __shared__ unsigned char smraw[];
  T* y = reinterpret_cast<T*>(smraw);
  __shared__ T part[NT / 32][32];
  const int P = blockIdx.x;
  const int rh = blockIdx.y;
  const int n = pn[P];
  const T* L = Lall + pfoff[P];
  const int32_t* dofs = pdofs + pdoff[P];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NT / 32;
  for (int i = tid; i < n; i += NT) y[i] = (T)r[rh * N + dofs[i]];
  __syncthreads();
  // forward: L y = b
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int kb = min(32, n - i0);
    for (int rr = warp; rr < kb; rr += nw) {
      const int i = i0 + rr;
      const T* Li = L + tri(i, 0);
      T s = 0;
      for (int j = lane; j < i0; j += 32) s += Li[j] * y[j];
      s = warp_sum(s);
      if (lane == 0) y[i] -= s;
    }
    __syncthreads();
    if (warp == 0) {
      T yi = (lane < kb) ? y[i0 + lane] : (T)0;
      const T* Lr = L + tri(i0 + min(lane, kb - 1), i0);
      for (int j = 0; j < kb; ++j) {
        const T yj = __shfl_sync(0xffffffffu, yi, j) / L[tri(i0 + j, i0 + j)];
        if (lane == j) yi = yj;
        if (lane > j && lane < kb) yi -= Lr[j] * yj;
      }
      if (lane < kb) y[i0 + lane] = yi;
    }
    __syncthreads();
  }
  // backward: L^T x = y
  const int nblk = (n + 31) / 32;
  for (int b = nblk - 1; b >= 0; --b) {
    const int i0 = b * 32;
    const int kb = min(32, n - i0);
    T s = 0;
    for (int j = i0 + kb + warp; j < n; j += nw) {
      const T yj = y[j];
      if (lane < kb) s += L[tri(j, i0 + lane)] * yj;
    }
    part[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
      T acc = 0;
      for (int w = 0; w < nw; ++w) acc += part[w][lane];
      T xi = (lane < kb) ? y[i0 + lane] - acc : (T)0;
      for (int j = kb - 1; j >= 0; --j) {
        const T xj = __shfl_sync(0xffffffffu, xi, j) / L[tri(i0 + j, i0 + j)];
        if (lane == j) xi = xj;
        if (lane < j) xi -= L[tri(i0 + j, i0 + lane)] * xj;
      }
      if (lane < kb) y[i0 + lane] = xi;
    }
    __syncthreads();
  }
  double* zp = zpatch + rh * zstride + pdoff[P];
  for (int i = tid; i < n; i += NT) zp[i] = (double)y[i];
}

// z = diag(A_II)^{-1} r on the interior, sum of patch results on the interface.
__global__ void k_precond_gather(int64_t N, int64_t nifd, const int64_t* __restrict__ ptr,
                                 const int32_t* __restrict__ pos, const double* __restrict__ zpatch, int64_t zstride,
                                 const double* __restrict__ dinv, const double* __restrict__ r, double* __restrict__ z,
                                 int nrhs) {
  const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (d >= N) return;
  for (int rh = 0; rh < nrhs; ++rh) {
    double s;
    if (d < nifd) {
      s = 0.0;
      for (int64_t k = ptr[d]; k < ptr[d + 1]; ++k) s += zpatch[rh * zstride + pos[k]];
    } else {
      s = dinv[d - nifd] * r[rh * N + d];
    }
    z[rh * N + d] = s;
  }
}

// ---------------------------------------------------------------------------
// a9: PCG vector kernels with deterministic two-stage reductions.
// scal layout (per right-hand side, stride 16): see riesz.cu
// ---------------------------------------------------------------------------
constexpr int RED_BLOCKS = 592;  // 4 x 148 partials, reduced in a fixed order

template <int K>
__device__ __forceinline__ void block_reduce_store(double (&v)[K], double* __restrict__ out) {
  __shared__ double sh[K][NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = (lane < NT / 32) ? sh[k][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) out[k * RED_BLOCKS + blockIdx.x] = s;
    }
  }
}

// partial sums of a.b (and a.c when c != nullptr)
__global__ void __launch_bounds__(NT) k_dot2(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                            const double* __restrict__ c, double* __restrict__ part) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)RED_BLOCKS * NT) {
    const double ai = a[i];
    v[0] = fma(ai, b[i], v[0]);
    if (c) v[1] = fma(ai, c[i], v[1]);
  }
  block_reduce_store<2>(v, part);
}

// Scalar step after a reduction.  op: 0 pAp -> alpha; 1 rr; 2 rz -> beta
// (classic); 3 rz, r.zold -> beta (Polak-Ribiere); 4 bb; 5 initial rz.
enum ScalarSlot { S_RZ = 0, S_PAP = 1, S_ALPHA = 2, S_RR = 3, S_BETA = 4, S_BB = 5, S_NONFINITE = 6 };
__global__ void k_scalar(const double* __restrict__ part, int op, double* __restrict__ scal) {
  __shared__ double sh[2][NT / 32];
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < RED_BLOCKS; i += NT) {
    v[0] += part[i];
    v[1] += part[RED_BLOCKS + i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 2; ++k) {
    double s = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < NT / 32; ++w) {
      s0 += sh[0][w];
      s1 += sh[1][w];
    }
    if (!isfinite(s0) || !isfinite(s1)) scal[S_NONFINITE] = 1.0;
    if (op == 0) {
      scal[S_PAP] = s0;
      scal[S_ALPHA] = scal[S_RZ] / s0;
    } else if (op == 1) {
      scal[S_RR] = s0;
    } else if (op == 2) {
      scal[S_BETA] = s0 / scal[S_RZ];
      scal[S_RZ] = s0;
    } else if (op == 3) {
      scal[S_BETA] = (s0 - s1) / scal[S_RZ];
      scal[S_RZ] = s0;
    } else if (op == 4) {
      scal[S_BB] = s0;
    } else if (op == 5) {
      scal[S_RZ] = s0;
    }
  }
}

// x += alpha p ; r -= alpha Ap ; partial r.r
__global__ void __launch_bounds__(NT) k_update_xr(int64_t n, const double* __restrict__ scal, double* __restrict__ x,
                                                 double* __restrict__ r, const double* __restrict__ p,
                                                 const double* __restrict__ Ap, double* __restrict__ part) {
  const double alpha = scal[S_ALPHA];
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)RED_BLOCKS * NT) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, Ap[i], r[i]);
    r[i] = ri;
    v[0] = fma(ri, ri, v[0]);
  }
  block_reduce_store<2>(v, part);
}

// p = z + beta p
__global__ void k_update_p(int64_t n, const double* __restrict__ scal, const double* __restrict__ z,
                           double* __restrict__ p) {
  const double beta = scal[S_BETA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

// r = b - Ap ; partial r.r
__global__ void __launch_bounds__(NT) k_residual(int64_t n, const double* __restrict__ b,
                                                const double* __restrict__ Ax, double* __restrict__ r,
                                                double* __restrict__ part) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)RED_BLOCKS * NT) {
    const double ri = b[i] - Ax[i];
    r[i] = ri;
    v[0] = fma(ri, ri, v[0]);
  }
  block_reduce_store<2>(v, part);
}

// ---------------------------------------------------------------------------
// right-hand side of an [CG_p]^k source: b_i = (f, phi_i)
// f_T in reference components: ft[l][a] = sum_m T_ml c_m,a with T from J.
// ---------------------------------------------------------------------------
__global__ void k_load(int space, int64_t C, int n, int nif, int ncg, const double* __restrict__ jac,
                       const int32_t* __restrict__ cg_cdofs, const double* __restrict__ fcg, int64_t Ncg,
                       const double* __restrict__ X, const int32_t* __restrict__ cdofs, double* __restrict__ b,
                       double* __restrict__ Ycell) {
  extern __shared__ double ft[];  // [ncomp][ncg]
  const int64_t c = blockIdx.x;
  const int ncomp = (space == 0) ? 1 : 3;
  double J[9];
  for (int k = 0; k < 9; ++k) J[k] = jac[c * 10 + k];
  const double det = jac[c * 10 + 9], ad = fabs(det);
  double Ji[9];
  Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
  Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
  Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
  Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
  Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
  Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
  Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
  Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
  Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
  for (int a = threadIdx.x; a < ncg; a += blockDim.x) {
    const int64_t gd = cg_cdofs[(int64_t)a * C + c];
    if (space == 0) {
      ft[a] = ad * fcg[gd];
    } else {
      double cm[3];
      for (int m = 0; m < 3; ++m) cm[m] = fcg[m * Ncg + gd];
      for (int l = 0; l < 3; ++l) {
        double s = 0.0;
        for (int m = 0; m < 3; ++m) {
          const double T = (space == 1) ? ad * Ji[l * 3 + m] : (det > 0 ? 1.0 : -1.0) * J[m * 3 + l];
          s += T * cm[m];
        }
        ft[l * ncg + a] = s;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int l = 0; l < ncomp; ++l)
      for (int a = 0; a < ncg; ++a) s += ft[l * ncg + a] * X[((int64_t)l * ncg + a) * n + i];
    if (i >= nif)
      b[cdofs[(int64_t)i * C + c]] = s;
    else
      Ycell[(int64_t)i * C + c] = s;
  }
}

}  // namespace dev
}  // namespace riesz
