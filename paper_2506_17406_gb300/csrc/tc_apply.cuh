// Matrix-free operator on the 5th-generation tensor cores (sm_103a tcgen05):
//   Y_c = sum_q g_q(c) R_q X_c           (Section 6.4; the Q reference matrices R_q
// of the pullbacks of Eq. (2.7) against per-cell geometric factors g_q) as one
// GEMM per tile of 128 (cell, right-hand side) rows:
//   D[m][i] = sum_{(q, j)} A[m][(q, j)] B[(q, j)][i],
//   A[m][(q, j)] = g_q(c_m) X_{c_m}[j],   B[(q, j)][i] = R_q[i][j]  (R_q symmetric),
// in split BF16 with FP32 accumulation: every operand value v is v_hi + v_lo with
// v_hi = bf16(v), v_lo = bf16(v - v_hi), and D accumulates A_hi B_hi + A_hi B_lo +
// A_lo B_hi (the A_lo B_lo term is below the FP32 accumulation error).
//
// Layout.  The accumulator D (128 lanes x NP FP32 columns, NP = n padded to a
// multiple of 16, at most 512) lives in tensor memory for the whole K loop.  K
// runs over stages (j-chunk of TC_KC, q): the B stage (hi and lo, NP rows x TC_KC K)
// is a precomputed table in the canonical K-major layout without swizzle (core
// matrices of 8 rows x 16 bytes, K-adjacent core matrices 128 B apart, 8-row
// groups TC_SBO bytes apart), so one bulk copy (cp.async.bulk) moves a stage into
// shared memory; the A stage (hi and lo, 128 rows x TC_KC K, same layout) is built
// by the four producer warps from the gathered X and g.  Ring of NSTAGE slots,
// mbarriers with bounded waits.
//
// Warp roles (576 threads): warp 0 allocates tensor memory and issues the B
// bulk copies (one lane); warps 1-16 gather X, build the A stages and run the
// epilogue: warp w serves row m = 32 (w % 4) + lane (tensor-memory lanes of
// its quarter) and the K part (w - 1) / 4 (4 values) of every stage, four
// producer warps per scheduler to hide the gathers' latency.  Warp 17 (one
// lane) issues the MMAs and commits them to the slot's "empty" barrier and,
// after the last stage, to "done".
//
// Epilogue: the accumulator leaves tensor memory in windows of up to 256
// columns through a shared-memory staging tile (the operand ring, free once
// "done" has fired): the four warps of a lane quarter read alternate 16-column
// chunks (tcgen05.ld) into rows of the tile, then all 512 epilogue threads
// write the window out in global order, consecutive threads on consecutive
// addresses: interior rows of a cell are contiguous in y (row-major over the
// window's interior columns), interface entries of one column are contiguous
// over the tile's cells in Ycell.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace riesz {
namespace dev {

constexpr int TC_PWARPS = 16;                  // producer warps (warps 1..16), four per scheduler
constexpr int TC_NT = (TC_PWARPS + 2) * 32;    // + the copy warp (0) and the MMA warp (TC_PWARPS + 1)
constexpr int TC_PRODUCERS = TC_PWARPS * 32;
constexpr int TC_ROWS = 128;   // M of one MMA (cta_group::1)
constexpr int TC_KC = 16;      // K per stage (BF16 elements): one MMA K step
constexpr int TC_KCORE = TC_KC / 8;        // core matrices along K per stage
constexpr int TC_SBO = TC_KCORE * 128;     // bytes between 8-row groups (stride byte offset)
constexpr int TC_NSTAGE = 8;   // most ring slots (as many as shared memory holds, at least 2)
constexpr int TC_MAXNP = 512;  // tensor-memory columns of one CTA
constexpr int TC_MAXN = 1024;  // largest n_ref: above 512 outputs the columns are split over two CTAs (grid z)
// columns of part z (0 or 1) of NP padded outputs: one part up to 512, else two halves rounded to 16
__host__ __device__ inline int tc_part_cols(int NP, int z) {
  if (NP <= TC_MAXNP) return z == 0 ? NP : 0;
  const int h = (NP / 2 + 15) / 16 * 16;
  return z == 0 ? h : NP - h;
}
__host__ __device__ inline int tc_parts(int NP) { return NP <= TC_MAXNP ? 1 : 2; }

// bytes of one A stage (hi + lo) and of one B stage (hi + lo) for NP rows
__host__ __device__ constexpr uint32_t tc_a_bytes() { return 2u * TC_ROWS * TC_KC * 2u; }
__host__ __device__ constexpr uint32_t tc_b_bytes(int NP) { return 2u * (uint32_t)NP * TC_KC * 2u; }
// epilogue staging: the accumulator passes through shared memory in windows of TC_SW columns, FP32,
// rows padded by one word (conflict-free column writes and row reads)
constexpr int TC_SW = 256;
__host__ __device__ inline int tc_stage_cols(int NP) { return NP < TC_SW ? NP : TC_SW; }
__host__ __device__ inline uint32_t tc_stage_bytes(int NP) {
  return (uint32_t)TC_ROWS * (uint32_t)(tc_stage_cols(NP) + 1) * 4u;
}
// the operand ring, reused by the staging buffer once every MMA has completed; barriers behind both
__host__ __device__ inline uint32_t tc_region_bytes(int NP, int nstage) {
  const uint32_t ring = (uint32_t)nstage * (tc_a_bytes() + tc_b_bytes(NP)), st = tc_stage_bytes(NP);
  return ring > st ? ring : st;
}
inline size_t tc_smem_bytes(int NP, int nstage) { return (size_t)tc_region_bytes(NP, nstage) + 256; }
// ring slots that fit in the 227 KB of shared memory a CTA may hold
inline int tc_stages(int NP) {
  int ns = TC_NSTAGE;
  while (ns > 2 && tc_smem_bytes(NP, ns) > 232448) --ns;
  return ns;
}

// Shared-memory matrix descriptor (K-major, no swizzle): start address, leading
// byte offset (between K-adjacent core matrices), stride byte offset (between
// 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N x M tile.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this warp's 32 tensor-memory lanes
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// Two FP32 values to packed BF16 (round to nearest even; a0 in the low half, a1 in the high half)
__device__ __forceinline__ uint32_t tc_bf16x2(float a0, float a1) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(a1), "f"(a0));
  return d;
}
// hi/lo split of a pair: hi = bf16(a), lo = bf16(a - hi) (the subtraction is exact in FP32)
__device__ __forceinline__ void tc_split2(float a0, float a1, uint32_t& hi, uint32_t& lo) {
  hi = tc_bf16x2(a0, a1);
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
  lo = tc_bf16x2(a0 - h0, a1 - h1);
}

// X_c[j0 .. j0 + 15] of row (c, r) as FP32 (zero outside the cell's n DOFs, and at Dirichlet DOFs)
constexpr int TC_KQ = TC_PWARPS / 4;  // K parts of a stage (one per producer warp of a lane quarter)
constexpr int TC_KH = TC_KC / TC_KQ;  // K values of a stage per producer thread
static_assert(TC_KH == 4, "a producer thread writes 4 BF16 values (8 bytes) of each row per stage");
__device__ __forceinline__ void tc_load_x(float (&xf)[TC_KH], bool valid, int j0, int n, int nif, int64_t C,
                                          int64_t c, int r, int64_t N, const int32_t* __restrict__ cdofs,
                                          const double* __restrict__ x, const uint8_t* __restrict__ dmask) {
#pragma unroll
  for (int e = 0; e < TC_KH; ++e) {
    const int j = j0 + e;
    float v = 0.f;
    if (valid && j < n) {
      const int64_t dof = cdofs[(int64_t)j * C + c];
      if (!(dmask && j < nif && dmask[dof])) v = (float)x[(int64_t)r * N + dof];
    }
    xf[e] = v;
  }
}

// y = A x (interior rows) and Ycell (interface rows, scattered by k_gather_iface)
// for tiles of CELLS = 128 / RT cells and RT right-hand sides: row m = r * CELLS + c.
// Bst: the B stages [KC][Q][hi | lo][NP / 8][TC_KCORE][8][8] BF16 (see the file comment).
// The interior DOFs of a cell are numbered contiguously (cell-major), so row m writes its interior
// outputs from the cell's first interior DOF on.  Q (the number of reference matrices) is a template
// parameter so that the producers keep the Q factors of their cell in registers.
template <int Q>
__global__ void __launch_bounds__(TC_NT, 1) k_apply_tc(int64_t C, int n, int nif, int NPt, int KC, int RT, int NS,
                                                      const uint16_t* __restrict__ Bst, const double* __restrict__ g,
                                                      const int32_t* __restrict__ cdofs, const double* __restrict__ x,
                                                      double* __restrict__ y, double* __restrict__ Ycell, int nrhs,
                                                      int64_t N, const uint8_t* __restrict__ dmask,
                                                      int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_sm[];
  // this CTA's output columns [col0, col0 + NP) of the NPt padded ones (grid z: the column part)
  const int NP = tc_part_cols(NPt, blockIdx.z), col0 = blockIdx.z == 0 ? 0 : tc_part_cols(NPt, 0);
  const int NPs = tc_part_cols(NPt, 0);  // the ring is sized for the widest part
  const uint32_t abytes = tc_a_bytes(), bbytes = tc_b_bytes(NP), bstride = tc_b_bytes(NPs);
  unsigned char* sA = tc_sm;                           // [NS][abytes]
  unsigned char* sB = tc_sm + (size_t)NS * abytes;     // [NS][bstride], this part's rows of each B stage
  uint64_t* bars = reinterpret_cast<uint64_t*>(tc_sm + tc_region_bytes(NPs, NS));
  uint64_t* full_a = bars;                   // [NS], TC_PRODUCERS producer arrivals
  uint64_t* full_b = bars + TC_NSTAGE;       // [NS], expect_tx
  uint64_t* empty = bars + 2 * TC_NSTAGE;    // [NS], MMA commit
  uint64_t* done = bars + 3 * TC_NSTAGE;     // accumulator complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * TC_NSTAGE + 1);
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int CELLS = TC_ROWS / RT;
  const int64_t c0 = (int64_t)blockIdx.x * CELLS;
  const int r0 = blockIdx.y * RT;
  const int nst = KC * Q;
  uint32_t ncols = 32;
  while ((int)ncols < NP) ncols <<= 1;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full_a[s], TC_PRODUCERS);
      mbar_init(&full_b[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // B stages: one bulk copy each into the ring
    if (lane == 0) {
      int issued = 0;
      for (int s = 0; s < nst; ++s) {
        const int slot = s % NS, use = s / NS;
        if (use > 0 && !mbar_wait(&empty[slot], (use - 1) & 1, err)) {
          abort_flag = 1;
          break;
        }
        // hi rows then lo rows of this part: contiguous row-group ranges of the stage's hi and lo blocks
        const uint16_t* src = Bst + (size_t)s * 2 * NPt * TC_KC + (size_t)col0 * TC_KC;
        unsigned char* dst = sB + (size_t)slot * bstride;
        mbar_expect_tx(&full_b[slot], bbytes);
        bulk_g2s(dst, src, bbytes / 2, &full_b[slot]);
        bulk_g2s(dst + bbytes / 2, src + (size_t)NPt * TC_KC, bbytes / 2, &full_b[slot]);
        issued = s + 1;
      }
      // no copy may still be landing when the CTA exits (they have all landed in a complete run)
      for (int s = issued > NS ? issued - NS : 0; s < issued; ++s) mbar_wait(&full_b[s % NS], (s / NS) & 1, err);
    }
  } else if (warp <= TC_PWARPS) {
    // A producers: row m of the tile, K part kh (TC_KH values) of each stage; the next chunk of X is
    // gathered while this one is used
    const int m = 32 * (warp & 3) + lane, kh = (warp - 1) >> 2;
    const int cl = m % CELLS, rl = m / CELLS;
    const int64_t c = c0 + cl;
    const int r = r0 + rl;
    const bool valid = c < C && r < nrhs;
    float gq[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) gq[q] = valid ? (float)g[q * C + c] : 0.f;
    // part kh covers K values kh*4 .. kh*4+3: core matrix kh/2, bytes (kh%2)*8 of the 16-byte core row
    const uint32_t rowoff = (uint32_t)(m >> 3) * TC_SBO + (uint32_t)(kh >> 1) * 128u + (uint32_t)(m & 7) * 16u +
                            (uint32_t)(kh & 1) * 8u;
    float xf[TC_KH], xn[TC_KH];
    tc_load_x(xf, valid, kh * TC_KH, n, nif, C, c, r, N, cdofs, x, dmask);
    bool ok = true;
    for (int jc = 0; jc < KC && ok; ++jc) {
      if (jc + 1 < KC) tc_load_x(xn, valid, (jc + 1) * TC_KC + kh * TC_KH, n, nif, C, c, r, N, cdofs, x, dmask);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int s = jc * Q + q, slot = s % NS, use = s / NS;
        if (use > 0 && !mbar_wait(&empty[slot], (use - 1) & 1, err)) {
          ok = false;
          abort_flag = 1;
          break;
        }
        unsigned char* hi = sA + (size_t)slot * abytes;
        unsigned char* lo = hi + abytes / 2;
        const float gv = gq[q];
        uint32_t ph[2], pl[2];
        tc_split2(gv * xf[0], gv * xf[1], ph[0], pl[0]);
        tc_split2(gv * xf[2], gv * xf[3], ph[1], pl[1]);
        *reinterpret_cast<uint2*>(hi + rowoff) = make_uint2(ph[0], ph[1]);
        *reinterpret_cast<uint2*>(lo + rowoff) = make_uint2(pl[0], pl[1]);
        fence_async_smem();
        mbar_arrive(&full_a[slot]);
      }
#pragma unroll
      for (int e = 0; e < TC_KH; ++e) xf[e] = xn[e];
    }
  } else {
    // MMA issuer
    if (lane == 0) {
      const uint32_t idesc0 = tc_idesc(TC_ROWS, NP <= 256 ? NP : (NP / 2 + 15) / 16 * 16);
      const int np0 = NP <= 256 ? NP : (NP / 2 + 15) / 16 * 16;  // first N piece
      const int np1 = NP - np0;                                 // second piece (0 if NP <= 256)
      const uint32_t idesc1 = np1 > 0 ? tc_idesc(TC_ROWS, np1) : 0u;
      bool ok = true;
      for (int s = 0; s < nst && ok; ++s) {
        const int slot = s % NS, use = s / NS;
        if (!mbar_wait(&full_a[slot], use & 1, err) || !mbar_wait(&full_b[slot], use & 1, err)) {
          ok = false;
          abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a_hi = smem_addr(sA + (size_t)slot * abytes), a_lo = a_hi + abytes / 2;
        const uint32_t b_hi = smem_addr(sB + (size_t)slot * bstride), b_lo = b_hi + bbytes / 2;
#pragma unroll
        for (int ks = 0; ks < TC_KC / 16; ++ks) {
          const uint32_t ko = (uint32_t)ks * 256u;  // two core matrices per K step of 16
          const uint64_t ah = tc_desc(a_hi + ko, 128, TC_SBO), al = tc_desc(a_lo + ko, 128, TC_SBO);
          const uint64_t bh0 = tc_desc(b_hi + ko, 128, TC_SBO), bl0 = tc_desc(b_lo + ko, 128, TC_SBO);
          const int acc0 = (s > 0 || ks > 0) ? 1 : 0;
          tc_mma(tmem, ah, bh0, idesc0, acc0);
          tc_mma(tmem, ah, bl0, idesc0, 1);
          tc_mma(tmem, al, bh0, idesc0, 1);
          if (np1 > 0) {
            const uint32_t bo = (uint32_t)(np0 / 8) * TC_SBO;
            const uint64_t bh1 = tc_desc(b_hi + bo + ko, 128, TC_SBO), bl1 = tc_desc(b_lo + bo + ko, 128, TC_SBO);
            const uint32_t d1 = tmem + (uint32_t)np0;
            tc_mma(d1, ah, bh1, idesc1, acc0);
            tc_mma(d1, ah, bl1, idesc1, 1);
            tc_mma(d1, al, bh1, idesc1, 1);
          }
        }
        tc_commit(&empty[slot]);
      }
      tc_commit(done);
    }
  }

  // epilogue (see the file comment)
  if (warp >= 1 && warp <= TC_PWARPS) {
    const int et = threadIdx.x - 32;  // epilogue thread 0..511
    if (!mbar_wait(done, 0, err)) abort_flag = 1;
    tc_fence_after();
    const int q4 = warp & 3, kh = (warp - 1) >> 2;
    const int SW = tc_stage_cols(NPs), ld = SW + 1;
    float* st = reinterpret_cast<float*>(tc_sm);  // [TC_ROWS][ld]
    const double bad = __longlong_as_double(0x7ff8000000000000ll);
    const int nvalid = min(NP, n - col0);  // this CTA's real output columns
    for (int w0 = 0; w0 < NP; w0 += SW) {
      const int wc = min(SW, NP - w0);
      for (int i0 = 16 * kh; i0 < wc; i0 += 16 * TC_KQ) {
        float v[16];
        tc_ld16(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(w0 + i0), v);
        float* row = st + (32 * q4 + lane) * ld + i0;
#pragma unroll
        for (int k = 0; k < 16; ++k) row[k] = v[k];
      }
      asm volatile("bar.sync 1, %0;" ::"r"(TC_PRODUCERS) : "memory");
      const bool ok = !abort_flag;
      // global columns [g0, g1) of this window; interface part [g0, gi), interior part [gi, g1)
      const int g0 = col0 + w0, g1 = col0 + w0 + min(wc, nvalid - w0);
      const int gi = min(max(g0, nif), g1);
      const int nI = gi - g0, nJ = g1 - gi;
      // interface entries: item = ((r_local * nI + column) * CELLS + cell), cells fastest
      for (int it = et; it < RT * nI * CELLS; it += TC_PRODUCERS) {
        const int cl = it % CELLS, rest = it / CELLS, col = rest % nI, rl = rest / nI;
        const int64_t c = c0 + cl;
        const int r = r0 + rl;
        if (c >= C || r >= nrhs) continue;
        const float v = st[(rl * CELLS + cl) * ld + col];
        Ycell[((int64_t)r * nif + g0 + col) * C + c] = ok ? (double)v : bad;
      }
      // interior entries: item = (row m, column), columns fastest; a cell's interior DOFs are contiguous
      for (int it = et; it < TC_ROWS * nJ; it += TC_PRODUCERS) {
        const int col = it % nJ, m = it / nJ;
        const int cl = m % CELLS, rl = m / CELLS;
        const int64_t c = c0 + cl;
        const int r = r0 + rl;
        if (c >= C || r >= nrhs) continue;
        const float v = st[m * ld + nI + col];
        y[(int64_t)r * N + cdofs[(int64_t)nif * C + c] + (gi + col - nif)] = ok ? (double)v : bad;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(TC_PRODUCERS) : "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

}  // namespace dev
}  // namespace riesz
