// Exact KDE on the tcgen05 tensor cores with FP32-level accuracy.
//
// KDE_X(y) = (1/n) sum_i K_h(x_i, y) (paper Section 2 definition), evaluated
// like the paper's "Naive" method (Appendix D: D^2 = |x|^2 + |y|^2 - 2 <x, y>
// by matrix multiplication) but with the distance matrix never leaving the
// chip: each 128 x 128 tile of inner products is reduced to per-query kernel
// sums in the epilogue.
//
// Accuracy: every FP32 operand v is split into three BF16 parts
// v = v0 + v1 + v2 (v0 = bf16(v), v1 = bf16(v - v0), v2 = bf16(v - v0 - v1));
// the six products that carry weight down to 2^-24 relative,
// a0b0 + a0b1 + a1b0 + a0b2 + a1b1 + a2b0, accumulate in FP32 in TMEM, a0b0
// in one accumulator and the five small corrections in another (each MMA
// rounds into its accumulator, so the large sum is rounded once per 16
// dimensions instead of six times); the epilogue adds the two.  Both
// sides are centred on the dataset mean first, which keeps the magnitudes the
// rounding scales with small.  Norms are computed in FP64 and rounded once.
// Per-tile kernel sums are FP32, running sums per query FP64, and slices of
// the dataset meet in FP64 atomics.
//
// Roles: warp 0 lane 0 streams (3 query parts + 3 point parts) x 64 dims per
// stage by TMA (128-byte swizzle, 2 stages of 96 KiB); warp 1 lane 0 issues
// tcgen05.mma (M = 128 queries, N = 128 points, K = 16) into a double-buffered
// TMEM accumulator; warps 2-17 (one TMEM lane = one query each; four warps
// per 32-lane quadrant, each on a quarter of the tile's points) form D^2,
// apply the kernel and sum.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace deann {

namespace {

constexpr int kQM = 128;                      // queries per CTA (MMA M)
constexpr int kPN = 128;                      // points per tile (MMA N)
constexpr int kKC = 64;                       // BF16 per 128-byte row
constexpr int kParts = 3;
constexpr int kPartBytes = 128 * 128;         // 128 rows x 128 bytes
constexpr int kStageBytes = 2 * kParts * kPartBytes;  // A parts then B parts
constexpr int kStages = 2;
constexpr int kEpiWarps = 16;                 // a multiple of 4 (the TMEM lane quadrants)
constexpr int kThreads = 64 + 32 * kEpiWarps;

struct ExactShared {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

// kArgmin: the same tiles for the k-means assignment: rows are the dataset
// points, columns the centroids, and each row keeps its two nearest columns,
// (distance, column) packed as keys so that ties go to the lower column;
// amin_out receives them per slice of columns, [slice][row][2].
template <bool kArgmin>
__global__ void __launch_bounds__(kThreads, 1)
    k_exact_tc(const __grid_constant__ CUtensorMap tmap_y, const __grid_constant__ CUtensorMap tmap_x,
               const float* __restrict__ yn, const float* __restrict__ xn, int64_t nq,
               int64_t nqp, int64_t n, int dpb, int64_t rows_per_slice, int kern, float inv,
               double* __restrict__ acc_out, unsigned long long* __restrict__ amin_out,
               uint32_t* __restrict__ err) {
  __shared__ ExactShared sh;
  extern __shared__ uint8_t dyn_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t raw = tc::smem_u32(dyn_raw);
  uint8_t* ring = dyn_raw + ((1024u - (raw & 1023u)) & 1023u);
  const int64_t q0 = (int64_t)blockIdx.x * kQM;
  const int64_t x_begin = (int64_t)blockIdx.y * rows_per_slice;
  const int64_t x_end = min(n, x_begin + rows_per_slice);
  const int ntiles = x_end > x_begin ? (int)((x_end - x_begin + kPN - 1) / kPN) : 0;
  const int KB = dpb / kKC;

  if (tid == 0) {
    sh.abort = 0;
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&sh.full[s], 1);
      tc::mbar_init(&sh.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&sh.tfull[b], 1);
      tc::mbar_init(&sh.tempty[b], kEpiWarps);
    }
    tc::mbar_init(&sh.drain, 1);
    tc::fence_mbar_init();
  }
  // TMEM: two buffers x (main accumulator, correction accumulator) x kPN columns
  if (warp == 1) tc::tmem_alloc(&sh.tmem_base, 4 * kPN);
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = sh.tmem_base;
  volatile int* abort = &sh.abort;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int t = 0; t < ntiles && !*abort; ++t) {
        const int xrow = (int)(x_begin + (int64_t)t * kPN);
        for (int kb = 0; kb < KB; ++kb) {
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!tc::mbar_wait(&sh.empty[s], ph ^ 1u, abort)) break;
          uint8_t* st = ring + s * kStageBytes;
          tc::mbar_arrive_expect_tx(&sh.full[s], kStageBytes);
          for (int p = 0; p < kParts; ++p) {
            tc::tma_load_2d(st + p * kPartBytes, &tmap_y, kb * kKC, (int)(p * nqp + q0),
                            &sh.full[s]);
            tc::tma_load_2d(st + (kParts + p) * kPartBytes, &tmap_x, kb * kKC,
                            (int)(p * n + xrow), &sh.full[s]);
          }
          ++it;
        }
      }
      if (*abort) {
        volatile int no_abort = 0;
        for (int j = it > kStages ? it - kStages : 0; j < it; ++j)
          tc::mbar_wait(&sh.full[j % kStages], (uint32_t)(j / kStages) & 1u, &no_abort);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tc::make_idesc(kQM, kPN, 1u);
      // the six partial products kept: (a part, b part)
      const int pa[6] = {0, 0, 1, 0, 1, 2};
      const int pb[6] = {0, 1, 0, 2, 1, 0};
      int it = 0;
      bool ok = true;
      for (int t = 0; t < ntiles && ok; ++t) {
        const int b = t & 1;
        const uint32_t tph = (uint32_t)(t >> 1) & 1u;
        if (!tc::mbar_wait(&sh.tempty[b], tph ^ 1u, abort)) break;
        tc::tc_fence_after();
        // a0 b0 accumulates alone; the five small correction products go to
        // a second accumulator, so the large one is rounded 6x less often
        const uint32_t d_main = tmem + (uint32_t)(b * 2 * kPN);
        const uint32_t d_corr = d_main + (uint32_t)kPN;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!tc::mbar_wait(&sh.full[s], ph, abort)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t st = tc::smem_u32(ring + s * kStageBytes);
          // the parts' descriptors once per stage; a K step of 16 BF16 (32
          // bytes) adds 2 to the start-address field
          uint64_t dA[kParts], dB[kParts];
#pragma unroll
          for (int p = 0; p < kParts; ++p) {
            dA[p] = tc::desc_sw128(st + p * kPartBytes);
            dB[p] = tc::desc_sw128(st + (kParts + p) * kPartBytes);
          }
#pragma unroll
          for (int kk = 0; kk < kKC / 16; ++kk) {
#pragma unroll
            for (int j = 0; j < 6; ++j) {
              const uint64_t da = dA[pa[j]] + (uint64_t)(2 * kk);
              const uint64_t db = dB[pb[j]] + (uint64_t)(2 * kk);
              if (j == 0)
                tc::mma_f16(d_main, da, db, idesc, (kb | kk) != 0 ? 1u : 0u);
              else
                tc::mma_f16(d_corr, da, db, idesc, (kb | kk | (j - 1)) != 0 ? 1u : 0u);
            }
          }
          tc::mma_commit(&sh.empty[s]);
        }
        if (ok) tc::mma_commit(&sh.tfull[b]);
      }
      tc::mma_commit(&sh.drain);
      volatile int no_abort = 0;
      tc::mbar_wait(&sh.drain, 0u, &no_abort);
    }
  } else {
    const int lg = (warp & 3) * 32;
    // the quadrant's warps take equal runs of the tile's points
    constexpr int kRun = kPN / (kEpiWarps / 4);
    const int cbeg = ((warp - 2) >> 2) * kRun;
    const int64_t q = q0 + lg + lane;
    const bool qvalid = q < nq;
    const float ynq = qvalid ? yn[q] : 0.f;
    const bool gauss = kern == KDE_KERN_GAUSSIAN;
    const float lam = 1.4426950408889634f * inv;  // log2(e) / (2 h^2) (Gaussian)
    const float lam2 = 2.f * lam, by = -lam * ynq;
    double rowsum = 0.0;
    unsigned long long top1 = ~0ull, top2 = ~0ull;
    for (int t = 0; t < ntiles; ++t) {
      const int b = t & 1;
      const uint32_t tph = (uint32_t)(t >> 1) & 1u;
      int ok = 1;
      if (lane == 0) ok = tc::mbar_wait(&sh.tfull[b], tph, abort) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc::tc_fence_after();
      const int64_t xrow = x_begin + (int64_t)t * kPN;
      const uint32_t taddr = tmem + ((uint32_t)lg << 16) + (uint32_t)(b * 2 * kPN);
      float part = 0.f;
      const bool full = xrow + cbeg + kRun <= x_end;  // every point of the run exists
      if (kArgmin) {
        for (int c0 = cbeg; c0 < cbeg + kRun; c0 += 16) {
          uint32_t v[16];
          uint32_t w[16];
          tc::tmem_ld16(taddr + (uint32_t)c0, v);
          tc::tmem_ld16(taddr + (uint32_t)(kPN + c0), w);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int64_t pt = xrow + c0 + j;
            if (pt < x_end) {
              const float dot = __uint_as_float(v[j]) + __uint_as_float(w[j]);
              const unsigned long long key = pack_key(xn[pt] + ynq - 2.f * dot, (int)pt);
              if (key < top1) {
                top2 = top1;
                top1 = key;
              } else if (key < top2) {
                top2 = key;
              }
            }
          }
        }
      } else if (gauss && full) {
        // Gaussian: K = 2^(lam (2 <x~, y~> - |x~|^2 - |y~|^2)), lam = log2(e) / (2 h^2),
        // the exponent clamped at 0 (D^2 >= 0); the run's norms in float4 loads
        // (the same addresses on every lane)
        const float4* xn4 = reinterpret_cast<const float4*>(xn + xrow + cbeg);
        for (int c0 = 0; c0 < kRun; c0 += 16) {
          uint32_t v[16];
          uint32_t w[16];
          tc::tmem_ld16(taddr + (uint32_t)(cbeg + c0), v);
          tc::tmem_ld16(taddr + (uint32_t)(kPN + cbeg + c0), w);
          float nx[16];
#pragma unroll
          for (int j4 = 0; j4 < 4; ++j4) {
            const float4 f = xn4[(c0 >> 2) + j4];
            nx[4 * j4 + 0] = f.x;
            nx[4 * j4 + 1] = f.y;
            nx[4 * j4 + 2] = f.z;
            nx[4 * j4 + 3] = f.w;
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float dot = __uint_as_float(v[j]) + __uint_as_float(w[j]);
            const float e = fmaf(lam2, dot, fmaf(-lam, nx[j], by));
            part += exp2f(fminf(e, 0.f));
          }
        }
      } else {
        for (int c0 = cbeg; c0 < cbeg + kRun; c0 += 16) {
          uint32_t v[16];
          uint32_t w[16];
          tc::tmem_ld16(taddr + (uint32_t)c0, v);
          tc::tmem_ld16(taddr + (uint32_t)(kPN + c0), w);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int64_t pt = xrow + c0 + j;
            if (pt < x_end) {
              const float dot = __uint_as_float(v[j]) + __uint_as_float(w[j]);
              const float d2 = xn[pt] + ynq - 2.f * dot;
              part += kernel_from_dist(kern, d2, inv);
            }
          }
        }
      }
      rowsum += (double)part;
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&sh.tempty[b]);
    }
    if (kArgmin) {
      // the ring is free (every tile's MMAs completed): the four warps of
      // this lane quadrant leave their column quarter's two nearest there
      unsigned long long* top = reinterpret_cast<unsigned long long*>(ring);
      const int quarter = (warp - 2) >> 2;
      top[(quarter * kQM + lg + lane) * 2 + 0] = top1;
      top[(quarter * kQM + lg + lane) * 2 + 1] = top2;
    } else if (qvalid && ntiles > 0) {
      atomicAdd(acc_out + q, rowsum);
    }
  }
  __syncthreads();
  if (kArgmin && tid < kQM && q0 + tid < nq) {
    const unsigned long long* top = reinterpret_cast<const unsigned long long*>(ring);
    unsigned long long t1 = ~0ull, t2 = ~0ull;
    for (int qq = 0; qq < kEpiWarps / 4; ++qq)
      for (int e = 0; e < 2; ++e) {
        const unsigned long long key = top[(qq * kQM + tid) * 2 + e];
        if (key < t1) {
          t2 = t1;
          t1 = key;
        } else if (key < t2) {
          t2 = key;
        }
      }
    unsigned long long* o = amin_out + ((int64_t)blockIdx.y * nq + q0 + tid) * 2;
    o[0] = t1;
    o[1] = t2;
  }
  if (tid == 0 && sh.abort) atomicOr(err, KDE_ERRBIT_TMA);
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 4 * kPN);
  }
}

// Query-centroid squared distances for the coarse quantiser on the tensor
// cores, FP32-level: D[q][c] = |y~|^2 + |c~|^2 - 2 <y~, c~> with both sides
// centred on the dataset mean and split into three BF16 parts (the six
// products above, main and correction accumulators).  One CTA = one tile of
// 128 centroids (MMA M; a thread per centroid in the epilogue, so a warp's
// stores for one query are 32 consecutive floats) x 128 queries (MMA N).
// Rows past rows_active (a device count; may be NULL) are not computed.
constexpr int kCoarseThreads = 64 + 32 * 4;

__global__ void __launch_bounds__(kCoarseThreads, 1)
    k_coarse_tc(const __grid_constant__ CUtensorMap tmap_c, const __grid_constant__ CUtensorMap tmap_y,
                const float* __restrict__ cn, int L, const float* __restrict__ yn, int64_t nq,
                int64_t nqp, int dpb, float* __restrict__ D, const int64_t* __restrict__ active,
                int64_t row0, uint32_t* __restrict__ err) {
  __shared__ ExactShared sh;
  extern __shared__ uint8_t dyn_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = blockIdx.x * kQM;
  const int64_t q0 = (int64_t)blockIdx.y * kPN;
  if (active != nullptr && row0 + q0 >= *active) return;
  const uint32_t raw = tc::smem_u32(dyn_raw);
  uint8_t* ring = dyn_raw + ((1024u - (raw & 1023u)) & 1023u);
  const int KB = dpb / kKC;
  if (tid == 0) {
    sh.abort = 0;
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&sh.full[s], 1);
      tc::mbar_init(&sh.empty[s], 1);
    }
    tc::mbar_init(&sh.tfull[0], 1);
    tc::mbar_init(&sh.drain, 1);
    tc::fence_mbar_init();
  }
  if (warp == 1) tc::tmem_alloc(&sh.tmem_base, 2 * kPN);  // main, correction
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = sh.tmem_base;
  volatile int* abort = &sh.abort;
  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int kb = 0; kb < KB && !*abort; ++kb, ++it) {
        const int s = it % kStages;
        const uint32_t ph = (uint32_t)(it / kStages) & 1u;
        if (!tc::mbar_wait(&sh.empty[s], ph ^ 1u, abort)) break;
        uint8_t* st = ring + s * kStageBytes;
        tc::mbar_arrive_expect_tx(&sh.full[s], kStageBytes);
        for (int p = 0; p < kParts; ++p) {
          tc::tma_load_2d(st + p * kPartBytes, &tmap_c, kb * kKC, p * L + c0, &sh.full[s]);
          tc::tma_load_2d(st + (kParts + p) * kPartBytes, &tmap_y, kb * kKC,
                          (int)(p * nqp + q0), &sh.full[s]);
        }
      }
      if (*abort) {
        volatile int no_abort = 0;
        for (int j = it > kStages ? it - kStages : 0; j < it; ++j)
          tc::mbar_wait(&sh.full[j % kStages], (uint32_t)(j / kStages) & 1u, &no_abort);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tc::make_idesc(kQM, kPN, 1u);
      const int pa[6] = {0, 0, 1, 0, 1, 2};
      const int pb[6] = {0, 1, 0, 2, 1, 0};
      bool ok = true;
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
        if (!tc::mbar_wait(&sh.full[s], ph, abort)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t st = tc::smem_u32(ring + s * kStageBytes);
        uint64_t dA[kParts], dB[kParts];
#pragma unroll
        for (int p = 0; p < kParts; ++p) {
          dA[p] = tc::desc_sw128(st + p * kPartBytes);
          dB[p] = tc::desc_sw128(st + (kParts + p) * kPartBytes);
        }
#pragma unroll
        for (int kk = 0; kk < kKC / 16; ++kk) {
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            const uint64_t da = dA[pa[j]] + (uint64_t)(2 * kk);
            const uint64_t db = dB[pb[j]] + (uint64_t)(2 * kk);
            if (j == 0)
              tc::mma_f16(tmem, da, db, idesc, (kb | kk) != 0 ? 1u : 0u);
            else
              tc::mma_f16(tmem + kPN, da, db, idesc, (kb | kk | (j - 1)) != 0 ? 1u : 0u);
          }
        }
        tc::mma_commit(&sh.empty[s]);
      }
      if (ok) tc::mma_commit(&sh.tfull[0]);
      tc::mma_commit(&sh.drain);
      volatile int no_abort = 0;
      tc::mbar_wait(&sh.drain, 0u, &no_abort);
    }
  } else {
    // one TMEM lane = one centroid per thread
    const int lg = (warp & 3) * 32;
    const int c = c0 + lg + lane;
    int ok = 1;
    if (lane == 0) ok = tc::mbar_wait(&sh.tfull[0], 0u, abort) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
      tc::tc_fence_after();
      const float cnc = c < L ? cn[c] : 0.f;
      const uint32_t taddr = tmem + ((uint32_t)lg << 16);
      for (int j0 = 0; j0 < kPN; j0 += 16) {
        uint32_t v[16], w[16];
        tc::tmem_ld16(taddr + (uint32_t)j0, v);
        tc::tmem_ld16(taddr + (uint32_t)(kPN + j0), w);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int64_t q = q0 + j0 + j;
          if (c < L && q < nq) {
            const float dot = __uint_as_float(v[j]) + __uint_as_float(w[j]);
            D[q * L + c] = fmaxf(yn[q] + cnc - 2.f * dot, 0.f);
          }
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0 && sh.abort) atomicOr(err, KDE_ERRBIT_TMA);
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 2 * kPN);
  }
}

// Three-way BF16 split of (v - mean) for rows of a row-major FP32 matrix:
// part p of row r goes to dst[(p * rows_pad + r) * dpb + j].  The squared
// norm of (v - mean) is accumulated in FP64 and rounded once.
__global__ void k_split3(const float* __restrict__ V, int64_t rows, int dp, const float* __restrict__ mean,
                         __nv_bfloat16* __restrict__ dst, int64_t rows_pad, int dpb,
                         float* __restrict__ norms) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  double s = 0.0;
  for (int j = lane; j < dpb; j += 32) {
    const float v = j < dp ? V[r * dp + j] - mean[j] : 0.f;
    const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(b0);
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b1);
    const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
    dst[(0 * rows_pad + r) * dpb + j] = b0;
    dst[(1 * rows_pad + r) * dpb + j] = b1;
    dst[(2 * rows_pad + r) * dpb + j] = b2;
    s += (double)v * (double)v;
  }
  s = warp_sum_d(s);
  if (lane == 0) norms[r] = (float)s;
}

// Column sums of X in FP64 over fixed row slices: block (bx, by) sums rows
// [by * rows, (by + 1) * rows) of the 32 columns from 32 bx, a warp per 32
// rows at a time in row order, then its 8 warps in order; part[by][j].
__global__ void k_col_partial(const float* __restrict__ X, int64_t n, int dp, int64_t rows,
                              double* __restrict__ part) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const int64_t r0 = (int64_t)blockIdx.y * rows, r1 = min(n, r0 + rows);
  double s = 0.0;
  if (j < dp)
    for (int64_t i = r0 + warp; i < r1; i += 8) s += (double)X[i * dp + j];
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && j < dp) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][lane];
    part[(int64_t)blockIdx.y * dp + j] = t;
  }
}

// Column means from the slices' partial sums, added in slice order.
__global__ void k_col_finish(const double* __restrict__ part, int slices, int64_t n, int dp,
                             float* __restrict__ mean) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= dp) return;
  double s = 0.0;
  for (int b = 0; b < slices; ++b) s += part[(int64_t)b * dp + j];
  mean[j] = (float)(s / (double)n);
}

__global__ void k_exact_finish_tc(const double* __restrict__ acc, int64_t nq, double inv_n,
                                  float* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nq) out[q] = (float)(acc[q] * inv_n);
}

// The assignment's last step: the two nearest centroids by the tensor-core
// distances (merged over the slices) are compared again by their FP32
// difference-form distances, one warp per point, ties to the lower id, so
// that the split distances' rounding (which scales with |x~|^2 + |c~|^2,
// not with the distance) cannot flip a near tie.
__global__ void k_assign_finish(const unsigned long long* __restrict__ top, int slices,
                                int64_t np, const float* __restrict__ X,
                                const float* __restrict__ C, int d, int dp,
                                int32_t* __restrict__ assign, float* __restrict__ best_d2) {
  const int lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (p >= np) return;
  unsigned long long t1 = ~0ull, t2 = ~0ull;
  for (int s = 0; s < slices; ++s)
    for (int e = 0; e < 2; ++e) {
      const unsigned long long key = top[((int64_t)s * np + p) * 2 + e];
      if (key < t1) {
        t2 = t1;
        t1 = key;
      } else if (key < t2) {
        t2 = key;
      }
    }
  const int c1 = (int)(t1 & 0xffffffffull);
  const int c2 = t2 == ~0ull ? c1 : (int)(t2 & 0xffffffffull);
  const float* x = X + p * dp;
  float s1 = 0.f, s2 = 0.f;
  for (int j = lane; j < d; j += 32) {
    const float a = x[j] - C[(int64_t)c1 * dp + j], b = x[j] - C[(int64_t)c2 * dp + j];
    s1 = fmaf(a, a, s1);
    s2 = fmaf(b, b, s2);
  }
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    const bool second = s2 < s1 || (s2 == s1 && c2 < c1);
    assign[p] = second ? c2 : c1;
    if (best_d2) best_d2[p] = second ? s2 : s1;
  }
}

bool encode_parts_map(CUtensorMap* map, const void* base, int64_t rows_total, int dpb) {
  tc::EncodeTiledFn enc = tc::tensor_map_encoder();
  if (enc == nullptr) return false;
  cuuint64_t dims[2] = {(cuuint64_t)dpb, (cuuint64_t)rows_total};
  cuuint64_t strides[1] = {(cuuint64_t)dpb * 2};
  cuuint32_t box[2] = {(cuuint32_t)kKC, 128u};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t exact_tc_smem() { return 1024 + (size_t)kStages * kStageBytes; }

int col_mean_slices(int64_t n) { return (int)std::min<int64_t>(256, (n + 4095) / 4096); }

void launch_col_mean(const float* X, int64_t n, int dp, float* mean, double* part,
                     cudaStream_t s) {
  const int slices = col_mean_slices(n);
  const int64_t rows = (n + slices - 1) / slices;
  k_col_partial<<<dim3((unsigned)((dp + 31) / 32), (unsigned)slices), 256, 0, s>>>(X, n, dp, rows,
                                                                                 part);
  k_col_finish<<<(unsigned)((dp + 127) / 128), 128, 0, s>>>(part, slices, n, dp, mean);
}

bool launch_coarse_tc(const void* tmap_c, const float* cn, int L, const void* Ys, const float* yn,
                      int64_t nq, int dpb, float* D, const int64_t* active, int64_t row0,
                      uint32_t* err, cudaStream_t s) {
  if (nq <= 0) return true;
  CUtensorMap tmap_y;
  if (!encode_parts_map(&tmap_y, Ys, kParts * nq, dpb)) return false;
  if (!set_dynamic_smem(reinterpret_cast<const void*>(&k_coarse_tc), exact_tc_smem()))
    return false;
  const dim3 grid((unsigned)((L + kQM - 1) / kQM), (unsigned)((nq + kPN - 1) / kPN));
  k_coarse_tc<<<grid, kCoarseThreads, exact_tc_smem(), s>>>(
      *reinterpret_cast<const CUtensorMap*>(tmap_c), tmap_y, cn, L, yn, nq, nq, dpb, D, active,
      row0, err);
  return true;
}

void launch_split3(const float* V, int64_t rows, int dp, const float* mean, void* dst,
                   int64_t rows_pad, int dpb, float* norms, cudaStream_t s) {
  if (rows <= 0) return;
  k_split3<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(
      V, rows, dp, mean, reinterpret_cast<__nv_bfloat16*>(dst), rows_pad, dpb, norms);
}

bool make_parts_map(void* map_out, const void* base, int64_t rows_total, int dpb) {
  return encode_parts_map(reinterpret_cast<CUtensorMap*>(map_out), base, rows_total, dpb);
}


bool launch_exact_tc(const void* tmap_x, const void* Ys, const float* yn, int64_t nq, int64_t nqp,
                     const float* xn, int64_t n, int dpb, int kern, float h, double* acc,
                     float* out, uint32_t* err, cudaStream_t s) {
  CUtensorMap tmap_y;
  if (!encode_parts_map(&tmap_y, Ys, kParts * nqp, dpb)) return false;
  if (!set_dynamic_smem(reinterpret_cast<const void*>(&k_exact_tc<false>), exact_tc_smem()))
    return false;
  cudaMemsetAsync(acc, 0, sizeof(double) * nq, s);
  const int64_t qtiles = (nq + kQM - 1) / kQM;
  // about two waves of the 152 SMs (one CTA per SM), slices of whole tiles
  const int64_t ptiles = (n + kPN - 1) / kPN;
  int64_t slices = (2 * 152 + qtiles - 1) / qtiles;
  if (slices > ptiles) slices = ptiles;
  if (slices < 1) slices = 1;
  const int64_t rows_per_slice = ((ptiles + slices - 1) / slices) * kPN;
  slices = (n + rows_per_slice - 1) / rows_per_slice;
  const dim3 grid((unsigned)qtiles, (unsigned)slices);
  k_exact_tc<false><<<grid, kThreads, exact_tc_smem(), s>>>(
      tmap_y, *reinterpret_cast<const CUtensorMap*>(tmap_x), yn, xn, nq, nqp, n, dpb,
      rows_per_slice, kern, kernel_inv(kern, h), acc, nullptr, err);
  k_exact_finish_tc<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(acc, nq, 1.0 / (double)n, out);
  return true;
}

int assign_tc_slices(int64_t np, int L) {
  // about two waves of the 152 SMs, slices of whole centroid tiles
  const int64_t ptiles = (np + kQM - 1) / kQM;
  const int64_t ctiles = (L + kPN - 1) / kPN;
  int64_t slices = (2 * 152 + ptiles - 1) / ptiles;
  if (slices > ctiles) slices = ctiles;
  if (slices < 1) slices = 1;
  const int64_t cols_per_slice = ((ctiles + slices - 1) / slices) * kPN;
  return (int)((L + cols_per_slice - 1) / cols_per_slice);
}

bool launch_assign_tc(const void* tmap_p, const float* pn, int64_t np, const void* tmap_c,
                      const float* cn, int L, int dpb, const float* X, const float* C, int d,
                      int dp, unsigned long long* amin, int32_t* assign, float* best_d2,
                      uint32_t* err, cudaStream_t s) {
  if (np <= 0) return true;
  if (!set_dynamic_smem(reinterpret_cast<const void*>(&k_exact_tc<true>), exact_tc_smem()))
    return false;
  const int64_t ptiles = (np + kQM - 1) / kQM;
  // about two waves of the 152 SMs, slices of whole centroid tiles
  const int64_t ctiles = (L + kPN - 1) / kPN;
  int64_t slices = (2 * 152 + ptiles - 1) / ptiles;
  if (slices > ctiles) slices = ctiles;
  if (slices < 1) slices = 1;
  const int64_t cols_per_slice = ((ctiles + slices - 1) / slices) * kPN;
  slices = (L + cols_per_slice - 1) / cols_per_slice;
  const dim3 grid((unsigned)ptiles, (unsigned)slices);
  k_exact_tc<true><<<grid, kThreads, exact_tc_smem(), s>>>(
      *reinterpret_cast<const CUtensorMap*>(tmap_p), *reinterpret_cast<const CUtensorMap*>(tmap_c),
      pn, cn, np, np, L, dpb, cols_per_slice, KDE_KERN_GAUSSIAN, 1.f, nullptr, amin, err);
  k_assign_finish<<<(unsigned)((np + 7) / 8), 256, 0, s>>>(amin, (int)slices, np, X, C, d, dp,
                                                           assign, best_d2);
  return true;
}

}  // namespace deann
