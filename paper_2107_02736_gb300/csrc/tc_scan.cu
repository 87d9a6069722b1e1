// IVF list scan on the 5th-generation tensor cores (tcgen05), BF16 operands,
// FP32 accumulation in TMEM.
//
// Squared distances by the identity |x - y|^2 = |x|^2 + |y|^2 - 2 <x, y>
// (paper Appendix D, Eq. "d2"): the inner products of one IVF list's points
// with the queries that probe that list form one GEMM, D = X_list Y^T.
//
// One CTA = one (list, group of up to BN probing queries).  Roles:
//   warp 0 (one lane): TMA producer, streams 128-point x 64-dim BF16 tiles of
//                      the list (128-byte swizzle) through a ring of stages;
//   warp 1 (one lane): MMA issuer, tcgen05.mma M=128 (points) x N (the
//                      CTA's queries rounded up to 16, at most BN) x K=16
//                      into a double-buffered TMEM
//                      accumulator; warp 1 also owns the TMEM allocation;
//   warps 2-9        : epilogue, one TMEM lane (= one list point) per thread:
//                      D^2 = |x|^2 + |y|^2 - 2 acc, clamped at 0, written to
//                      each query's candidate segment (coalesced along points;
//                      the segment's padding to 32 floats gets +inf).  Two
//                      warps share each 32-lane TMEM quadrant and take
//                      alternate groups of 16 query columns, so twice as many
//                      warps keep candidate stores in flight.
// Both operands are centred on the list's centroid c_l (x~ = x - c_l, stored
// that way at build time; y~ = y - c_l, formed here), which leaves the
// distances unchanged but shrinks the magnitudes that the rounding error
// scales with from |x||y| to |x~||y~|.  The centred queries (B operand) are
// staged once per CTA by all threads into the swizzled layout and stay
// resident for the whole list.
//
// Two operand precisions (template Split):
//   plain BF16: one part each, one MMA per 16 dimensions; the distances only
//     rank candidates, and the selection rescores the best in FP32
//     difference form;
//   three-way split: every operand v = v0 + v1 + v2 in BF16 (to 2^-27 |v|),
//     the six products that carry weight down to 2^-24 (a0b0 into a main
//     accumulator, a0b1 + a1b0 + a0b2 + a1b1 + a2b0 into a correction one, so
//     the large sum is rounded six times less often), squared norms carried
//     beyond FP32 (the points' in FP64 at build, the queries' as double-word
//     FP32 sums) and rounded once:
//     FP32-level distances, which the selection uses as they are.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace deann {

namespace {

constexpr int kBM = 128;          // points per tile (MMA M)
constexpr int kBK = 64;           // BF16 elements per 128-byte row chunk
constexpr int kPartBytes = kBM * 128;  // one part of one 128 x 64 tile
constexpr int kEpiWarps = 8;     // epilogue warps, a multiple of 4 (the TMEM lane quadrants)
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kMaxStages = 4;
constexpr int kAhead = 2;  // tiles of the list requested into L2 ahead of their loads
// plain BF16: 3 stages of one part (so that two CTAs fit an SM at d <= 128);
// split: 2 stages of three parts
template <bool Split>
struct ScanCfg {
  static constexpr int kParts = Split ? 3 : 1;
  static constexpr int kStages = Split ? 2 : 3;
  static constexpr int kStageBytes = kParts * kPartBytes;
};
constexpr size_t kDynBudget = 222 * 1024;  // dynamic shared memory of one CTA (+ ~4 KB static)

struct ScanShared {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
  int list;
  int pos;  // the list's place in the scan order
  int issued;  // ring loads issued before the queries' staging
  int64_t dst[256];
  float yn[256];
  int qrow[256];
};

template <bool Split>
__global__ void __launch_bounds__(kThreads, 1)
    k_scan_tc(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ Yp,
              const float* __restrict__ C, int dp, const float* __restrict__ XLcn, int64_t n,
              const int64_t* __restrict__ list_off, int L, int dpb, int BN,
              const int32_t* __restrict__ pair_q, const int64_t* __restrict__ pair_dst,
              const int64_t* __restrict__ bucket_off, const int64_t* __restrict__ tile_off,
              const int32_t* __restrict__ lorder, float* __restrict__ cand,
              uint32_t* __restrict__ err) {
  using Cfg = ScanCfg<Split>;
  constexpr int kParts = Cfg::kParts, kStages = Cfg::kStages, kStageBytes = Cfg::kStageBytes;
  __shared__ ScanShared sh;
  extern __shared__ uint8_t dyn_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t t = blockIdx.x;
  if (t >= tile_off[L]) return;

  // 1024-byte aligned operand area: A ring, then the resident B parts
  const uint32_t raw = tc::smem_u32(dyn_raw);
  uint8_t* base = dyn_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t* A = base;
  uint8_t* B = base + kStages * kStageBytes;
  const int KB = dpb / kBK;
  const size_t b_part = (size_t)KB * BN * 128;  // one part of the resident queries

  int pos0 = 0;
  if (warp == 0) {
    // the list of tile t: the last scan position whose first tile is <= t,
    // found by warp 0 in 32-way steps (tile_off is nondecreasing and
    // tile_off[0] = 0 <= t)
    int lo = 0, hi = L - 1;
    while (hi - lo >= 32) {
      const int step = (hi - lo + 32) / 32;
      const int probe = lo + lane * step;
      const unsigned m = __ballot_sync(0xffffffffu, probe <= hi && tile_off[probe] <= t);
      lo += (31 - __clz(m)) * step;
      hi = min(hi, lo + step - 1);
    }
    const int probe = lo + lane;
    const unsigned m = __ballot_sync(0xffffffffu, probe <= hi && tile_off[probe] <= t);
    pos0 = lo + 31 - __clz(m);
  }
  if (tid == 0) {
    sh.pos = pos0;
    sh.list = lorder[pos0];
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
    // the ring is empty: its first loads go out now, ahead of the queries'
    // staging (the producer below continues from sh.issued)
    const int l0 = sh.list;
    const int64_t xb0 = list_off[l0];
    const int nt0 = (int)((list_off[l0 + 1] - xb0 + kBM - 1) / kBM);
    const int total = nt0 * (dpb / kBK);
    int it = 0;
    for (; it < kStages && it < total; ++it) {
      const int tt = it / (dpb / kBK), kb = it - tt * (dpb / kBK);
      tc::mbar_arrive_expect_tx(&sh.full[it], kStageBytes);
      const int row = (int)(xb0 + (int64_t)tt * kBM);
#pragma unroll
      for (int p = 0; p < kParts; ++p)
        tc::tma_load_2d(A + it * kStageBytes + p * kPartBytes, &tmap, kb * kBK,
                        (int)((int64_t)p * n + row), &sh.full[it]);
    }
    sh.issued = it;
    // and the next kAhead tiles are requested into L2, so that their loads,
    // when the ring frees, wait on L2 rather than HBM
    for (int tt = 1; tt <= kAhead && tt < nt0; ++tt)
      for (int kb = 0; kb < dpb / kBK; ++kb)
#pragma unroll
        for (int p = 0; p < kParts; ++p)
          tc::tma_prefetch_2d(&tmap, kb * kBK, (int)((int64_t)p * n + xb0 + (int64_t)tt * kBM));
  }
  __syncthreads();
  const int l = sh.list;
  const int64_t pb = bucket_off[l] + (t - tile_off[sh.pos]) * BN;
  const int64_t left_pairs = bucket_off[l + 1] - pb;
  const int npairs = left_pairs < (int64_t)BN ? (int)left_pairs : BN;
  // the MMA's N: this CTA's queries rounded up to a multiple of 16 (rows past
  // npairs are zero and their columns are never read)
  const int nN = (npairs + 15) & ~15;
  const int64_t xb = list_off[l];
  const int64_t len = list_off[l + 1] - xb;
  const int ntiles = (int)((len + kBM - 1) / kBM);

  // this CTA's queries (ids and candidate destinations), all loads at once
  for (int r = tid; r < nN; r += kThreads) {
    sh.qrow[r] = r < npairs ? pair_q[pb + r] : -1;
    sh.dst[r] = r < npairs ? pair_dst[pb + r] : -1;
  }
  __syncthreads();
  // stage the queries centred on this list's centroid, y~ = y - c_l, in BF16
  // (split: three parts): row r of block kb of part p at
  // B + p*b_part + kb*BN*128 + r*128, 16-byte chunk c stored at chunk
  // position c ^ (r & 7) (the 128-byte swizzle), and |y~|^2 (for the split
  // scan as a double-word FP32 sum, rounded once).  G lanes take the C8 chunks of 8 dimensions of
  // one row (G the smallest power of two >= C8, at most 32), so a warp stages
  // 32 / G rows at once, two such groups of rows with their loads issued
  // together; a row's chunk sums are added over its lanes in a fixed order.
  {
    const float* cl = C + (int64_t)l * dp;
    const int C8 = KB * 8;
    int G = 32;
    while (G / 2 >= C8) G >>= 1;
    const int R = 32 / G, gl = lane & (G - 1), gr = lane / G;
    constexpr int kU = 2;
    const int rstep = (kThreads / 32) * R;
    for (int r0 = warp * R; r0 < nN; r0 += kU * rstep) {
      float sh_[kU], sl_[kU];  // |y~|^2 as an unevaluated sum hi + lo (split) or plain (sh_)
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        sh_[u] = 0.f;
        sl_[u] = 0.f;
      }
      for (int c8 = gl; c8 < C8; c8 += G) {
        const int kb = c8 >> 3, c = c8 & 7, j0 = c8 * 8;
        float4 y[kU][2];
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 c0 = j0 < dp ? *reinterpret_cast<const float4*>(cl + j0) : z;
        const float4 c1 = j0 + 4 < dp ? *reinterpret_cast<const float4*>(cl + j0 + 4) : z;
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int r = r0 + u * rstep + gr;
          const int qr = r < nN ? sh.qrow[r] : -1;
          const float* yq = Yp + (int64_t)(qr >= 0 ? qr : 0) * dp;
          y[u][0] = qr >= 0 && j0 < dp ? *reinterpret_cast<const float4*>(yq + j0) : c0;
          y[u][1] = qr >= 0 && j0 + 4 < dp ? *reinterpret_cast<const float4*>(yq + j0 + 4) : c1;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int r = r0 + u * rstep + gr;
          if (r >= nN) continue;
          const float f[8] = {y[u][0].x - c0.x, y[u][0].y - c0.y, y[u][0].z - c0.z,
                              y[u][0].w - c0.w, y[u][1].x - c1.x, y[u][1].y - c1.y,
                              y[u][1].z - c1.z, y[u][1].w - c1.w};
          uint32_t w[kParts][4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const float f0 = f[2 * t], f1 = f[2 * t + 1];
            const __nv_bfloat162 h0 = __floats2bfloat162_rn(f0, f1);
            w[0][t] = *reinterpret_cast<const uint32_t*>(&h0);
            if (Split) {
              const float2 g0 = __bfloat1622float2(h0);
              const float e0 = f0 - g0.x, e1 = f1 - g0.y;  // exact
              const __nv_bfloat162 h1 = __floats2bfloat162_rn(e0, e1);
              const float2 g1 = __bfloat1622float2(h1);
              const __nv_bfloat162 h2 = __floats2bfloat162_rn(e0 - g1.x, e1 - g1.y);
              w[kParts > 1 ? 1 : 0][t] = *reinterpret_cast<const uint32_t*>(&h1);
              w[kParts > 2 ? 2 : 0][t] = *reinterpret_cast<const uint32_t*>(&h2);
              // squares exact as p + e (FMA), added with TwoSum: the
              // double-word sum carries far more than the FP32 result keeps
              const float p0 = f0 * f0, q0 = fmaf(f0, f0, -p0);
              const float p1 = f1 * f1, q1 = fmaf(f1, f1, -p1);
              float t0, d0, t1, d1;
              two_sum(sh_[u], p0, t0, d0);
              two_sum(t0, p1, t1, d1);
              sh_[u] = t1;
              sl_[u] += (d0 + d1) + (q0 + q1);
            } else {
              sh_[u] = fmaf(f0, f0, fmaf(f1, f1, sh_[u]));
            }
          }
#pragma unroll
          for (int p = 0; p < kParts; ++p)
            *reinterpret_cast<uint4*>(B + p * b_part + (size_t)kb * BN * 128 + r * 128 +
                                      ((c ^ (r & 7)) << 4)) =
                make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        for (int o = G / 2; o > 0; o >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, sh_[u], o);
          const float ol = __shfl_xor_sync(0xffffffffu, sl_[u], o);
          if (Split) {
            float t, d;
            two_sum(sh_[u], oh, t, d);
            sh_[u] = t;
            sl_[u] += ol + d;
          } else {
            sh_[u] += oh;
          }
        }
        const int r = r0 + u * rstep + gr;
        if (gl == 0 && r < nN) sh.yn[r] = sh.qrow[r] >= 0 ? sh_[u] + sl_[u] : 0.f;
      }
    }
  }
  tc::fence_proxy_async_smem();
  // TMEM: two accumulator buffers of BN columns (split: main and correction
  // accumulators in each)
  const uint32_t acc_cols = (uint32_t)(Split ? 2 * BN : BN);
  uint32_t ncols = 32;
  while (ncols < 2 * acc_cols) ncols <<= 1;
  if (warp == 1) tc::tmem_alloc(&sh.tmem_base, ncols);
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = sh.tmem_base;
  volatile int* abort = &sh.abort;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int it = 0;  // loads issued so far
      const int pre = sh.issued;
      for (int tt = 0; tt < ntiles && !*abort; ++tt) {
        if (tt >= 1 && tt + kAhead < ntiles) {
          const int prow = (int)(xb + (int64_t)(tt + kAhead) * kBM);
          for (int kb = 0; kb < KB; ++kb)
#pragma unroll
            for (int p = 0; p < kParts; ++p)
              tc::tma_prefetch_2d(&tmap, kb * kBK, (int)((int64_t)p * n + prow));
        }
        for (int kb = 0; kb < KB; ++kb) {
          if (it < pre) {  // issued before the staging
            ++it;
            continue;
          }
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!tc::mbar_wait(&sh.empty[s], ph ^ 1u, abort)) break;
          tc::mbar_arrive_expect_tx(&sh.full[s], kStageBytes);
          const int row = (int)(xb + (int64_t)tt * kBM);
#pragma unroll
          for (int p = 0; p < kParts; ++p)
            tc::tma_load_2d(A + s * kStageBytes + p * kPartBytes, &tmap, kb * kBK,
                            (int)((int64_t)p * n + row), &sh.full[s]);
          ++it;
        }
      }
      if (*abort) {
        // let the last (at most kStages) loads land before the CTA's shared
        // memory goes away; every earlier load was consumed by the MMA warp
        volatile int no_abort = 0;
        if (it < pre) it = pre;
        for (int j = it > kStages ? it - kStages : 0; j < it; ++j)
          tc::mbar_wait(&sh.full[j % kStages], (uint32_t)(j / kStages) & 1u, &no_abort);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = tc::make_idesc(kBM, nN, 1u);
      // split: the six partial products kept, (point part, query part)
      const int pa[6] = {0, 0, 1, 0, 1, 2};
      const int pq[6] = {0, 1, 0, 2, 1, 0};
      int it = 0;
      bool ok = true;
      for (int tt = 0; tt < ntiles && ok; ++tt) {
        const int b = tt & 1;
        const uint32_t tph = (uint32_t)(tt >> 1) & 1u;
        if (!tc::mbar_wait(&sh.tempty[b], tph ^ 1u, abort)) break;
        tc::tc_fence_after();
        const uint32_t d_main = tmem + (uint32_t)b * acc_cols;
        const uint32_t d_corr = d_main + (uint32_t)BN;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!tc::mbar_wait(&sh.full[s], ph, abort)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t a0 = tc::smem_u32(A + s * kStageBytes);
          const uint32_t b0 = tc::smem_u32(B + (size_t)kb * BN * 128);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            if (!Split) {
              tc::mma_f16(d_main, tc::desc_sw128(a0 + kk * 32), tc::desc_sw128(b0 + kk * 32),
                          idesc, (kb | kk) != 0 ? 1u : 0u);
            } else {
#pragma unroll
              for (int j = 0; j < 6; ++j) {
                const uint64_t da = tc::desc_sw128(a0 + pa[j] * kPartBytes + kk * 32);
                const uint64_t db =
                    tc::desc_sw128(b0 + (uint32_t)(pq[j] * b_part) + kk * 32);
                if (j == 0)
                  tc::mma_f16(d_main, da, db, idesc, (kb | kk) != 0 ? 1u : 0u);
                else
                  tc::mma_f16(d_corr, da, db, idesc, (kb | kk | (j - 1)) != 0 ? 1u : 0u);
              }
            }
          }
          tc::mma_commit(&sh.empty[s]);
        }
        if (ok) tc::mma_commit(&sh.tfull[b]);
      }
      // all issued MMAs complete before TMEM is released
      tc::mma_commit(&sh.drain);
      volatile int no_abort = 0;
      tc::mbar_wait(&sh.drain, 0u, &no_abort);
    }
  } else {
    // ---------------- epilogue: warps 2..9 ----------------
    // one TMEM lane (= one list point) per thread.  A warp reads only its own
    // lane quadrant (warp id mod 4); the second warp of a quadrant starts at
    // column 16.  Each group of 16 query columns goes through a 16 x 32
    // transpose tile in shared memory, so that every lane stores 4
    // consecutive points of one query with one 16-byte store: a warp's store
    // instruction covers 128 bytes of four queries' candidate segments.
    // Points past the list up to its 32-float padded length get +inf (the
    // segment's padding).
    const int lg = (warp & 3) * 32;
    const int cstart = ((warp - 2) >> 2) * 16;
    constexpr int cstep = 16 * (kEpiWarps / 4);
    const int row = lg + lane;
    const int64_t padlen = (len + 31) & ~(int64_t)31;
    float* tp = reinterpret_cast<float*>(B + kParts * b_part) + (warp - 2) * (16 * 32);
    const int tj = lane >> 3, ti = lane & 7;  // the lane's column (+ 4 g) and row quad
    // the point norms of the next tile are loaded while this one's
    // accumulator is awaited and stored
    float xn_next = row < len ? XLcn[xb + row] : 0.f;
    for (int tt = 0; tt < ntiles; ++tt) {
      const int b = tt & 1;
      const uint32_t tph = (uint32_t)(tt >> 1) & 1u;
      const int64_t pt = (int64_t)tt * kBM + row;
      const bool valid = pt < len;
      // the warp's 32 points lie in the segment's padded length, or all past it
      const bool live = (int64_t)tt * kBM + lg < padlen;
      const float xn = xn_next;
      xn_next = pt + kBM < len ? XLcn[xb + pt + kBM] : 0.f;
      int ok = 1;
      if (lane == 0) ok = tc::mbar_wait(&sh.tfull[b], tph, abort) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc::tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)lg << 16) + (uint32_t)b * acc_cols;
      float* dst_tile = cand + (int64_t)tt * kBM + lg + 4 * ti;
      for (int c0 = cstart; c0 < npairs && live; c0 += cstep) {
        uint32_t v[16];
        tc::tmem_ld16(taddr + (uint32_t)c0, v);
        if (Split) {
          uint32_t w[16];
          tc::tmem_ld16(taddr + (uint32_t)(BN + c0), w);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            v[j] = __float_as_uint(__uint_as_float(v[j]) + __uint_as_float(w[j]));
        }
#pragma unroll
        for (int j = 0; j < 16; ++j)
          tp[j * 32 + lane] = valid ? fmaxf(xn + sh.yn[c0 + j] - 2.f * __uint_as_float(v[j]), 0.f)
                                    : __int_as_float(0x7f800000);
        __syncwarp();
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int j = tj + 4 * g, col = c0 + j;
          const float4 q4 = *reinterpret_cast<const float4*>(tp + j * 32 + 4 * ti);
          if (col < npairs) *reinterpret_cast<float4*>(dst_tile + sh.dst[col]) = q4;
        }
        __syncwarp();
      }
      // the accumulator was read synchronously (tcgen05.wait::ld): a relaxed
      // arrive frees it without waiting for this tile's stores to land
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive_relaxed(&sh.tempty[b]);
    }
  }
  __syncthreads();
  if (tid == 0 && sh.abort) atomicOr(err, KDE_ERRBIT_TMA);
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, ncols);
  }
}

}  // namespace

size_t scan_tc_smem(int dpb, int BN, bool split) {
  // alignment slack, the A ring, the resident queries, the epilogue warps'
  // transpose tiles
  const size_t ring = split ? (size_t)ScanCfg<true>::kStages * ScanCfg<true>::kStageBytes
                            : (size_t)ScanCfg<false>::kStages * ScanCfg<false>::kStageBytes;
  return 1024 + ring + (size_t)(split ? 3 : 1) * (dpb / kBK) * BN * 128 +
         (size_t)kEpiWarps * 16 * 32 * sizeof(float);
}

int scan_tc_bn(int dpb, bool split) {
  // the largest multiple of 16 (at most 128) whose operands fit; 0 if none
  int bn = 128;
  while (bn > 16 && scan_tc_smem(dpb, bn, split) > kDynBudget) bn -= 16;
  return scan_tc_smem(dpb, bn, split) <= kDynBudget ? bn : 0;
}

bool make_bf16_row_map(void* map_out, const void* base, int64_t rows, int dpb) {
  tc::EncodeTiledFn enc = tc::tensor_map_encoder();
  if (enc == nullptr) return false;
  CUtensorMap* map = reinterpret_cast<CUtensorMap*>(map_out);
  cuuint64_t dims[2] = {(cuuint64_t)dpb, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)dpb * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool launch_scan_tc(bool split, const void* tmap, const float* Yp, const float* C, int dp,
                    const float* xn, int64_t n, const int64_t* list_off, int L, int dpb, int BN,
                    const ScanPlan& plan, float* cand, uint32_t* err, cudaStream_t s) {
  if (plan.max_tiles <= 0) return true;
  if (BN < 16 || BN > 128 || BN % 16 != 0) return false;
  const size_t smem = scan_tc_smem(dpb, BN, split);
  const CUtensorMap& map = *reinterpret_cast<const CUtensorMap*>(tmap);
  const unsigned grid = (unsigned)plan.max_tiles;
  if (split) {
    if (!set_dynamic_smem(reinterpret_cast<const void*>(&k_scan_tc<true>), smem)) return false;
    k_scan_tc<true><<<grid, kThreads, smem, s>>>(map, Yp, C, dp, xn, n, list_off, L, dpb, BN,
                                                 plan.pair_q, plan.pair_dst, plan.bucket_off,
                                                 plan.tile_off, plan.lorder, cand, err);
  } else {
    if (!set_dynamic_smem(reinterpret_cast<const void*>(&k_scan_tc<false>), smem)) return false;
    k_scan_tc<false><<<grid, kThreads, smem, s>>>(map, Yp, C, dp, xn, n, list_off, L, dpb, BN,
                                                  plan.pair_q, plan.pair_dst, plan.bucket_off,
                                                  plan.tile_off, plan.lorder, cand, err);
  }
  return true;
}

}  // namespace deann
