// IVF list scan on the 5th-generation tensor cores (tcgen05), BF16 operands,
// FP32 accumulation in TMEM.
//
// Squared distances by the identity |x - y|^2 = |x|^2 + |y|^2 - 2 <x, y>
// (paper Appendix D, Eq. "d2"): the inner products of one IVF list's points
// with the queries that probe that list form one GEMM, D = X_list Y^T.
//
// One CTA = one (list, group of up to BN probing queries).  Roles:
//   warp 0 (one lane): TMA producer, streams 128-point x 64-dim BF16 tiles of
//                      the list (128-byte swizzle) through a 4-stage ring;
//   warp 1 (one lane): MMA issuer, tcgen05.mma M=128 (points) x N (the
//                      CTA's queries rounded up to 16, at most BN) x K=16
//                      into a double-buffered TMEM
//                      accumulator; warp 1 also owns the TMEM allocation;
//   warps 2-9        : epilogue, one TMEM lane (= one list point) per thread,
//                      D^2 = |x|^2 + |y|^2 - 2 acc clamped at 0.  Two warps
//                      share each 32-lane TMEM quadrant and take alternate
//                      groups of 16 query columns.
// Both operands are centred on the list's centroid c_l (x~ = x - c_l, stored
// that way at build time; y~ = y - c_l, formed here), which leaves the
// distances unchanged but shrinks the magnitudes that the BF16 rounding error
// scales with from |x||y| to |x~||y~|.  The centred queries (B operand) are
// staged once per CTA by all threads into the swizzled layout and stay
// resident for the whole list.
//
// What the epilogue does with D^2 (the launch's mode):
//   kScanCand  writes it to each query's candidate segment (coalesced along
//              points; a segment's padding to 32 floats gets +inf);
//   kScanHist  counts it into the query's histogram (shared memory per CTA,
//              added to the query's global histogram at the end): the first
//              pass of the two-pass selection;
//   kScanRefine for a query whose k-th bin holds many candidates, counts the
//              candidates of that bin into sub-bins (a CTA with no such query
//              returns at once);
//   kScanEmit  the last pass: for the points whose bin (or sub-bin) lies below
//              the query's k-th (region A) or whose D^2 is within the band
//              edge (region B), the warp computes the FP32 difference-form
//              distance from the list-ordered FP32 rows, eight lanes per
//              (point, query) pair, and appends its (distance, id) key.  The
//              rows of a list are shared by the CTA's queries, so the
//              rescoring reads them from L1/L2 rather than once per query.
// The approximate distances only rank candidates; returned distances and
// kernel values always come from FP32 difference-form rescoring.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace deann {

namespace {

constexpr int kBM = 128;          // points per tile (MMA M)
constexpr int kBK = 64;           // BF16 elements per 128-byte row chunk
constexpr int kStages = 4;
constexpr int kStageBytes = kBM * 128;
constexpr int kEpiWarps = 8;     // epilogue warps, a multiple of 4 (the TMEM lane quadrants)
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kMaxBN = 128;       // largest query group (MMA N)
// dynamic shared memory budget: alignment slack, A ring, resident queries,
// and (histogram pass) the group's histograms
constexpr size_t kDynBudget = 210 * 1024;

struct ScanShared {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
  int list;
  int pos;  // the list's place in the scan order
  int64_t dst[kMaxBN];
  float yn[kMaxBN];
  // two-pass modes, per query column: its row, histogram bounds, band edge
  // and k-th bin
  int q[kMaxBN];
  float lo[kMaxBN], scale[kMaxBN], thr[kMaxBN];
  int bstar[kMaxBN];
  int rbin[kMaxBN], fstar[kMaxBN];  // refined bin (-1: none) and the k-th's sub-bin
  float flo[kMaxBN], fscale[kMaxBN];
  int any;  // refinement pass: some column of this CTA is refined
};

template <int Mode>
__global__ void __launch_bounds__(kThreads, 1)
    k_scan_tc(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ Yp,
              const float* __restrict__ C, int dp, const float* __restrict__ XLcn,
              const int64_t* __restrict__ list_off, int L, int dpb, int BN,
              const int32_t* __restrict__ pair_q, const int64_t* __restrict__ pair_dst,
              const int64_t* __restrict__ bucket_off, const int64_t* __restrict__ tile_off,
              const int32_t* __restrict__ lorder, float* __restrict__ cand, const TwoPass tp,
              const float* __restrict__ XL, const int32_t* __restrict__ perm,
              uint32_t* __restrict__ err) {
  __shared__ ScanShared sh;
  extern __shared__ uint8_t dyn_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t t = blockIdx.x;
  if (t >= tile_off[L]) return;

  // 1024-byte aligned operand area: A ring, then the resident B block, then
  // (histogram pass) one histogram per query column
  const uint32_t raw = tc::smem_u32(dyn_raw);
  uint8_t* base = dyn_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t* A = base;
  uint8_t* B = base + kStages * kStageBytes;
  const int KB = dpb / kBK;
  uint32_t* hs = reinterpret_cast<uint32_t*>(B + (size_t)KB * BN * 128);

  if (tid == 0) {
    int lo = 0, hi = L - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    sh.pos = lo;
    sh.list = lorder[lo];
    sh.abort = 0;
    sh.any = 0;
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

  // stage the queries centred on this list's centroid, y~ = y - c_l, in BF16:
  // row r of block kb at B + kb*BN*128 + r*128, 16-byte chunk c stored at
  // chunk position c ^ (r & 7) (the 128-byte swizzle)
  const float* cl = C + (int64_t)l * dp;
  const int chunks = nN * KB * 8;
  for (int i = tid; i < chunks; i += kThreads) {
    const int r = i / (KB * 8);
    const int rem = i - r * (KB * 8);
    const int kb = rem >> 3, c = rem & 7;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (r < npairs) {
      const float* yq = Yp + (int64_t)pair_q[pb + r] * dp;
      const int j0 = kb * kBK + c * 8;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + 2 * u;
        const float f0 = j < dp ? yq[j] - cl[j] : 0.f;
        const float f1 = j + 1 < dp ? yq[j + 1] - cl[j + 1] : 0.f;
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(f0, f1);
        w[u] = *reinterpret_cast<const uint32_t*>(&h2);
      }
    }
    *reinterpret_cast<uint4*>(B + (size_t)kb * BN * 128 + r * 128 + ((c ^ (r & 7)) << 4)) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
  if (Mode == kScanHist || Mode == kScanRefine)
    for (int i = tid; i < npairs * kHistBins; i += kThreads) hs[i] = 0u;
  // |y~|^2 in FP32 and each column's destination or selection state, one
  // warp per query row
  for (int r = warp; r < nN; r += kThreads / 32) {
    float s = 0.f;
    if (r < npairs) {
      const float* yq = Yp + (int64_t)pair_q[pb + r] * dp;
      for (int j = lane; j < dp; j += 32) {
        const float v = yq[j] - cl[j];
        s = fmaf(v, v, s);
      }
      s = warp_sum(s);
    }
    if (lane == 0) {
      sh.yn[r] = s;
      if (Mode == kScanCand) {
        sh.dst[r] = r < npairs ? pair_dst[pb + r] : -1;
      } else if (r < npairs) {
        const int q = pair_q[pb + r];
        sh.q[r] = q;
        sh.lo[r] = tp.hlo[q];
        sh.scale[r] = tp.hscale[q];
        if (Mode == kScanEmit || Mode == kScanRefine) {
          const int rb = tp.rbin[q];
          sh.rbin[r] = rb;
          if (rb >= 0) {
            sh.flo[r] = tp.flo[q];
            sh.fscale[r] = tp.fscale[q];
            if (Mode == kScanRefine) sh.any = 1;
          }
        }
        if (Mode == kScanEmit) {
          sh.thr[r] = tp.thr[q];
          sh.bstar[r] = tp.bstar[q];
          sh.fstar[r] = tp.fstar[q];
        }
      }
    }
  }
  if (Mode == kScanRefine) {
    __syncthreads();
    if (!sh.any) return;  // no refined query among this CTA's: nothing to count
  }
  tc::fence_proxy_async_smem();
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(2 * BN)) ncols <<= 1;
  if (warp == 1) tc::tmem_alloc(&sh.tmem_base, ncols);
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = sh.tmem_base;
  volatile int* abort = &sh.abort;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int it = 0;  // loads issued so far
      for (int tt = 0; tt < ntiles && !*abort; ++tt) {
        for (int kb = 0; kb < KB; ++kb) {
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!tc::mbar_wait(&sh.empty[s], ph ^ 1u, abort)) break;
          tc::mbar_arrive_expect_tx(&sh.full[s], kStageBytes);
          tc::tma_load_2d(A + s * kStageBytes, &tmap, kb * kBK, (int)(xb + (int64_t)tt * kBM),
                          &sh.full[s]);
          ++it;
        }
      }
      if (*abort) {
        // let the last (at most kStages) loads land before the CTA's shared
        // memory goes away; every earlier load was consumed by the MMA warp
        volatile int no_abort = 0;
        for (int j = it > kStages ? it - kStages : 0; j < it; ++j)
          tc::mbar_wait(&sh.full[j % kStages], (uint32_t)(j / kStages) & 1u, &no_abort);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = tc::make_idesc(kBM, nN, 1u);
      int it = 0;
      bool ok = true;
      for (int tt = 0; tt < ntiles && ok; ++tt) {
        const int b = tt & 1;
        const uint32_t tph = (uint32_t)(tt >> 1) & 1u;
        if (!tc::mbar_wait(&sh.tempty[b], tph ^ 1u, abort)) break;
        tc::tc_fence_after();
        const uint32_t d_tmem = tmem + (uint32_t)(b * BN);
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
            tc::mma_f16(d_tmem, tc::desc_sw128(a0 + kk * 32), tc::desc_sw128(b0 + kk * 32),
                        idesc, (kb | kk) != 0 ? 1u : 0u);
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
    // column 16.
    const int lg = (warp & 3) * 32;
    const int cstart = ((warp - 2) >> 2) * 16;
    constexpr int cstep = 16 * (kEpiWarps / 4);
    const int row = lg + lane;
    const int64_t padlen = (len + 31) & ~(int64_t)31;
    const int dp4 = dp >> 2;
    const int lane8 = lane & 7, grp = lane >> 3;
    const int cap_b = kSelectCap - tp.kA;
    for (int tt = 0; tt < ntiles; ++tt) {
      const int b = tt & 1;
      const uint32_t tph = (uint32_t)(tt >> 1) & 1u;
      int ok = 1;
      if (lane == 0) ok = tc::mbar_wait(&sh.tfull[b], tph, abort) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc::tc_fence_after();
      const int64_t pt = (int64_t)tt * kBM + row;
      const bool valid = pt < len, pad = !valid && pt < padlen;
      const float xn = valid ? XLcn[xb + pt] : 0.f;
      const uint32_t taddr = tmem + ((uint32_t)lg << 16) + (uint32_t)(b * BN);
      for (int c0 = cstart; c0 < npairs; c0 += cstep) {
        uint32_t v[16];
        tc::tmem_ld16(taddr + (uint32_t)c0, v);
        if (Mode == kScanCand) {
          // every candidate (and the +inf padding of its segment) to HBM,
          // coalesced: the warp's 32 points of one query in one 128-byte store
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = c0 + j;
            if ((valid || pad) && col < npairs)
              cand[sh.dst[col] + pt] =
                  valid ? fmaxf(xn + sh.yn[col] - 2.f * __uint_as_float(v[j]), 0.f)
                        : __int_as_float(0x7f800000);
          }
        } else if (Mode == kScanHist) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = c0 + j;
            if (valid && col < npairs) {
              const float a = fmaxf(xn + sh.yn[col] - 2.f * __uint_as_float(v[j]), 0.f);
              atomicAdd(hs + col * kHistBins + hist_bin(a, sh.lo[col], sh.scale[col]), 1u);
            }
          }
        } else if (Mode == kScanRefine) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = c0 + j;
            if (valid && col < npairs && sh.rbin[col] >= 0) {
              const float a = fmaxf(xn + sh.yn[col] - 2.f * __uint_as_float(v[j]), 0.f);
              if (hist_bin(a, sh.lo[col], sh.scale[col]) == sh.rbin[col])
                atomicAdd(hs + col * kHistBins + hist_bin(a, sh.flo[col], sh.fscale[col]), 1u);
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = c0 + j;
            if (col >= npairs) continue;  // the same for every lane of the warp
            const float a =
                valid ? fmaxf(xn + sh.yn[col] - 2.f * __uint_as_float(v[j]), 0.f) : 0.f;
            // region A: below the k-th bin, or (refined queries) inside it
            // below the k-th sub-bin
            const int cb = hist_bin(a, sh.lo[col], sh.scale[col]);
            const bool inA =
                valid && (cb < sh.bstar[col] ||
                          (cb == sh.rbin[col] &&
                           hist_bin(a, sh.flo[col], sh.fscale[col]) < sh.fstar[col]));
            const bool inB = valid && !inA && a <= sh.thr[col];
            const unsigned mA = __ballot_sync(0xffffffffu, inA);
            const unsigned mB = __ballot_sync(0xffffffffu, inB);
            unsigned m = mA | mB;
            if (m == 0u) continue;
            const int qrow = sh.q[col];
            int baseA = 0, baseB = 0;
            if (lane == 0) {
              if (mA) baseA = atomicAdd(tp.cntA + qrow, __popc(mA));
              if (mB) baseB = atomicAdd(tp.cntB + qrow, __popc(mB));
            }
            baseA = __shfl_sync(0xffffffffu, baseA, 0);
            baseB = __shfl_sync(0xffffffffu, baseB, 0);
            const float4* y4 = reinterpret_cast<const float4*>(Yp + (int64_t)qrow * dp);
            unsigned long long* kq = tp.keys + (int64_t)qrow * kSelectCap;
            while (m != 0u) {
              // up to four marked points at a time, eight lanes each: group g
              // takes the g-th lowest marked lane
              unsigned rest = m;
              for (int i = 0; i < grp; ++i) rest &= rest - 1u;
              const int bit = rest != 0u ? __ffs(rest) - 1 : -1;
#pragma unroll
              for (int i = 0; i < 4; ++i) m &= m - 1u;
              const int64_t prow = xb + (int64_t)tt * kBM + lg + (bit < 0 ? 0 : bit);
              float acc = 0.f;
              if (bit >= 0) {
                const float4* x4 = reinterpret_cast<const float4*>(XL + prow * dp);
                for (int c4 = lane8; c4 < dp4; c4 += 8) {
                  const float4 xv = x4[c4], yv = y4[c4];
                  const float t0 = xv.x - yv.x, t1 = xv.y - yv.y, t2 = xv.z - yv.z,
                              t3 = xv.w - yv.w;
                  acc = fmaf(t0, t0, acc);
                  acc = fmaf(t1, t1, acc);
                  acc = fmaf(t2, t2, acc);
                  acc = fmaf(t3, t3, acc);
                }
              }
              acc += __shfl_xor_sync(0xffffffffu, acc, 4);
              acc += __shfl_xor_sync(0xffffffffu, acc, 2);
              acc += __shfl_xor_sync(0xffffffffu, acc, 1);
              if (bit >= 0 && lane8 == 0) {
                const unsigned below = (1u << bit) - 1u;
                const unsigned long long key = pack_key(acc, perm[prow]);
                if ((mA >> bit) & 1u) {
                  const int slot = baseA + __popc(mA & below);
                  if (slot < tp.kA) kq[slot] = key;
                } else {
                  const int slot = baseB + __popc(mB & below);
                  if (slot < cap_b) kq[tp.kA + slot] = key;
                }
              }
            }
          }
        }
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
  if (Mode == kScanHist || Mode == kScanRefine) {
    // the group's histograms into the queries' global ones
    uint32_t* dst = Mode == kScanHist ? tp.hist : tp.hist2;
    for (int i = tid; i < npairs * kHistBins; i += kThreads) {
      const uint32_t c = hs[i];
      if (c != 0u)
        atomicAdd(dst + (int64_t)sh.q[i / kHistBins] * kHistBins + (i % kHistBins), c);
    }
  }
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, ncols);
  }
}

}  // namespace

size_t scan_tc_smem(int dpb, int BN, int mode) {
  size_t b = 1024 + (size_t)kStages * kStageBytes + (size_t)(dpb / kBK) * BN * 128;
  if (mode == kScanHist || mode == kScanRefine) b += (size_t)BN * kHistBins * sizeof(uint32_t);
  return b;
}

int scan_tc_bn(int dpb) {
  // the largest multiple of 16 (at most kMaxBN) whose histogram pass fits
  int bn = kMaxBN;
  while (bn > 16 && scan_tc_smem(dpb, bn, kScanHist) > kDynBudget) bn -= 16;
  return bn;
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

bool launch_scan_tc(int mode, const void* tmap, const float* Yp, const float* C, int dp,
                    const float* XLcn, const int64_t* list_off, int L, int dpb, int BN,
                    const ScanPlan& plan, float* cand, const TwoPass& tp, const float* XL,
                    const int32_t* perm, uint32_t* err, cudaStream_t s) {
  if (plan.max_tiles <= 0) return true;
  if (BN > kMaxBN || BN % 16 != 0) return false;
  const size_t smem = scan_tc_smem(dpb, BN, mode);
  const CUtensorMap& map = *reinterpret_cast<const CUtensorMap*>(tmap);
  const unsigned grid = (unsigned)plan.max_tiles;
#define DEANN_SCAN_LAUNCH(M)                                                                  \
  do {                                                                                        \
    if (!set_dynamic_smem(reinterpret_cast<const void*>(&k_scan_tc<M>), smem)) return false; \
    k_scan_tc<M><<<grid, kThreads, smem, s>>>(map, Yp, C, dp, XLcn, list_off, L, dpb, BN,     \
                                              plan.pair_q, plan.pair_dst, plan.bucket_off,    \
                                              plan.tile_off, plan.lorder, cand, tp, XL, perm, \
                                              err);                                           \
  } while (0)
  if (mode == kScanCand) DEANN_SCAN_LAUNCH(kScanCand);
  else if (mode == kScanHist) DEANN_SCAN_LAUNCH(kScanHist);
  else if (mode == kScanRefine) DEANN_SCAN_LAUNCH(kScanRefine);
  else DEANN_SCAN_LAUNCH(kScanEmit);
#undef DEANN_SCAN_LAUNCH
  return true;
}

}  // namespace deann
