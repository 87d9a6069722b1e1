// Candidate selection for the IVF search (paper Section 4: the inverted file
// scans the lists of the n_q nearest centroids and returns the k nearest
// points).
//
//  * query norms |y|^2;
//  * probe selection: the nprobe nearest centroids of each query (radix
//    select of a margin, FP32 rescoring, sort);
//  * the (query, probe) work plan that groups pairs by list for the
//    list-major scan, candidate segments aligned to 32 floats, and the order
//    in which queries are selected (grouped by nearest list);
//  * neighbour selection, one CTA per query, from the approximate distances
//    the scan wrote: t_k, the k-th smallest approximate distance, is
//    bracketed by a histogram; every candidate whose approximate distance is
//    within 2E of t_k is collected (E bounds the scan's error for this query:
//    the true k-th distance is at most t_k + E and every true top-k point has
//    an approximate distance at most t_k + 2E, so the set holds the exact top
//    k); those rows are rescored in FP32 difference form, and only the
//    candidates inside the FP32 error band of the k-th are re-ranked with
//    compensated arithmetic.  Returned: the k neighbours (sorted by (distance,
//    id), or as a set for the query path) and the exact neighbour
//    contribution s1 = sum_{X_1} K_h(x, y) (Algorithm 1).
//
// More than the kept-candidate capacity in the band cannot all be kept: the
// smallest that fit are rescored and the query is counted as uncertified in
// the device error word (kde_stats).
#include "common.cuh"

namespace deann {

namespace {

constexpr int kNT = 256;
constexpr int kNW = kNT / 32;

__global__ void k_query_norms(const float* __restrict__ Y, int64_t nq, int dp,
                              float* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  float s = 0.f;
  for (int j = lane; j < dp; j += 32) {
    const float v = Y[q * dp + j];
    s = fmaf(v, v, s);
  }
  s = warp_sum(s);
  if (lane == 0) out[q] = s;
}

template <int Cap>
struct SelectSmemT {
  static constexpr int kCap = Cap;
  int hist[256];
  int warp_a[kNW];
  int warp_b[kNW];
  int digit, before;
  int slot[Cap];
  unsigned long long key[Cap];
};
using SelectSmem = SelectSmemT<kSelectCap>;  // neighbour selection
// for k <= kSmallCapMaxK on the split scan's values: 3,072 candidates kept,
// small enough (with 48 registers a thread) for five blocks an SM instead of
// four
constexpr int kSmallCap = 3072;
constexpr int kSmallCapMaxK = 1536;
using SelectSmemSmall = SelectSmemT<kSmallCap>;
constexpr int kProbeCap = 512;               // probe selection: nprobe + margin <= 384
using ProbeSmem = SelectSmemT<kProbeCap>;

// Selects the K smallest of vals[0..cnt) (1 <= K <= min(cnt, the capacity)):
// sm.slot[0..K) receives their indices (those strictly below the K-th key in
// index order, then the lowest-index ties).  Returns the K-th key.
template <class SM>
__device__ uint32_t block_select(const float* __restrict__ vals, int64_t cnt, int K, SM& sm,
                                 bool collect = true) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t prefix = 0, pmask = 0;
  int want = K;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int i = tid; i < 256; i += kNT) sm.hist[i] = 0;
    __syncthreads();
    // four independent loads per thread per iteration keep more reads in flight
    for (int64_t i0 = tid; i0 < cnt; i0 += 4 * kNT) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + u * kNT;
        v[u] = i < cnt ? vals[i] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (i0 + u * kNT >= cnt) continue;
        const uint32_t key = dist_key(v[u]);
        if ((key & pmask) == prefix) atomicAdd(&sm.hist[(key >> shift) & 255], 1);
      }
    }
    __syncthreads();
    if (warp == 0) {
      int c[8], s = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        c[b] = sm.hist[lane * 8 + b];
        s += c[b];
      }
      int incl = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int excl = incl - s;
      if (excl < want && want <= incl) {
        int run = excl;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          if (run < want && want <= run + c[b]) {
            sm.digit = lane * 8 + b;
            sm.before = run;
          }
          run += c[b];
        }
      }
    }
    __syncthreads();
    prefix |= (uint32_t)sm.digit << shift;
    pmask |= 255u << shift;
    want -= sm.before;
    __syncthreads();
  }
  if (!collect) return prefix;
  // collect: keys < thr in index order, then the first `want` keys == thr
  const uint32_t thr = prefix;
  const int n_lt = K - want;
  int base_lt = 0, base_eq = 0;
  for (int64_t b0 = 0; b0 < cnt; b0 += kNT) {
    const int64_t i = b0 + tid;
    uint32_t key = 0xffffffffu;
    if (i < cnt) key = dist_key(vals[i]);
    const bool lt = i < cnt && key < thr;
    const bool eq = i < cnt && key == thr;
    const unsigned mlt = __ballot_sync(0xffffffffu, lt);
    const unsigned meq = __ballot_sync(0xffffffffu, eq);
    if (lane == 0) {
      sm.warp_a[warp] = __popc(mlt);
      sm.warp_b[warp] = __popc(meq);
    }
    __syncthreads();
    int off_lt = base_lt, off_eq = base_eq, tot_lt = 0, tot_eq = 0;
#pragma unroll
    for (int w = 0; w < kNW; ++w) {
      if (w < warp) {
        off_lt += sm.warp_a[w];
        off_eq += sm.warp_b[w];
      }
      tot_lt += sm.warp_a[w];
      tot_eq += sm.warp_b[w];
    }
    const unsigned below = (1u << lane) - 1u;
    if (lt) {
      const int r = off_lt + __popc(mlt & below);
      if (r < n_lt) sm.slot[r] = (int)i;
    }
    if (eq) {
      const int r = off_eq + __popc(meq & below);
      if (r < want) sm.slot[n_lt + r] = (int)i;
    }
    base_lt += tot_lt;
    base_eq += tot_eq;
    __syncthreads();
  }
  return thr;
}

// A query's candidate values start on a 16-byte boundary (segments are
// padded to multiples of 4 floats); entries at cnt and beyond are padding.
// Calls f(i, v) for this thread's candidates, kU float4 loads in flight.
constexpr int kU = 4;
template <typename F>
__device__ __forceinline__ void for_each_cand(const float* __restrict__ vals, int64_t cnt, F f) {
  const float4* v4 = reinterpret_cast<const float4*>(vals);
  const int64_t n4 = (cnt + 3) >> 2;
  for (int64_t b = threadIdx.x; b < n4; b += (int64_t)kU * kNT) {
    float4 v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i4 = b + (int64_t)u * kNT;
      v[u] = i4 < n4 ? v4[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = (b + (int64_t)u * kNT) * 4;
      if (i + 0 < cnt) f(i + 0, v[u].x);
      if (i + 1 < cnt) f(i + 1, v[u].y);
      if (i + 2 < cnt) f(i + 2, v[u].z);
      if (i + 3 < cnt) f(i + 3, v[u].w);
    }
  }
}

constexpr uint32_t kInfKey = 0x7f800000u;  // dist_key(+inf)

// Collects the indices of all finite keys <= thr into sm.slot[0..cap) in a fixed
// order (rounds of kU * kNT float4s; within a round, thread by thread).
// Returns the total count, which may exceed cap (then the slots hold only
// the first cap).
template <class SM>
__device__ int block_collect_le(const float* __restrict__ vals, int64_t cnt, uint32_t thr, int cap,
                                SM& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float4* v4 = reinterpret_cast<const float4*>(vals);
  const int64_t n4 = (cnt + 3) >> 2;
  int base = 0;
  for (int64_t r0 = 0; r0 < n4; r0 += (int64_t)kU * kNT) {
    float4 v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i4 = r0 + (int64_t)u * kNT + tid;
      v[u] = i4 < n4 ? v4[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    unsigned take = 0u;  // bit 4u + c: component c of load u
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = (r0 + (int64_t)u * kNT + tid) * 4;
      const float c4[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint32_t key = dist_key(c4[c]);
        // +inf marks the padding of the candidate segments: never a candidate
        if (i + c < cnt && key <= thr && key < kInfKey) take |= 1u << (4 * u + c);
      }
    }
    const int mine = __popc(take);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) sm.warp_a[warp] = incl;
    __syncthreads();
    int before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kNW; ++w) {
      if (w < warp) before += sm.warp_a[w];
      tot += sm.warp_a[w];
    }
    int r = base + before + incl - mine;
    while (take != 0u) {
      const int bit = __ffs(take) - 1;
      take &= take - 1u;
      if (r < cap) sm.slot[r] = (int)((r0 + (int64_t)(bit >> 2) * kNT + tid) * 4 + (bit & 3));
      ++r;
    }
    base += tot;
    __syncthreads();
  }
  return base;
}

// Brackets the k-th smallest of the nonnegative vals[0..cnt) (1 <= k <= cnt)
// with two passes: the minimum and maximum, then a 4096-bin histogram on the
// linear scale between them.  Returns lo <= (k-th smallest) <= hi, the bounds
// of the bin that holds it, widened by a few units of rounding.
template <class SM>
__device__ void block_kth_bracket(const float* __restrict__ vals, int64_t cnt, int k,
                                  SM& sm, float& lo_out, float& hi_out,
                                  float lo_hint, float hi_hint) {
  constexpr int kBins = 4096;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ float s_mn[kNW], s_mx[kNW];
  __shared__ int s_scan[kNW];
  __shared__ float s_lo, s_hi;
  int* hist = reinterpret_cast<int*>(sm.key);  // 16 KiB, free until rescoring
  // the histogram spans [mn, mx]: the caller's bounds on every value when
  // it has them (0 <= lo_hint <= hi_hint), else a min/max pass
  const bool hinted = lo_hint >= 0.f && hi_hint >= lo_hint;
  float mn = hinted ? lo_hint : __int_as_float(0x7f800000), mx = hinted ? hi_hint : 0.f;
  if (!hinted)
    for_each_cand(vals, cnt, [&](int64_t, float v) {
      if (v < __int_as_float(0x7f800000)) {  // the +inf padding is no candidate
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
      }
    });
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    s_mn[warp] = mn;
    s_mx[warp] = mx;
  }
  for (int b = tid; b < kBins; b += kNT) hist[b] = 0;
  __syncthreads();
  mn = s_mn[0];
  mx = s_mx[0];
  for (int w = 1; w < kNW; ++w) {
    mn = fminf(mn, s_mn[w]);
    mx = fmaxf(mx, s_mx[w]);
  }
  const float scale = mx > mn ? (float)kBins / (mx - mn) : 0.f;
  for_each_cand(vals, cnt, [&](int64_t, float v) {
    const int bin = v >= mx ? kBins - 1 : min(kBins - 1, max(0, (int)((v - mn) * scale)));
    atomicAdd(&hist[bin], 1);
  });
  __syncthreads();
  // thread t owns bins [16 t, 16 t + 16)
  constexpr int kPer = kBins / kNT;
  int c[kPer], s = 0;
#pragma unroll
  for (int b = 0; b < kPer; ++b) {
    c[b] = hist[tid * kPer + b];
    s += c[b];
  }
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_scan[warp] = incl;
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += s_scan[w];
  incl += before;
  const int excl = incl - s;
  if (excl < k && k <= incl) {
    int run = excl, bin = tid * kPer;
#pragma unroll
    for (int b = 0; b < kPer; ++b) {
      if (run < k && k <= run + c[b]) bin = tid * kPer + b;
      run += c[b];
    }
    if (scale > 0.f) {
      const float lo = mn + (float)bin / scale, hi = mn + (float)(bin + 1) / scale;
      s_lo = fmaxf(0.f, lo - fabsf(lo) * 1e-6f - 1e-30f);
      s_hi = hi + fabsf(hi) * 1e-6f + 1e-30f;
      // end bins also hold any value beyond the bounds: open them
      if (bin == 0) s_lo = 0.f;
      if (bin == kBins - 1) s_hi = __int_as_float(0x7f800000);
    } else if (hinted) {
      s_lo = 0.f;
      s_hi = __int_as_float(0x7f800000);
    } else {
      s_lo = mn;
      s_hi = mx;
    }
  }
  __syncthreads();
  lo_out = s_lo;
  hi_out = s_hi;
}

// k-th smallest distance key (upper 32 bits) among sm.key[0..K), 1 <= k <= K,
// by four 8-bit radix passes over shared memory.
template <class SM>
__device__ uint32_t smem_kth_dist(SM& sm, int K, int k) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t prefix = 0, pmask = 0;
  int want = k;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int i = tid; i < 256; i += kNT) sm.hist[i] = 0;
    __syncthreads();
    for (int j = tid; j < K; j += kNT) {
      const uint32_t key = (uint32_t)(sm.key[j] >> 32);
      if ((key & pmask) == prefix) atomicAdd(&sm.hist[(key >> shift) & 255], 1);
    }
    __syncthreads();
    if (warp == 0) {
      int c[8], s = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        c[b] = sm.hist[lane * 8 + b];
        s += c[b];
      }
      int incl = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int excl = incl - s;
      if (excl < want && want <= incl) {
        int run = excl;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          if (run < want && want <= run + c[b]) {
            sm.digit = lane * 8 + b;
            sm.before = run;
          }
          run += c[b];
        }
      }
    }
    __syncthreads();
    prefix |= (uint32_t)sm.digit << shift;
    pmask |= 255u << shift;
    want -= sm.before;
    __syncthreads();
  }
  return prefix;
}

// Bitonic sort of sm.key[0..cnt) ascending (cnt padded to a power of two
// with all-ones keys).
template <class SM>
__device__ void block_sort_keys(SM& sm, int cnt) {
  int P2 = 1;
  while (P2 < cnt) P2 <<= 1;
  for (int i = cnt + threadIdx.x; i < P2; i += kNT) sm.key[i] = ~0ull;
  __syncthreads();
  for (int size = 2; size <= P2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P2 / 2; i += kNT) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const unsigned long long a = sm.key[lo], b = sm.key[hi];
        if ((a > b) == up) {
          sm.key[lo] = b;
          sm.key[hi] = a;
        }
      }
      __syncthreads();
    }
  }
}


// --------------------------------------------------------------------------
// Probe selection: nprobe nearest centroids (ties to the lower id).
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kNT) k_select_probes(const float* __restrict__ D, int64_t nq,
                                                       int L, const float* __restrict__ Y, int d,
                                                       int dp, const float* __restrict__ C,
                                                       int nprobe, int kprime,
                                                       int32_t* __restrict__ probes,
                                                       float* __restrict__ probe_d2,
                                                       const int64_t* __restrict__ active,
                                                       int64_t q0) {
  extern __shared__ uint4 sel_dyn4[];  // SelectSmem, in dynamic shared memory (> 48 KB)
  ProbeSmem& sm = *reinterpret_cast<ProbeSmem*>(sel_dyn4);
  const int64_t q = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (active != nullptr && q0 + q >= *active) {  // an inactive row probes no list
    for (int j = threadIdx.x; j < nprobe; j += kNT) {
      probes[q * nprobe + j] = -1;
      probe_d2[q * nprobe + j] = __int_as_float(0x7f800000);
    }
    return;
  }
  const float* vals = D + q * L;
  const int K = min(kprime, L);
  if (K < L) {
    block_select(vals, L, K, sm);
  } else {
    for (int i = threadIdx.x; i < L; i += kNT) sm.slot[i] = i;
    __syncthreads();
  }
  const float* y = Y + q * dp;
  for (int j = warp; j < K; j += kNW) {
    const int c = sm.slot[j];
    const float d2 = precise_sq_dist<32>(C + (int64_t)c * dp, y, d, lane);
    if (lane == 0) sm.key[j] = pack_key(d2, c);
  }
  __syncthreads();
  block_sort_keys(sm, K);
  for (int j = threadIdx.x; j < nprobe; j += kNT) {
    probes[q * nprobe + j] = j < K ? (int32_t)(sm.key[j] & 0xffffffffu) : -1;
    probe_d2[q * nprobe + j] =
        j < K ? __uint_as_float((uint32_t)(sm.key[j] >> 32)) : __int_as_float(0x7f800000);
  }
}

// The same selection with one warp per query, for kprime <= 32 (the usual
// nprobe).  Pairs (approximate key, id) are totally ordered; each lane keeps
// the four smallest of its own pairs in registers, and each of kprime rounds
// takes the smallest lane head over the warp, so the pairs come out in order:
// the set the block version selects.  A lane whose four are used up scans its
// pairs again for the next four above the last it gave.  Lane j keeps the
// j-th with its compensated FP32 distance, and a rank count orders them by
// (distance, id).
__global__ void __launch_bounds__(kNT) k_select_probes_warp(
    const float* __restrict__ D, int64_t nq, int L, const float* __restrict__ Y, int d, int dp,
    const float* __restrict__ C, int nprobe, int kprime, int32_t* __restrict__ probes,
    float* __restrict__ probe_d2, const int64_t* __restrict__ active, int64_t q0) {
  using u64 = unsigned long long;
  const int lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * kNW + (threadIdx.x >> 5);
  if (q >= nq) return;
  int K = min(kprime, L);
  if (active != nullptr && q0 + q >= *active) K = 0;  // an inactive row probes no list
  const float* vals = D + q * L;
  const float* y = Y + q * dp;
  constexpr u64 kNone = ~0ull;
  u64 b0 = kNone, b1 = kNone, b2 = kNone, b3 = kNone;
  // the four smallest of this lane's pairs above `floor` (pairs are stored + 1,
  // so floor 0 is below all of them)
  auto fill = [&](u64 floor) {
    b0 = b1 = b2 = b3 = kNone;
    for (int i = lane; i < L; i += 32) {
      const u64 c = (((u64)dist_key(vals[i]) << 32) | (unsigned)i) + 1ull;
      if (c > floor && c < b3) {
        const u64 n3 = c < b2 ? b2 : c;
        const u64 n2 = c < b2 ? (c < b1 ? b1 : c) : b2;
        const u64 n1 = c < b1 ? (c < b0 ? b0 : c) : b1;
        b0 = c < b0 ? c : b0;
        b1 = n1;
        b2 = n2;
        b3 = n3;
      }
    }
  };
  if (K > 0) fill(0ull);
  // the K smallest approximate distances: lane r keeps the r-th one's list
  int cand = 0;
  for (int r = 0; r < K; ++r) {
    u64 best = b0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const u64 t = __shfl_xor_sync(0xffffffffu, best, o);
      best = t < best ? t : best;
    }
    if (b0 == best) {  // this lane's head (pairs are distinct): pop it
      b0 = b1;
      b1 = b2;
      b2 = b3;
      b3 = kNone;
      if (b0 == kNone) fill(best);
    }
    if (lane == r) cand = (int)((best - 1ull) & 0xffffffffull);
  }
  // their compensated distances, 8 lanes a list and four lists at once (the
  // rows' loads in flight together); lane r receives its own list's
  u64 mine = kNone;
  const int grp = lane >> 3, lig = lane & 7;
  for (int r0 = 0; r0 < K; r0 += 4) {
    const int c = __shfl_sync(0xffffffffu, cand, min(r0 + grp, 31));
    const float d2 = precise_sq_dist<8>(C + (int64_t)c * dp, y, d, lig);
    const float d2r = __shfl_sync(0xffffffffu, d2, ((lane - r0) & 3) * 8);
    if (lane >= r0 && lane < r0 + 4 && lane < K) mine = pack_key(d2r, cand);
  }
  // rank of lane j's key among the K keys (all distinct: they carry the id)
  int rank = 0;
  for (int j = 0; j < K; ++j) {
    const unsigned long long t = __shfl_sync(0xffffffffu, mine, j);
    rank += t < mine ? 1 : 0;
  }
  if (lane < K && rank < nprobe) {
    probes[q * nprobe + rank] = (int32_t)(mine & 0xffffffffu);
    probe_d2[q * nprobe + rank] = __uint_as_float((uint32_t)(mine >> 32));
  }
  for (int j = K + lane; j < nprobe; j += 32) {
    probes[q * nprobe + j] = -1;
    probe_d2[q * nprobe + j] = __int_as_float(0x7f800000);
  }
}

// --------------------------------------------------------------------------
// Work plan of the list-major scan.
// --------------------------------------------------------------------------
// Candidate segments: query q's values for probe p start at seg_off[q P + p]
// within its region, each segment padded to a multiple of 32 floats (whole
// 128-byte lines; the scans fill the padding with +inf).  q_count holds the
// padded total, q_real the candidates.
__global__ void k_plan_segments(const int32_t* __restrict__ probes, int64_t nq, int P,
                                const int64_t* __restrict__ list_off,
                                int64_t* __restrict__ q_count, int64_t* __restrict__ q_real,
                                int64_t* __restrict__ seg_off, int64_t* __restrict__ list_cnt) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  int64_t run = 0, real = 0;
  for (int p = 0; p < P; ++p) {
    const int l = probes[q * P + p];
    seg_off[q * P + p] = run;
    if (l >= 0) {
      const int64_t len = list_off[l + 1] - list_off[l];
      run += (len + 31) & ~(int64_t)31;
      real += len;
      atomicAdd(reinterpret_cast<unsigned long long*>(list_cnt + l), 1ull);
    }
  }
  q_count[q] = run;
  q_real[q] = real;
}

__global__ void k_plan_fill(const int32_t* __restrict__ probes, int64_t nq, int P,
                            const int64_t* __restrict__ q_off,
                            const int64_t* __restrict__ seg_off,
                            const int64_t* __restrict__ bucket_off,
                            int64_t* __restrict__ bucket_fill, int32_t* __restrict__ pair_q,
                            int64_t* __restrict__ pair_dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * P) return;
  const int64_t q = i / P;
  const int l = probes[i];
  if (l < 0) return;
  const int64_t slot =
      bucket_off[l] +
      (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(bucket_fill + l), 1ull);
  pair_q[slot] = (int32_t)q;
  pair_dst[slot] = q_off[q] + seg_off[i];
}

// Selection order: queries grouped by their nearest probed list, so that the
// queries that rescore rows of the same list run together and share them in
// L2.  Only the schedule changes; each query's result does not depend on it.
__global__ void k_order_count(const int32_t* __restrict__ probes, int64_t nq, int P,
                              int64_t* __restrict__ cnt) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int l = max(0, probes[q * P]);
  atomicAdd(reinterpret_cast<unsigned long long*>(cnt + l), 1ull);
}

__global__ void k_order_fill(const int32_t* __restrict__ probes, int64_t nq, int P,
                             const int64_t* __restrict__ off, int64_t* __restrict__ fill,
                             int32_t* __restrict__ order) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int l = max(0, probes[q * P]);
  const int64_t slot =
      off[l] + (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(fill + l), 1ull);
  order[slot] = (int32_t)q;
}

// tile_cnt in scan order: entry i counts the query tiles of list lorder[i]
__global__ void k_plan_tiles(const int64_t* __restrict__ list_cnt, int L, int qtile,
                             const int32_t* __restrict__ lorder,
                             int64_t* __restrict__ tile_cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L) tile_cnt[i] = (list_cnt[lorder[i]] + qtile - 1) / qtile;
}

// Single-block exclusive scan; out has count + 1 entries (the last = total).
// Each input is first rounded up to a multiple of `align`.
__global__ void __launch_bounds__(1024) k_exclusive_scan(const int64_t* __restrict__ in,
                                                         int64_t count,
                                                         int64_t* __restrict__ out,
                                                         int64_t align) {
  __shared__ int64_t part[1024];
  const int tid = threadIdx.x;
  const int64_t per = (count + 1023) / 1024;
  const int64_t b = tid * per, e = min(count, b + per);
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += (in[i] + align - 1) / align * align;
  part[tid] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int64_t t = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += t;
    __syncthreads();
  }
  int64_t run = part[tid] - s;
  for (int64_t i = b; i < e; ++i) {
    const int64_t v = (in[i] + align - 1) / align * align;
    out[i] = run;
    run += v;
  }
  if (tid == 1023) out[count] = part[1023];
}

// Ranks the K keys in sm.key (distance key << 32 | id; ~0 for an empty
// slot) of query q and writes its outputs: the k nearest (as a set with s1 on
// the query path, else sorted with their distances), k' and s1.  Only
// candidates inside the error band of the k-th distance are re-ranked with
// compensated distances.  Called by the whole block after a barrier.
// band_abs widens the re-ranked band to the keys' own error bound when they
// come unrescored from the split scan (0 for FP32-rescored keys).  tk_lo >= 0
// is a lower bound on the k-th smallest distance that the keys' own values
// were bracketed with (then the k-th is found among the keys at or above it),
// else -1.  kmin is the smallest key when the caller has it, else ~0.
template <class SM>
__device__ void rank_keys(const SelectArgs& a, SM& sm, int K, int64_t q,
                          const float* __restrict__ y, float band_abs, float tk_lo,
                          unsigned long long kmin) {
  __shared__ float s_red[kNW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (a.ids_only && a.kern != KDE_KERN_LAPLACIAN) {
    // The query path needs the set and s1, not the order: find the k-th
    // smallest distance T, take every candidate clearly below it, and rank
    // only those within the error band of T by compensated distance.  With
    // K <= k every candidate is a neighbour.
    const int k = a.k;
    unsigned long long* amb = reinterpret_cast<unsigned long long*>(sm.slot);  // 1024 keys
    __shared__ int s_cnt[3];  // keys below tk_lo, keys at or above it, ambiguous keys
    __shared__ uint32_t s_T;
    __shared__ int s_ws[kNW];
    if (tid == 0) {
      s_cnt[0] = 0;
      s_cnt[1] = 0;
      s_cnt[2] = 0;
      s_T = kInfKey;
    }
    if (kmin == ~0ull) {
      unsigned long long mn = ~0ull;
      for (int j = tid; j < K; j += kNT) mn = min(mn, sm.key[j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      __shared__ unsigned long long s_mn[kNW];
      if (lane == 0) s_mn[warp] = mn;
      __syncthreads();
      kmin = s_mn[0];
      for (int w = 1; w < kNW; ++w) kmin = min(kmin, s_mn[w]);
    }
    __syncthreads();
    float T = __int_as_float(0x7f800000);
    if (K > k) {
      bool found = false;
      if (tk_lo >= 0.f) {
        // Every key below tk_lo is among the k nearest; the k-th is the
        // (k - below)-th smallest of the rest, a short list (the bracketing
        // bin and the band above it) ranked by comparing all its pairs.
        const uint32_t lob = dist_key(tk_lo);
        int below = 0;
        for (int j = tid; j < K; j += kNT) {
          const unsigned long long key = sm.key[j];
          if ((uint32_t)(key >> 32) < lob) {
            ++below;
          } else {
            const int r = atomicAdd(&s_cnt[1], 1);
            if (r < 1024) amb[r] = key;
          }
        }
        below = __reduce_add_sync(0xffffffffu, below);
        if (lane == 0) atomicAdd(&s_cnt[0], below);
        __syncthreads();
        const int M = s_cnt[1], want = k - s_cnt[0];
        if (M <= 1024 && want >= 1 && want <= M) {
          for (int t = tid; t < M; t += kNT) {
            const unsigned long long v = amb[t];
            int r = 0;
            for (int i = 0; i < M; ++i) r += amb[i] < v ? 1 : 0;
            if (r == want - 1) s_T = (uint32_t)(v >> 32);
          }
          found = true;
        }
        __syncthreads();
      }
      T = found ? __uint_as_float(s_T) : __uint_as_float(smem_kth_dist(sm, K, k));
    }
    uint32_t lo_key = kInfKey, hi_key = 0u;  // K <= k: every key is a neighbour
    if (K > k) {
      const float bw =
          fmaxf(4.f * (float)((a.d + 7) / 8 + 8) * (1.0f / 16777216.0f) * T, band_abs);
      lo_key = T - bw > 0.f ? dist_key(T - bw) : 0u;
      hi_key = dist_key(T + bw);
    }
    const float inv = kernel_inv(a.kern, a.h);
    // s1 is summed in 64-bit fixed point with its unit 2^-52 of the largest
    // term (the nearest candidate's kernel value), so that the sum does not
    // depend on the order in which the keys arrived: integer addition is
    // associative.  Each term is truncated by less than 2^-51 of the largest.
    int ex = 0;
    if (kmin != ~0ull)
      frexpf(kernel_from_dist(a.kern, __uint_as_float((uint32_t)(kmin >> 32)), inv), &ex);
    const int fx_shift = 52 - ex;  // every term is below 2^ex: its fixed value below 2^52
    unsigned long long part = 0ull;
    auto add_term = [&](uint32_t dk) {
      part += (unsigned long long)ldexpf(kernel_from_dist(a.kern, __uint_as_float(dk), inv),
                                         fx_shift);
    };
    // each thread takes a contiguous run of keys: the certain neighbours are
    // written in key order after one block scan of the runs' counts; the
    // ambiguous ones are gathered (any order: they are ranked below) and
    // their rows requested into L2 for the compensated distances
    const int run = (K + kNT - 1) / kNT;
    const int j_beg = min(K, tid * run), j_end = min(K, j_beg + run);
    const int lines = (a.dp * 4 + 127) >> 7;
    int mine = 0;
    for (int j = j_beg; j < j_end; ++j) {
      const unsigned long long key = sm.key[j];
      const uint32_t dk = (uint32_t)(key >> 32);
      if (dk < lo_key) {
        ++mine;
      } else if (dk <= hi_key) {
        const int r = atomicAdd(&s_cnt[2], 1);
        if (r < 1024) amb[r] = key;
        const int64_t id = (int64_t)(key & 0xffffffffu);
        if (id < a.n) {
          const char* row = reinterpret_cast<const char*>(a.X + id * a.dp);
          for (int ln = 0; ln < lines; ++ln) prefetch_l2(row + ((size_t)ln << 7));
        }
      }
    }
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_ws[warp] = incl;
    __syncthreads();
    int before = 0, c_in = 0;
#pragma unroll
    for (int w = 0; w < kNW; ++w) {
      if (w < warp) before += s_ws[w];
      c_in += s_ws[w];
    }
    int o = before + incl - mine;
    for (int j = j_beg; j < j_end; ++j) {
      const unsigned long long key = sm.key[j];
      const uint32_t dk = (uint32_t)(key >> 32);
      if (dk < lo_key) {
        a.nbr[q * k + o++] = (int32_t)(key & 0xffffffffu);
        add_term(dk);
      }
    }
    const int n_amb = s_cnt[2];
    const int need = k - c_in;  // 1 <= need <= n_amb when K > k; K <= k: padding
    if (n_amb <= 1024) {
      // compensated distances for the ambiguous candidates, then their order
      const int grp = lane >> 3, lig = lane & 7;
      for (int j0 = warp * 4; j0 < n_amb; j0 += kNW * 4) {
        const int j = j0 + grp;
        const bool valid = j < n_amb;
        const int64_t id = valid ? (int64_t)(amb[j] & 0xffffffffu) : 0;
        const bool row = id < a.n;  // an empty slot's key carries id -1
        float d2 = precise_sq_dist<8>(a.X + (row ? id : 0) * a.dp, y, a.d, lig);
        if (!row) d2 = __int_as_float(0x7f800000);
        if (valid && lig == 0) amb[j] = pack_key(d2, (int)id);
      }
      __syncthreads();
      // rank of each (unique) key among the ambiguous ones; the need smallest
      // are the remaining neighbours
      for (int t = tid; t < n_amb; t += kNT) {
        const unsigned long long v = amb[t];
        int r = 0;
        for (int i = 0; i < n_amb; ++i) r += amb[i] < v ? 1 : 0;
        if (r < need) {
          a.nbr[q * k + c_in + r] = (int32_t)(v & 0xffffffffu);
          add_term((uint32_t)(v >> 32));
        }
      }
      for (int j = n_amb + tid; j < need; j += kNT) a.nbr[q * k + c_in + j] = -1;
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) part += __shfl_xor_sync(0xffffffffu, part, sh);
      __shared__ unsigned long long s_fx[kNW];
      if (lane == 0) s_fx[warp] = part;
      __syncthreads();
      if (tid == 0) {
        unsigned long long t = 0ull;
        for (int w = 0; w < kNW; ++w) t += s_fx[w];
        if (a.s1) a.s1[q] = (float)ldexp((double)t, -fx_shift);
      }
      return;
    }
    // a very wide ambiguous band (many equal distances): fall through to the
    // full sort below, which rewrites the whole output
    __syncthreads();
  }
  block_sort_keys(sm, K);
  const int kk = min(a.k, K);
  // Only candidates whose plain distance lies within the FP32 error band of
  // the k-th can be misordered across the k-th place: recompute those with the
  // compensated distance (relative error a few 2^-24) and re-sort that range.
  if (kk > 0 && kk < K) {
    __shared__ int s_lo, s_hi;
    // four times the plain distance's error bound (ceil(d/8) + 3 + 2 units)
    const float band_rel = 4.f * (float)((a.d + 7) / 8 + 8) * (1.0f / 16777216.0f);
    if (tid == 0) {
      const float dk = __uint_as_float((uint32_t)(sm.key[kk - 1] >> 32));
      const float band = fmaxf(band_rel * dk, band_abs);
      int lo = kk - 1, hi = kk;
      while (lo > 0 && __uint_as_float((uint32_t)(sm.key[lo - 1] >> 32)) >= dk - band) --lo;
      while (hi < K && __uint_as_float((uint32_t)(sm.key[hi] >> 32)) <= dk + band) ++hi;
      s_lo = lo;
      s_hi = hi;
    }
    __syncthreads();
    const int lo = s_lo, hi = s_hi;
    if (hi - lo > 1) {
      const int grp = lane >> 3, lig = lane & 7;
      for (int j0 = lo + warp * 4; j0 < hi; j0 += kNW * 4) {
        const int j = j0 + grp;
        const bool valid = j < hi;
        const int64_t id = valid ? (int64_t)(sm.key[j] & 0xffffffffu) : 0;
        const bool row = id < a.n;  // an empty slot's key carries id -1
        float d2 = precise_sq_dist<8>(a.X + (row ? id : 0) * a.dp, y, a.d, lig);
        if (!row) d2 = __int_as_float(0x7f800000);
        if (valid && lig == 0) sm.key[j] = pack_key(d2, (int)id);
      }
      __syncthreads();
      if (hi - lo <= 64) {
        if (tid == 0) {  // a short band (the usual case): insertion sort
          for (int i = lo + 1; i < hi; ++i) {
            const unsigned long long v = sm.key[i];
            int j = i - 1;
            while (j >= lo && sm.key[j] > v) {
              sm.key[j + 1] = sm.key[j];
              --j;
            }
            sm.key[j + 1] = v;
          }
        }
        __syncthreads();
      } else {
        block_sort_keys(sm, K);  // many near-equal distances: sort everything again
      }
    }
  }
  for (int j = tid; j < a.k; j += kNT) {
    if (j < kk) {
      a.nbr[q * a.k + j] = (int32_t)(sm.key[j] & 0xffffffffu);
      if (a.nd2) a.nd2[q * a.k + j] = __uint_as_float((uint32_t)(sm.key[j] >> 32));
    } else {
      a.nbr[q * a.k + j] = -1;
      if (a.nd2) a.nd2[q * a.k + j] = __int_as_float(0x7f800000);
    }
  }
  // exact neighbour contribution s1 and k'
  if (a.s1 != nullptr || a.kcount != nullptr) {
    const float inv = kernel_inv(a.kern, a.h);
    float part = 0.f;
    if (a.kern == KDE_KERN_LAPLACIAN) {
      // the IVF ranks by Euclidean distance; the Laplacian kernel needs L1
      for (int j = warp; j < kk; j += kNW) {
        const int64_t id = (int64_t)(sm.key[j] & 0xffffffffu);
        const bool row = id < a.n;  // an empty slot's key carries id -1
        const float l1 = precise_l1_dist<32>(a.X + (row ? id : 0) * a.dp, y, a.d, lane);
        if (lane == 0 && row) part += kernel_from_dist(a.kern, l1, inv);
      }
    } else {
      for (int j = tid; j < kk; j += kNT)
        part += kernel_from_dist(a.kern, __uint_as_float((uint32_t)(sm.key[j] >> 32)), inv);
    }
    part = warp_sum(part);
    if (lane == 0) s_red[warp] = part;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < kNW; ++w) t += s_red[w];
      if (a.s1) a.s1[q] = t;
      if (a.kcount) a.kcount[q] = kk;
    }
  }
}

// --------------------------------------------------------------------------
// Neighbour selection from the scan's candidate buffer.
// --------------------------------------------------------------------------
template <class SM>
__host__ __device__ constexpr size_t select_tables_offset() {
  return (sizeof(SM) + 15) & ~size_t(15);
}
template <class SM>
size_t select_smem_bytes(int P) {
  return select_tables_offset<SM>() + (size_t)(3 * P + 1) * sizeof(int64_t) +
         (size_t)P * sizeof(float);
}

template <class SM, int kMinBlocks>
__global__ void __launch_bounds__(kNT, kMinBlocks) k_select_neighbors(SelectArgs a) {
  // SM, then the per-probe tables sized by P, in dynamic shared memory
  // (> 48 KB; sized so that kMinBlocks blocks fit an SM)
  extern __shared__ uint4 sel_dyn4[];
  SM& sm = *reinterpret_cast<SM*>(sel_dyn4);
  constexpr int kCap = SM::kCap;
  int64_t* s_seg = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(sel_dyn4) +
                                              select_tables_offset<SM>());  // [P + 1]
  int64_t* s_lstart = s_seg + (a.P + 1);                              // [P]
  int64_t* s_llen = s_lstart + a.P;                                   // [P]
  float* s_dc = reinterpret_cast<float*>(s_llen + a.P);               // [P] |y - c_l|
  const int64_t q = a.order != nullptr ? (int64_t)a.order[blockIdx.x] : (int64_t)blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (a.active != nullptr && a.q0 + q >= *a.active) {  // inactive row: empty neighbour set
    for (int j = tid; j < a.k; j += kNT) {
      a.nbr[q * a.k + j] = -1;
      if (a.nd2) a.nd2[q * a.k + j] = __int_as_float(0x7f800000);
    }
    if (tid == 0) {
      if (a.s1) a.s1[q] = 0.f;
      if (a.kcount) a.kcount[q] = 0;
    }
    return;
  }
  const int64_t cnt = a.q_count[q];      // slots, with +inf in the padding
  const int64_t cnt_real = a.q_real[q];  // candidates
  const float* vals = a.cand + a.q_off[q];
  const float* y = a.Y + q * a.dp;
  // Error bound E of the scan's distances for this query: |approx - exact|
  // <= err_scale r^2 with r = |x| + |y| (|x| <= the dataset's largest norm),
  // or, for the centred scan, r = |x~| + |y~| <= list radius + |y - c_probe|.
  // Every candidate of list l is within rad_l of c_l, so its exact distance
  // lies in [(|y - c_l| - rad_l)^2, (|y - c_l| + rad_l)^2], and the scan's
  // value within E of it: bounds for the histogram of t_k.  Warp 0 takes the
  // probes a lane each (with the probe's candidate segment and list) and
  // reduces.
  __shared__ float s_E, s_hint_lo, s_hint_hi;
  if (warp == 0) {
    float lo = __int_as_float(0x7f800000), hi = 0.f;
    for (int p = lane; p < a.P; p += 32) {
      const int l = a.probes[q * a.P + p];
      s_seg[p] = a.seg_off[q * a.P + p];
      s_lstart[p] = l >= 0 ? a.list_off[l] : 0;
      s_llen[p] = l >= 0 ? a.list_off[l + 1] - a.list_off[l] : 0;
      s_dc[p] = 0.f;
      if (l < 0) continue;
      const float dc = sqrtf(a.probe_d2[q * a.P + p]), rl = a.rad[l];
      s_dc[p] = dc;
      lo = fminf(lo, fmaxf(0.f, dc - rl));
      hi = fmaxf(hi, dc + rl);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      s_seg[a.P] = cnt;
      // r = max over the probes of |y - c_l| + rad_l (0 with no valid probe)
      const float r = a.centered ? hi : a.xmax + sqrtf(a.Yn[q]);
      s_E = a.err_scale * r * r;
      s_hint_lo = hi >= lo ? fmaxf(0.f, lo * lo * (1.f - 1e-5f) - s_E) : -1.f;
      s_hint_hi = hi >= lo ? hi * hi * (1.f + 1e-5f) + s_E : -1.f;
    }
  }
  __syncthreads();
  // Candidates to rescore: every one whose approximate distance is within 2E
  // of the k-th smallest approximate distance t_k.  The true k-th distance is
  // at most t_k + E, and a point of the true top k has an approximate
  // distance at most (t_k + E) + E, so this set always contains the exact
  // top k.  Beyond kCap candidates the kCap smallest are kept and
  // the query is counted as uncertified.
  int K;
  float tk_lo = -1.f, tk_hi;  // t_k lies in [tk_lo, tk_hi]
  if (cnt_real <= (int64_t)a.k) {
    K = block_collect_le(vals, cnt, kInfKey, kCap, sm);  // every finite value
  } else {
    block_kth_bracket(vals, cnt, a.k, sm, tk_lo, tk_hi, s_hint_lo, s_hint_hi);
    const uint32_t thr = dist_key(tk_hi + 2.f * s_E);
    K = block_collect_le(vals, cnt, thr, kCap, sm);
    if (K > kCap) {
      block_select(vals, cnt, kCap, sm);
      K = kCap;
      if (tid == 0) {
        atomicOr(a.err, KDE_ERRBIT_MARGIN);
        atomicAdd(a.err + 1, 1u);
      }
    }
  }
  // rescore in plain FP32 difference form: a warp takes 8 rows at once, each
  // lane one 16-byte piece of every row, all 8 loads issued together; a
  // reduce-scatter over the warp leaves row 4 b4 + 2 b3 + b2 (b_i the lane's
  // bits) on the lanes with b1 = b0 = 0, which write its key.  The split
  // scan's values are FP32-level already: their keys are formed directly.
  //
  // The split scan's keys are used unrescored when the kernel values they
  // give are accurate enough for this query.  The D^2 error of a candidate is
  // taken as a.acc_scale r^2 with r = |x~| + |y~| its centred operands'
  // magnitude (the scale the split's FP32 accumulation error follows; the
  // constant is 2 to 2.5 times the largest measured), which bounds the
  // relative error of the neighbour sum by sum K e / sum K over the collected
  // candidates.  The query's rows are rescored like the BF16 scan's when that
  // bound is above a.acc_tol and above the bound of the FP32 difference form
  // itself, ((d + 7) / 8 + 8) 2^-24 D^2 per candidate: where the split's bound
  // is the smaller one (queries far from every probed list, where both are
  // set by the FP32 rounding of D^2), rescoring would not tighten it.  A
  // caller that asks for the neighbours' distances (kde_search) gets FP32
  // difference-form ones, so those calls rescore too.
  //
  // The keys are formed six candidates a thread at a time, so that the loads
  // of their values, ids and norms are all in flight together.
  __shared__ int s_rescore;
  __shared__ unsigned long long s_kmin;
  bool rescore = a.rescore != 0 || a.nd2 != nullptr;
  unsigned long long kmin = ~0ull;
  if (!rescore) {
    const float inv = kernel_inv(a.kern, a.h);
    const float c32 = (float)((a.d + 7) / 8 + 8) * (1.0f / 16777216.0f);
    const bool lap = a.kern == KDE_KERN_LAPLACIAN;
    float ksum = 0.f, esum = 0.f, e32sum = 0.f;
    constexpr int kKU = 6;
    for (int j0 = tid; j0 < K; j0 += kKU * kNT) {
      int sl[kKU], pr[kKU];
      int64_t pos[kKU];
      bool row[kKU];
#pragma unroll
      for (int u = 0; u < kKU; ++u) {
        const int j = j0 + u * kNT;
        const int s = j < K ? sm.slot[j] : 0;
        int lo = 0, hi = a.P - 1;  // last segment with start <= s
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_seg[mid] <= s) lo = mid; else hi = mid - 1;
        }
        const int64_t off = s - s_seg[lo];
        sl[u] = s;
        pr[u] = lo;
        row[u] = j < K && off < s_llen[lo];
        pos[u] = s_lstart[lo] + off;  // list-order row of the candidate
      }
      float d2[kKU], xs[kKU];
      int32_t id[kKU];
#pragma unroll
      for (int u = 0; u < kKU; ++u) {
        d2[u] = j0 + u * kNT < K ? vals[sl[u]] : 0.f;
        id[u] = row[u] ? a.perm[pos[u]] : 0;
        xs[u] = row[u] && !lap ? a.XLsn[pos[u]] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kKU; ++u) {
        const int j = j0 + u * kNT;
        if (j >= K) continue;
        const unsigned long long key = row[u] ? pack_key(d2[u], id[u]) : ~0ull;
        sm.key[j] = key;
        kmin = min(kmin, key);
        if (row[u] && !lap) {
          const float kv = kernel_from_dist(a.kern, d2[u], inv);
          const float r = sqrtf(xs[u]) + s_dc[pr[u]];
          const float ed = a.acc_scale * r * r;  // the D^2 error taken
          const float e32 = c32 * d2[u];         // the FP32 difference form's
          // d log K / d D^2: 1 / (2 h^2) (Gaussian), 1 / (2 h r) (exponential)
          const float g = a.kern == KDE_KERN_GAUSSIAN
                              ? inv
                              : inv / (2.f * sqrtf(fmaxf(d2[u], fmaxf(ed, e32))));
          ksum += kv;
          esum += kv * fminf(ed * g, 1.f);
          e32sum += kv * fminf(e32 * g, 1.f);
        }
      }
    }
    ksum = warp_sum(ksum);
    esum = warp_sum(esum);
    e32sum = warp_sum(e32sum);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    __shared__ float s_ks[kNW], s_es[kNW], s_e32[kNW];
    __shared__ unsigned long long s_km[kNW];
    if (lane == 0) {
      s_ks[warp] = ksum;
      s_es[warp] = esum;
      s_e32[warp] = e32sum;
      s_km[warp] = kmin;
    }
    __syncthreads();
    if (tid == 0) {
      float kt = 0.f, et = 0.f, e32t = 0.f;
      unsigned long long km = ~0ull;
      for (int w = 0; w < kNW; ++w) {
        kt += s_ks[w];
        et += s_es[w];
        e32t += s_e32[w];
        km = min(km, s_km[w]);
      }
      s_rescore = et > a.acc_tol * kt && et > e32t ? 1 : 0;
      s_kmin = km;
    }
    __syncthreads();
    rescore = s_rescore != 0;
    kmin = rescore ? ~0ull : s_kmin;
  }
  if (rescore) {
    const int dp4 = a.dp >> 2;
    const float4* y4 = reinterpret_cast<const float4*>(y);
    const float4* X4 = reinterpret_cast<const float4*>(a.XL);
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
    const int myrow = (h4 ? 4 : 0) + (h3 ? 2 : 0) + (h2 ? 1 : 0);
    // the row of candidate j in the list-ordered copy, or -1
    auto locate = [&](int j) -> int64_t {
      if (j >= K) return -1;
      const int s = sm.slot[j];
      int lo = 0, hi = a.P - 1;  // last segment with start <= s
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_seg[mid] <= s) lo = mid; else hi = mid - 1;
      }
      // a slot past its list (the segment's padding) is never a row
      return s - s_seg[lo] < s_llen[lo] ? s_lstart[lo] + (s - s_seg[lo]) : -1;
    };
    const int lines = (a.dp * 4 + 127) >> 7;  // 128-byte lines of a row
    // lane u (u < 8) locates row j0 + u of the warp's group
    int64_t p_own = locate(warp * 8 + (lane & 7));
    for (int j0 = warp * 8; j0 < K; j0 += kNW * 8) {
      // the next group's rows are requested into L2 now, one group ahead of
      // their loads: lane l takes lines l & 3, (l & 3) + 4, ... of row l >> 2
      const int64_t p_next = locate(j0 + kNW * 8 + (lane & 7));
      {
        const int64_t pf = __shfl_sync(0xffffffffu, p_next, lane >> 2);
        if (pf >= 0) {
          const char* row = reinterpret_cast<const char*>(a.XL + pf * a.dp);
          for (int ln = lane & 3; ln < lines; ln += 4) prefetch_l2(row + ((size_t)ln << 7));
        }
      }
      int64_t pos[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) pos[u] = __shfl_sync(0xffffffffu, p_own, u);
      const int64_t p_mine = __shfl_sync(0xffffffffu, p_own, myrow);
      const int32_t id = (lane & 3) == 0 && p_mine >= 0 ? a.perm[p_mine] : 0;
      float acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = 0.f;
      for (int c4 = lane; c4 < dp4; c4 += 32) {
        const float4 yv = y4[c4];
        float4 xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) xv[u] = pos[u] >= 0 ? __ldg(X4 + pos[u] * dp4 + c4) : yv;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float t0 = xv[u].x - yv.x, t1 = xv[u].y - yv.y, t2 = xv[u].z - yv.z,
                      t3 = xv[u].w - yv.w;
          acc[u] = fmaf(t0, t0, acc[u]);
          acc[u] = fmaf(t1, t1, acc[u]);
          acc[u] = fmaf(t2, t2, acc[u]);
          acc[u] = fmaf(t3, t3, acc[u]);
        }
      }
      float v4[4], v2[2], v1;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float keep = h4 ? acc[i + 4] : acc[i], send = h4 ? acc[i] : acc[i + 4];
        v4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float keep = h3 ? v4[i + 2] : v4[i], send = h3 ? v4[i] : v4[i + 2];
        v2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
      }
      {
        const float keep = h2 ? v2[1] : v2[0], send = h2 ? v2[0] : v2[1];
        v1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
      }
      v1 += __shfl_xor_sync(0xffffffffu, v1, 2);
      v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
      if ((lane & 3) == 0 && j0 + myrow < K)
        sm.key[j0 + myrow] = p_mine >= 0 ? pack_key(v1, id) : ~0ull;  // ~0: +inf, id -1
      p_own = p_next;
    }
  }
  __syncthreads();
  // the split scan's keys are the values the bracket was taken on
  rank_keys(a, sm, K, q, y, rescore ? 0.f : 2.f * s_E, rescore ? -1.f : tk_lo, kmin);
}

}  // namespace

void launch_query_norms(const float* Y, int64_t nq, int dp, float* out, cudaStream_t s) {
  if (nq <= 0) return;
  k_query_norms<<<(unsigned)((nq + 7) / 8), 256, 0, s>>>(Y, nq, dp, out);
}

void launch_exclusive_scan_i64(const int64_t* in, int64_t count, int64_t* out, cudaStream_t s) {
  k_exclusive_scan<<<1, 1024, 0, s>>>(in, count, out, 1);
}

void launch_select_probes(const float* D, int64_t nq, int L, const float* Y, int d, int dp,
                          const float* C, int nprobe, int margin, int32_t* probes,
                          float* probe_d2, const int64_t* active, int64_t q0, cudaStream_t s) {
  if (nq <= 0) return;
  int kprime = nprobe + margin;
  if (kprime > kProbeCap) kprime = kProbeCap;
  if (kprime <= 32) {
    k_select_probes_warp<<<(unsigned)((nq + kNW - 1) / kNW), kNT, 0, s>>>(
        D, nq, L, Y, d, dp, C, nprobe, kprime, probes, probe_d2, active, q0);
    return;
  }
  set_dynamic_smem(reinterpret_cast<const void*>(&k_select_probes), sizeof(ProbeSmem));
  k_select_probes<<<(unsigned)nq, kNT, sizeof(ProbeSmem), s>>>(D, nq, L, Y, d, dp, C, nprobe,
                                                              kprime, probes, probe_d2, active,
                                                              q0);
}

void launch_plan_pairs(const int32_t* probes, int64_t nq, int P, const int64_t* list_off, int L,
                       int64_t* q_count, int64_t* q_real, int64_t* q_off, int64_t* seg_off,
                       int64_t* list_cnt,
                       int64_t* bucket_off, int64_t* bucket_fill, int32_t* pair_q,
                       int64_t* pair_dst, int64_t* tile_cnt, int64_t* tile_off,
                       const int32_t* lorder, int qtile, cudaStream_t s) {
  cudaMemsetAsync(list_cnt, 0, sizeof(int64_t) * L, s);
  cudaMemsetAsync(bucket_fill, 0, sizeof(int64_t) * L, s);
  k_plan_segments<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(probes, nq, P, list_off, q_count,
                                                              q_real, seg_off, list_cnt);
  k_exclusive_scan<<<1, 1024, 0, s>>>(q_count, nq, q_off, 32);  // 128-byte aligned regions
  k_exclusive_scan<<<1, 1024, 0, s>>>(list_cnt, L, bucket_off, 1);
  const int64_t np = nq * P;
  k_plan_fill<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(probes, nq, P, q_off, seg_off,
                                                           bucket_off, bucket_fill, pair_q,
                                                           pair_dst);
  k_plan_tiles<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(list_cnt, L, qtile, lorder,
                                                           tile_cnt);
  k_exclusive_scan<<<1, 1024, 0, s>>>(tile_cnt, L, tile_off, 1);
}

void launch_select_order(const int32_t* probes, int64_t nq, int P, int L, int64_t* ord_cnt,
                         int64_t* ord_off, int64_t* ord_fill, int32_t* order, cudaStream_t s) {
  if (nq <= 0) return;
  cudaMemsetAsync(ord_cnt, 0, sizeof(int64_t) * L, s);
  cudaMemsetAsync(ord_fill, 0, sizeof(int64_t) * L, s);
  const unsigned g = (unsigned)((nq + 255) / 256);
  k_order_count<<<g, 256, 0, s>>>(probes, nq, P, ord_cnt);
  k_exclusive_scan<<<1, 1024, 0, s>>>(ord_cnt, L, ord_off, 1);
  k_order_fill<<<g, 256, 0, s>>>(probes, nq, P, ord_off, ord_fill, order);
}

void launch_select_neighbors(const SelectArgs& a, cudaStream_t s) {
  if (a.nq <= 0) return;
  // the five-block instance spills a few registers: worth it where no rows
  // are rescored (the split scan's keys), not in the rescoring loop
  if (a.k <= kSmallCapMaxK && a.rescore == 0 && a.nd2 == nullptr) {
    set_dynamic_smem(reinterpret_cast<const void*>(&k_select_neighbors<SelectSmemSmall, 5>),
                     select_smem_bytes<SelectSmemSmall>(kMaxProbe));
    k_select_neighbors<SelectSmemSmall, 5>
        <<<(unsigned)a.nq, kNT, select_smem_bytes<SelectSmemSmall>(a.P), s>>>(a);
  } else {
    set_dynamic_smem(reinterpret_cast<const void*>(&k_select_neighbors<SelectSmem, 4>),
                     select_smem_bytes<SelectSmem>(kMaxProbe));
    k_select_neighbors<SelectSmem, 4><<<(unsigned)a.nq, kNT, select_smem_bytes<SelectSmem>(a.P), s>>>(a);
  }
}

}  // namespace deann
