// The DEANN estimator's sampling half (Algorithm 1) and random
// sampling (Lemma RS), plus the adjoint of both.
//
// One CTA of 256 threads serves one query:
//  1. the neighbour set X_1 (k ids, -1 padding, duplicates allowed) is sorted
//     and deduplicated in shared memory: k' = |X_1|;
//  2. s1 = sum_{X_1} K_h(x, y) (or taken from the selection kernel);
//  3. the sample S: Philox draws t = 0, 1, 2, ... of the query's stream are
//     mapped to indices in [0, n); draws that fall in X_1 are rejected (binary
//     search in shared memory) and the first m accepted ones are kept, so S is
//     uniform on X \ X_1 with repetition.  Draws are generated 256 at a time
//     and ranked with warp ballots, which reproduces the sequential order
//     exactly.  Past 64 m + 4096 draws the query is abandoned with an error
//     flag (reachable only when k' is close to n);
//  4. the sampled rows are gathered with coalesced 16-byte loads (G lanes per
//     row, several rows in flight per group) and s2 = sum_S K_h(x, y);
//  5. out = (s1 + ((n - k') / m) s2) / n.
// "drop" mode (sample_mode 1) instead takes draws 0..m-1 from all of X and
// gives the ones in X_1 weight zero: out = s1 / n + s2 / m.
// Permuted mode (sample_mode 2, Algorithm 2) reads the window of m
// consecutive rows of the permuted dataset XP (XP[i] = X[pi(i)]) starting at
// ell = (qid m) mod n, wrapping at n; window entries whose id pi(j) is in X_1
// are dropped and the m' kept ones are normalised by m':
// out = (s1 + ((n - k') / m') s2) / n (s1 / n when m' = 0).
#include <algorithm>

#include "common.cuh"

namespace deann {

namespace {

constexpr int kNT = 256;
constexpr int kNW = kNT / 32;
constexpr int kChunk = 2048;   // samples staged per gather round
constexpr int kUnroll = 8;     // rows in flight per lane group

constexpr int kFiltWords = 1024;  // membership filter: 32,768 bits
struct EstSmem {
  int nb[kMaxK];               // sorted distinct neighbour ids
  uint32_t filt[kFiltWords];   // bit (id mod 32768) set for every id in nb
  int S[kChunk];
  int warp_cnt[kNW];
  float red[kNW];
  int kk;
  int cnt;
  int64_t tnext;
  int status;
  int dup;                     // the hash set met a repeated id
  static constexpr bool kSorted = true;  // nb holds X_1 sorted (binary search)
};

// The phased estimator's draw kernel needs X_1 only as the hash set and its
// filter; its draws go straight to the caller's array.
struct PhaseSmem {
  uint32_t filt[kFiltWords];
  int warp_cnt[kNW];
  int kk;
  int cnt;
  int64_t tnext;
  int status;
  int dup;
  static constexpr bool kSorted = false;
};

__device__ __forceinline__ bool is_member(const int* nb, int kk, int64_t id) {
  int lo = 0, hi = kk;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (nb[mid] < id) lo = mid + 1; else hi = mid;
  }
  return lo < kk && nb[lo] == id;
}

// The same test, with the filter first: a clear bit rules the id out at the
// cost of one shared load, a set bit (a member, or another id with the same
// residue) falls back to the search.
__device__ __forceinline__ bool is_member_f(const EstSmem& sm, int kk, int64_t id) {
  const uint32_t w = sm.filt[(id >> 5) & (kFiltWords - 1)];
  if (((w >> (id & 31)) & 1u) == 0u) return false;
  return is_member(sm.nb, kk, id);
}

// Hash set of the neighbour ids (open addressing, linear probing, at most
// kMaxK ids in twice as many slots), for the query path, where the estimator
// needs X_1 only for membership and k': it replaces the sort.  Slots hold an
// id or -1.
constexpr int kHashBits = 12;
constexpr int kHashSlots = 1 << kHashBits;
static_assert(kHashSlots >= 2 * kMaxK, "the hash set keeps its load at most 1/2");
__device__ __forceinline__ uint32_t hash_slot(int id) {
  return ((uint32_t)id * 2654435761u) >> (32 - kHashBits);  // Knuth's multiplicative hash
}

__device__ __forceinline__ bool hash_has(const int* hs, int id) {
  uint32_t h = hash_slot(id);
  for (int p = 0; p < kHashSlots; ++p) {  // ends at the id or at the first empty slot
    const int v = hs[h];
    if (v == id) return true;
    if (v < 0) return false;
    h = (h + 1) & (kHashSlots - 1);
  }
  return false;
}

// Membership with the filter first (one shared load rules most ids out).
template <class SMT>
__device__ __forceinline__ bool is_member_h(const SMT& sm, const int* hs, int64_t id) {
  const uint32_t w = sm.filt[(id >> 5) & (kFiltWords - 1)];
  if (((w >> (id & 31)) & 1u) == 0u) return false;
  return hash_has(hs, (int)id);
}

// Ascending bitonic sort of v[0..P2) (P2 a power of two) by the whole CTA;
// ends with a barrier.
__device__ void block_bitonic_sort(int* v, int P2) {
  const int tid = threadIdx.x;
  for (int size = 2; size <= P2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < P2 / 2; i += kNT) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const int a = v[lo], b = v[hi];
        if ((a > b) == up) {
          v[lo] = b;
          v[hi] = a;
        }
      }
      __syncthreads();
    }
}

// Loads, sorts and deduplicates the neighbour row into sm.nb; sets sm.kk, or
// sm.status = 1 when an id is >= n.
__device__ void load_neighbours(const int32_t* __restrict__ row, int k, int64_t n, EstSmem& sm,
                                int* tmp /* >= next_pow2(k) ints */) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int P2 = 1;
  while (P2 < k) P2 <<= 1;
  if (tid == 0) sm.status = 0;
  __syncthreads();
  for (int i = tid; i < P2; i += kNT) {
    int v = 0x7fffffff;
    if (i < k) {
      const int32_t id = row[i];
      if (id >= 0) {
        if ((int64_t)id >= n) sm.status = 1;
        else v = id;
      }
    }
    tmp[i] = v;
  }
  __syncthreads();
  block_bitonic_sort(tmp, P2);
  // compact the distinct valid ids, keeping sorted order
  int base = 0;
  for (int b0 = 0; b0 < P2; b0 += kNT) {
    const int i = b0 + tid;
    const bool keep = i < P2 && tmp[i] != 0x7fffffff && (i == 0 || tmp[i] != tmp[i - 1]);
    const unsigned mk = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) sm.warp_cnt[warp] = __popc(mk);
    __syncthreads();
    int off = base, tot = 0;
    for (int w = 0; w < kNW; ++w) {
      if (w < warp) off += sm.warp_cnt[w];
      tot += sm.warp_cnt[w];
    }
    if (keep) sm.nb[off + __popc(mk & ((1u << lane) - 1u))] = tmp[i];
    base += tot;
    __syncthreads();
  }
  if (tid == 0) sm.kk = base;
  for (int i = tid; i < kFiltWords; i += kNT) sm.filt[i] = 0u;
  __syncthreads();
  for (int i = tid; i < base; i += kNT) {
    const int id = sm.nb[i];
    atomicOr(&sm.filt[(id >> 5) & (kFiltWords - 1)], 1u << (id & 31));
  }
  __syncthreads();
}

// Inserts the neighbour row into the hash set hs and the filter: sm.kk
// receives the number of distinct valid ids, sm.status = 1 when an id is >= n.
template <class SMT>
__device__ void load_neighbours_hash(const int32_t* __restrict__ row, int k, int64_t n,
                                     SMT& sm, int* hs) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < kHashSlots; i += kNT) hs[i] = -1;
  for (int i = tid; i < kFiltWords; i += kNT) sm.filt[i] = 0u;
  if (tid == 0) {
    sm.status = 0;
    sm.kk = 0;
    sm.dup = 0;
  }
  __syncthreads();
  int mine = 0;
  for (int i = tid; i < k; i += kNT) {
    const int32_t id = row[i];
    if (id < 0) continue;
    if ((int64_t)id >= n) {
      sm.status = 1;
      continue;
    }
    uint32_t h = hash_slot(id);
    for (int p = 0; p < kHashSlots; ++p) {
      const int prev = atomicCAS(&hs[h], -1, id);
      if (prev == -1) {
        ++mine;
        atomicOr(&sm.filt[(id >> 5) & (kFiltWords - 1)], 1u << (id & 31));
        break;
      }
      if (prev == id) {  // a duplicate
        sm.dup = 1;
        break;
      }
      h = (h + 1) & (kHashSlots - 1);
    }
  }
  mine = __reduce_add_sync(0xffffffffu, mine);
  if (lane == 0) atomicAdd(&sm.kk, mine);
  __syncthreads();
}

// Fills S_out[0..sm.cnt) (sm.S when S_out is null) with the next accepted
// sample indices (at most `room`), starting at draw t0; sets sm.tnext to the
// first unused draw.
// mode 0 rejects members of X_1; mode 1 accepts every draw.  Returns false
// when the draw cap is reached.  A round covers kNT * kDraws consecutive
// draws, thread i taking kDraws of them in a row, so the accepted draws are
// ranked in draw order by a block prefix sum of the per-thread counts.
constexpr int kDraws = 4;
// Membership is tested on the hash set hs when given, else on sm.nb (an
// SMT without the sorted set always takes hs and S_out).
template <class SMT>
__device__ bool draw_chunk(uint64_t seed, uint64_t qid, uint64_t n, int64_t t0, int64_t cap,
                           int room, int mode, const SMT& smc, SMT& sm,
                           const int* hs = nullptr, int* S_out = nullptr) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int* S;
  if constexpr (SMT::kSorted) S = S_out != nullptr ? S_out : sm.S;
  else S = S_out;
  int filled = 0;
  int64_t t = t0;
  bool ok = true;
  while (filled < room) {
    if (t >= cap) {
      ok = false;
      break;
    }
    const int64_t tb = t + (int64_t)tid * kDraws;
    int ids[kDraws];
    unsigned accm = 0u;
#pragma unroll
    for (int r = 0; r < kDraws; ++r) {
      ids[r] = 0;
      if (tb + r < cap) {
        ids[r] = (int)draw_index(seed, qid, (uint32_t)(tb + r), 0u, n);
        bool member;
        if constexpr (SMT::kSorted)
          member = hs != nullptr ? is_member_h(smc, hs, ids[r]) : is_member_f(smc, smc.kk, ids[r]);
        else
          member = is_member_h(smc, hs, ids[r]);
        if (mode == 1 || !member) accm |= 1u << r;
      }
    }
    const int mine = __popc(accm);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) sm.warp_cnt[warp] = incl;
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < kNW; ++w) {
      if (w < warp) off += sm.warp_cnt[w];
      tot += sm.warp_cnt[w];
    }
    int rank = off + incl - mine;
    const int left = room - filled;
#pragma unroll
    for (int r = 0; r < kDraws; ++r) {
      if ((accm >> r) & 1u) {
        if (rank < left) {
          S[filled + rank] = ids[r];
          if (rank == left - 1) sm.tnext = tb + r + 1;
        }
        ++rank;
      }
    }
    if (tot >= left) {
      filled = room;
    } else {
      filled += tot;
      t += (int64_t)kNT * kDraws;
      if (t > cap) t = cap;
      if (tid == 0) sm.tnext = t;
    }
    __syncthreads();
  }
  if (tid == 0) sm.cnt = filled;
  __syncthreads();
  return ok;
}

// Algorithm 2 window, positions t in [t0, t0 + room): row j = (w0 + t) mod n
// of XP holds original id pi(j) = wperm[j].  Rows whose id is not in X_1 go to
// sm.S in window order and sm.cnt counts them; srow (nullable) receives
// pi(j), or -1 for a dropped entry, at its window position t.
__device__ void window_chunk(const int32_t* __restrict__ wperm, int64_t n, int64_t w0, int t0,
                             int room, EstSmem& sm, int32_t* srow) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int filled = 0;
  for (int b0 = 0; b0 < room; b0 += kNT) {
    const int t = t0 + b0 + tid;
    bool keep = false;
    int j = 0;
    if (b0 + tid < room) {
      int64_t jj = w0 + t;  // w0 < n and t < m <= n
      if (jj >= n) jj -= n;
      j = (int)jj;
      const int32_t id = wperm[j];
      keep = !is_member_f(sm, sm.kk, id);
      if (srow) srow[t] = keep ? id : -1;
    }
    const unsigned mk = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) sm.warp_cnt[warp] = __popc(mk);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < kNW; ++w) {
      if (w < warp) off += sm.warp_cnt[w];
      tot += sm.warp_cnt[w];
    }
    if (keep) sm.S[filled + off + __popc(mk & ((1u << lane) - 1u))] = j;
    filled += tot;
    __syncthreads();
  }
  if (tid == 0) sm.cnt = filled;
  __syncthreads();
}

// Requests rows ids[nb .. nb + 8) of X into L2 ahead of a warp's loads of
// them: lane l takes lines l & 3, (l & 3) + 4, ... of row nb + (l >> 2).
__device__ __forceinline__ void prefetch_next_rows(const float* __restrict__ X, int dp,
                                                   const int* ids, int cnt, int nb) {
  const int lane = threadIdx.x & 31, j = nb + (lane >> 2);
  if (j >= cnt) return;
  const int rid = ids[j];
  if (rid < 0) return;
  const char* row = reinterpret_cast<const char*>(X + (size_t)rid * dp);
  const int lines = (dp * 4 + 127) >> 7;
  for (int ln = lane & 3; ln < lines; ln += 4) prefetch_l2(row + ((size_t)ln << 7));
}

// Sum of kernel values over rows ids[0..cnt) of X, by groups of G lanes.
// Returns this thread's partial (lane-in-group 0 holds the group sums).
// kPf: request the next rows into L2 ahead of their loads (G = 32), for rows
// that come from HBM; the phased estimator's rows are L2 hits already.
template <int G, bool L1, bool kPf = true>
__device__ float gather_sum(const float* __restrict__ X, int dp, const float* __restrict__ ys,
                            const int* ids, int cnt, int kern, float inv) {
  const int tid = threadIdx.x;
  const int lig = tid & (G - 1);
  constexpr int kGpw = 32 / G;  // groups per warp
  const int gw = (tid & 31) / G, warp = tid >> 5;
  const int dp4 = dp >> 2;
  const float4* y4 = reinterpret_cast<const float4*>(ys);
  float part = 0.f;
  // warp-uniform trip count: the group reductions below need all 32 lanes
  for (int wb = warp * kGpw * kUnroll; wb < cnt; wb += kNW * kGpw * kUnroll) {
    const int base = wb + gw * kUnroll;
    // 32-bit row ids keep the register footprint small; kUnroll independent
    // 16-byte loads per lane are in flight at once
    int rid[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) rid[u] = base + u < cnt ? ids[base + u] : -1;
    if (G == 32 && kPf) prefetch_next_rows(X, dp, ids, cnt, wb + kNW * kUnroll);
    const float4* X4 = reinterpret_cast<const float4*>(X);
    float acc[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) acc[u] = 0.f;
    for (int j4 = lig; j4 < dp4; j4 += G) {
      const float4 yv = y4[j4];
      float4 xv[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        xv[u] = rid[u] >= 0 ? __ldg(X4 + (size_t)rid[u] * dp4 + j4) : yv;
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const float a = xv[u].x - yv.x, b = xv[u].y - yv.y, c = xv[u].z - yv.z,
                    e = xv[u].w - yv.w;
        if (L1) {
          acc[u] += (fabsf(a) + fabsf(b)) + (fabsf(c) + fabsf(e));
        } else {
          acc[u] = fmaf(a, a, acc[u]);
          acc[u] = fmaf(b, b, acc[u]);
          acc[u] = fmaf(c, c, acc[u]);
          acc[u] = fmaf(e, e, acc[u]);
        }
      }
    }
    if (G == 32) {
      // reduce-scatter of the kUnroll = 8 rows over the warp: three halving
      // exchanges leave lane l with a partial of row 4 b4 + 2 b3 + b2 (b_i
      // its bits), two butterflies finish it; the kernel is then evaluated
      // once per row, on 8 lanes at once
      static_assert(kUnroll == 8, "the reduce-scatter splits 8 rows");
      const int lane = tid & 31;
      float v4[4], v2[2], v1;
      const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
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
      const int row = (h4 ? 4 : 0) + (h3 ? 2 : 0) + (h2 ? 1 : 0);
      if ((lane & 3) == 0 && base + row < cnt) part += kernel_from_dist(kern, v1, inv);
    } else if (G == 8 && !kPf) {
      // (the phased gathers) reduce-scatter of the 8 rows over the group's 8
      // lanes: three halving exchanges leave lane l of the group with the
      // whole sum of row l (the same pairwise sums as group_sum, so the same
      // distance bits), and the kernel is evaluated once per row on all lanes
      float v4[4], v2[2], v1;
      const bool h4 = lig & 4, h2 = lig & 2, h1 = lig & 1;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float keep = h4 ? acc[i + 4] : acc[i], send = h4 ? acc[i] : acc[i + 4];
        v4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float keep = h2 ? v4[i + 2] : v4[i], send = h2 ? v4[i] : v4[i + 2];
        v2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
      }
      {
        const float keep = h1 ? v2[1] : v2[0], send = h1 ? v2[0] : v2[1];
        v1 = keep + __shfl_xor_sync(0xffffffffu, send, 1);
      }
      if (base + lig < cnt) part += kernel_from_dist(kern, v1, inv);
    } else {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const float dist = group_sum<G>(acc[u]);
        if (lig == 0 && base + u < cnt) part += kernel_from_dist(kern, dist, inv);
      }
    }
  }
  return part;
}

template <int G, bool kPf = true>
__device__ float gather_sum_k(const float* X, int dp, const float* ys, const int* ids, int cnt,
                              int kern, float inv) {
  return kern == KDE_KERN_LAPLACIAN ? gather_sum<G, true, kPf>(X, dp, ys, ids, cnt, kern, inv)
                                    : gather_sum<G, false, kPf>(X, dp, ys, ids, cnt, kern, inv);
}

__device__ float block_sum(float v, EstSmem& sm) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm.red[warp] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < kNW; ++w) t += sm.red[w];
  __syncthreads();
  return t;
}

// Permuted mode: the queries of a batch whose rows agree mod P = n / gcd(n, m)
// read the same window.  Block b serves the b-th query in (q mod P, q) order,
// so the blocks that share a window are scheduled together and its rows come
// from HBM about once, the other reads hitting L2.  A bijection of [0, nq):
// with nq = A P + B, the first B residue classes hold A + 1 queries, the rest A.
__device__ __forceinline__ int64_t window_order(int64_t b, int64_t nq, int64_t P) {
  if (P >= nq) return b;
  const int64_t A = nq / P, B = nq % P;
  int64_t s, j;
  if (b < B * (A + 1)) {
    s = b / (A + 1);
    j = b % (A + 1);
  } else {
    const int64_t c = b - B * (A + 1);
    s = B + c / A;
    j = c % A;
  }
  return s + j * P;
}

template <int G>
__global__ void __launch_bounds__(kNT, 4) k_estimate(SampleArgs a) {
  __shared__ EstSmem sm;
  // the sort's scratch, or the hash set of X_1 on the query path (s1 given,
  // rejection sampling): there only membership and k' are needed
  __shared__ int tmp[kHashSlots];
  extern __shared__ float4 ys4[];
  float* ys = reinterpret_cast<float*>(ys4);
  const int64_t q = a.mode == 2 ? window_order(blockIdx.x, a.nq, a.win_period) : blockIdx.x;
  const int tid = threadIdx.x;
  if (a.active != nullptr && q >= *a.active) return;  // inactive row: no output
  const uint64_t qid = a.qid_offset + (a.dev_qid != nullptr ? *a.dev_qid : 0ull) + (uint64_t)q;
  for (int j = tid; j < a.dp; j += kNT) ys[j] = a.Y[q * a.dp + j];
  const int k = a.rs ? 0 : a.k;
  const bool hashed = k > 0 && a.s1_in != nullptr && a.mode == 0;
  if (hashed) {
    load_neighbours_hash(a.nbr + q * a.k, k, a.n, sm, tmp);
  } else if (k > 0) {
    load_neighbours(a.nbr + q * a.k, k, a.n, sm, tmp);
  } else {
    if (tid == 0) {
      sm.kk = 0;
      sm.status = 0;
    }
    __syncthreads();
  }
  if (sm.status) {
    if (tid == 0) {
      atomicOr(a.err, KDE_ERRBIT_BADNBR);
      if (a.out) a.out[q] = __int_as_float(0x7fc00000);
    }
    return;
  }
  const int kk = sm.kk;
  const float inv = kernel_inv(a.kern, a.h);
  float s1 = 0.f;
  if (a.s1_in != nullptr) {
    s1 = a.s1_in[q];
  } else if (kk > 0 && a.out) {
    s1 = block_sum(gather_sum_k<G>(a.X, a.dp, ys, sm.nb, kk, a.kern, inv), sm);
  }
  const bool sampled = !((int64_t)kk == a.n || a.m == 0);
  float s2 = 0.f;
  bool ok = true;
  int kept = a.m;  // m' of the permuted mode
  if (sampled && a.mode == 2) {
    const int64_t w0 = (int64_t)(((qid % (uint64_t)a.n) * (uint64_t)a.m) % (uint64_t)a.n);
    float part = 0.f;
    kept = 0;
    for (int t0 = 0; t0 < a.m; t0 += kChunk) {
      const int room = min(kChunk, a.m - t0);
      window_chunk(a.wperm, a.n, w0, t0, room, sm, a.samples ? a.samples + q * a.m : nullptr);
      if (a.out) part += gather_sum_k<G>(a.XP, a.dp, ys, sm.S, sm.cnt, a.kern, inv);
      kept += sm.cnt;
      __syncthreads();
    }
    if (a.out) s2 = block_sum(part, sm);
  } else if (sampled) {
    const int64_t cap = a.mode == 1 ? (int64_t)a.m : 64 * (int64_t)a.m + 4096;
    int64_t t0 = 0;
    int got = 0;
    float part = 0.f;
    while (got < a.m) {
      const int room = min(kChunk, a.m - got);
      if (!draw_chunk(a.seed, qid, (uint64_t)a.n, t0, cap, room, a.mode, sm, sm,
                      hashed ? tmp : nullptr)) {
        ok = false;
        break;
      }
      const int cnt = sm.cnt;
      t0 = sm.tnext;
      if (a.samples)
        for (int i = tid; i < cnt; i += kNT) a.samples[q * a.m + got + i] = sm.S[i];
      if (a.out) {
        if (a.mode == 1) {
          // draws inside X_1 carry weight zero: compact them away first
          __syncthreads();
          if (tid == 0) {
            int w = 0;
            for (int i = 0; i < cnt; ++i)
              if (!is_member(sm.nb, kk, sm.S[i])) sm.S[w++] = sm.S[i];
            sm.cnt = w;
          }
          __syncthreads();
        }
        part += gather_sum_k<G>(a.X, a.dp, ys, sm.S, sm.cnt, a.kern, inv);
      }
      got += cnt;
      __syncthreads();
    }
    if (a.out) s2 = block_sum(part, sm);
  }
  if (tid == 0) {
    if (!ok) {
      atomicOr(a.err, KDE_ERRBIT_DRAWCAP);
      if (a.out) a.out[q] = __int_as_float(0x7fc00000);
      if (a.samples)
        for (int i = 0; i < a.m; ++i) a.samples[q * a.m + i] = -1;
    } else if (a.out) {
      const double n = (double)a.n;
      double est;
      if (!sampled || kept == 0) est = (double)s1 / n;
      else if (a.mode == 1) est = (double)s1 / n + (double)s2 / (double)a.m;
      else if (a.mode == 2) est = ((double)s1 + (n - (double)kk) / (double)kept * (double)s2) / n;
      else est = ((double)s1 + (n - (double)kk) / (double)a.m * (double)s2) / n;
      a.out[q] = (float)est;
    }
    if (sampled == false && a.samples)
      for (int i = 0; i < a.m; ++i) a.samples[q * a.m + i] = -1;
  }
}

// ---------------------------------------------------------------------------
// Phased estimator.  The sum s2 over the sample does not depend on the order
// of its terms, so the batch's draws are regrouped by the window of X they
// fall in, and the windows are read one after another: a window of tens of
// megabytes stays in L2 while every query's rows inside it are gathered, and
// X comes from HBM about once per call instead of once per draw.
// ---------------------------------------------------------------------------

// Per query: X_1 as a hash set, the m accepted draws of Algorithm 1 (the same
// Philox stream and rejection as k_estimate) into shared memory, then a
// stable counting sort of them by window (window-major, then warp, then draw
// order) written to ph.ids, with the run starts in ph.off and k' in ph.info.
__global__ void __launch_bounds__(kNT) k_draw_phased(SampleArgs a, PhaseArgs ph) {
  __shared__ PhaseSmem sm;
  __shared__ int hs[kHashSlots];
  extern __shared__ int dsm[];
  int* drawn = dsm;          // [m] accepted draws in draw order
  int* wc = dsm + a.m;       // [kNW x P] per-warp window counts, then run starts
  const int64_t q = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (a.active != nullptr && q >= *a.active) return;  // inactive row: no output
  const uint64_t qid = a.qid_offset + (a.dev_qid != nullptr ? *a.dev_qid : 0ull) + (uint64_t)q;
  const int P = ph.P;
  int32_t* off = ph.off + q * (P + 1);
  load_neighbours_hash(a.nbr + q * a.k, a.k, a.n, sm, hs);
  if (sm.status) {
    for (int p = tid; p <= P; p += kNT) off[p] = 0;
    if (tid == 0) {
      atomicOr(a.err, KDE_ERRBIT_BADNBR);
      ph.info[q] = -1;
    }
    return;
  }
  const int kk = sm.kk;
  if ((int64_t)kk == a.n) {  // X_1 is all of X: nothing is sampled
    for (int p = tid; p <= P; p += kNT) off[p] = 0;
    if (tid == 0) ph.info[q] = kk;
    return;
  }
  const int64_t cap = 64 * (int64_t)a.m + 4096;
  int64_t t0 = 0;
  int got = 0;
  while (got < a.m) {
    const int room = min(kChunk, a.m - got);
    if (!draw_chunk(a.seed, qid, (uint64_t)a.n, t0, cap, room, 0, sm, sm, hs, drawn + got)) {
      for (int p = tid; p <= P; p += kNT) off[p] = 0;
      if (tid == 0) {
        atomicOr(a.err, KDE_ERRBIT_DRAWCAP);
        ph.info[q] = -1;
      }
      return;
    }
    t0 = sm.tnext;
    got += sm.cnt;
    __syncthreads();
  }
  for (int i = tid; i < kNW * P; i += kNT) wc[i] = 0;
  __syncthreads();
  // warp w sorts draws [s0, s1) of the query; lanes holding the same window
  // find one another with a match, the lowest of them counts for all
  const int sh = ph.shift;  // window of row id: id >> sh
  const int seg = (a.m + kNW - 1) / kNW;
  const int s0 = min(a.m, warp * seg), s1 = min(a.m, s0 + seg);
  for (int r = s0; r < s1; r += 32) {
    const int i = r + lane;
    const int b = i < s1 ? drawn[i] >> sh : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    if (b >= 0 && lane == __ffs(peers) - 1) wc[warp * P + b] += __popc(peers);
  }
  __syncthreads();
  // exclusive scan in (window, warp) order: wc[w P + b] becomes the start of
  // warp w's part of window b's run; off[b] the start of the run
  if (warp == 0) {
    int run = 0;
    for (int f0 = 0; f0 < P * kNW; f0 += 32) {
      const int f = f0 + lane;
      const int b = f / kNW, w = f % kNW;
      const int v = f < P * kNW ? wc[w * P + b] : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      if (f < P * kNW) {
        wc[w * P + b] = run + incl - v;
        if (w == 0) off[b] = run + incl - v;
      }
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) off[P] = run;
  }
  __syncthreads();
  // scatter in draw order: a lane's place is its warp's cursor for the window
  // plus the lanes below it with the same window
  int32_t* dst = ph.ids + q * (int64_t)a.m;
  for (int r = s0; r < s1; r += 32) {
    const int i = r + lane;
    const int id = i < s1 ? drawn[i] : 0;
    const int b = i < s1 ? id >> sh : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int base = b >= 0 ? wc[warp * P + b] : 0;
    __syncwarp();
    if (b >= 0) {
      dst[base + __popc(peers & ((1u << lane) - 1u))] = id;
      if (lane == __ffs(peers) - 1) wc[warp * P + b] = base + __popc(peers);
    }
    __syncwarp();
  }
  if (tid == 0) ph.info[q] = kk;
}

// Block (p, q) of a phase-major grid (blockIdx = p nq + q): the sums of the
// kernel values of query q's draws inside window p, one per warp.  No block
// barrier: the query row is read straight from global memory (L1 keeps it)
// and each warp writes its own partial.
static_assert(kNW == kPhaseWarps, "one partial per warp of the phased gather");
template <int G>
__global__ void __launch_bounds__(kNT, 4) k_gather_phase(SampleArgs a, PhaseArgs ph) {
  const int p = (int)(blockIdx.x / (uint64_t)a.nq);
  const int64_t q = (int64_t)(blockIdx.x % (uint64_t)a.nq);
  const int tid = threadIdx.x;
  if (a.active != nullptr && q >= *a.active) return;
  // a failed query's runs are all empty: the finish writes its NaN
  const int32_t* off = ph.off + q * (ph.P + 1);
  const int lo = off[p], hi = off[p + 1];
  float part = 0.f;
  if (hi > lo)
    part = gather_sum_k<G, false>(a.X, a.dp, a.Y + q * a.dp, ph.ids + q * (int64_t)a.m + lo,
                                  hi - lo, a.kern, kernel_inv(a.kern, a.h));
  part = warp_sum(part);
  if ((tid & 31) == 0) ph.part[((int64_t)p * a.nq + q) * kNW + (tid >> 5)] = part;
}

// out = (s1 + ((n - k') / m) s2) / n with s2 the warps' window sums added in
// (window, warp) order (s1 / n when nothing is sampled, NaN for a failed
// query).
__global__ void k_phase_finish(SampleArgs a, PhaseArgs ph) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nq) return;
  if (a.active != nullptr && q >= *a.active) return;
  const int kk = ph.info[q];
  if (kk < 0) {
    a.out[q] = __int_as_float(0x7fc00000);
    return;
  }
  const double n = (double)a.n;
  const float s1 = a.s1_in[q];
  double est;
  if ((int64_t)kk == a.n) {
    est = (double)s1 / n;
  } else {
    float s2 = 0.f;
    for (int p = 0; p < ph.P; ++p) {
      const float* w = ph.part + ((int64_t)p * a.nq + q) * kNW;
#pragma unroll
      for (int i = 0; i < kNW; ++i) s2 += w[i];
    }
    est = ((double)s1 + (n - (double)kk) / (double)a.m * (double)s2) / n;
  }
  a.out[q] = (float)est;
}

// Permuted windows shared by many queries (the tiled path): per query, the
// neighbour set, s1, and the sorted window positions of the members of X_1.
// A member x_id sits at window position (pi^-1(id) - ell) mod n when that is
// below m.
template <int G>
__global__ void __launch_bounds__(kNT, 4)
    k_window_prep(SampleArgs a, int32_t* __restrict__ drops, int dstride,
                  int32_t* __restrict__ dcnt, int32_t* __restrict__ kko,
                  float* __restrict__ s1o) {
  __shared__ EstSmem sm;
  __shared__ int tmp[kMaxK];
  extern __shared__ float4 ys4[];
  float* ys = reinterpret_cast<float*>(ys4);
  const int64_t q = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t qid = a.qid_offset + (a.dev_qid != nullptr ? *a.dev_qid : 0ull) + (uint64_t)q;
  const bool need_s1 = a.s1_in == nullptr;
  if (need_s1)
    for (int j = tid; j < a.dp; j += kNT) ys[j] = a.Y[q * a.dp + j];
  const int k = a.rs ? 0 : a.k;
  // ids that come from the search are distinct (and s1 comes with them): no
  // sort or deduplication is needed, only the count of valid ids
  const bool fast = a.nbr_distinct && k > 0 && !need_s1;
  const int32_t* row = k > 0 ? a.nbr + q * a.k : nullptr;
  if (k > 0 && !fast) {
    load_neighbours(row, k, a.n, sm, tmp);
  } else {
    if (tid == 0) {
      sm.kk = 0;
      sm.status = 0;
    }
    __syncthreads();
  }
  if (sm.status) {
    if (tid == 0) {
      atomicOr(a.err, KDE_ERRBIT_BADNBR);
      kko[q] = -1;
      dcnt[q] = 0;
      s1o[q] = 0.f;
    }
    return;
  }
  float s1 = 0.f;
  if (!need_s1) {
    s1 = a.s1_in[q];
  } else if (sm.kk > 0) {
    s1 = block_sum(
        gather_sum_k<G>(a.X, a.dp, ys, sm.nb, sm.kk, a.kern, kernel_inv(a.kern, a.h)), sm);
  }
  const int64_t w0 = (int64_t)(((qid % (uint64_t)a.n) * (uint64_t)a.m) % (uint64_t)a.n);
  __shared__ int vcnt[kNW];
  const int kscan = fast ? k : sm.kk;
  int cnt = 0, nvalid = 0;
  for (int b0 = 0; b0 < kscan; b0 += kNT) {
    const int t = b0 + tid;
    bool in = false, valid = false;
    int pos = 0;
    if (t < kscan) {
      const int32_t id = fast ? row[t] : sm.nb[t];
      valid = id >= 0 && (int64_t)id < a.n;
      if (valid) {
        int64_t pp = (int64_t)a.wpinv[id] - w0;
        if (pp < 0) pp += a.n;
        in = pp < (int64_t)a.m;
        pos = (int)pp;
      }
    }
    const unsigned mk = __ballot_sync(0xffffffffu, in);
    const unsigned mv = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) {
      sm.warp_cnt[warp] = __popc(mk);
      vcnt[warp] = __popc(mv);
    }
    __syncthreads();
    int off = cnt, tot = 0;
    for (int w = 0; w < kNW; ++w) {
      if (w < warp) off += sm.warp_cnt[w];
      tot += sm.warp_cnt[w];
      nvalid += vcnt[w];
    }
    if (in) tmp[off + __popc(mk & ((1u << lane) - 1u))] = pos;
    cnt += tot;
    __syncthreads();
  }
  const int kk = fast ? nvalid : sm.kk;
  int P2 = 1;
  while (P2 < cnt) P2 <<= 1;
  for (int i = cnt + tid; i < P2; i += kNT) tmp[i] = 0x7fffffff;
  __syncthreads();
  block_bitonic_sort(tmp, P2);
  for (int i = tid; i < cnt; i += kNT) drops[q * dstride + i] = tmp[i];
  if (tid == 0) {
    dcnt[q] = cnt;
    kko[q] = kk;
    s1o[q] = s1;
  }
}

__global__ void k_window_finish(int64_t nq, int64_t n, int m, int nslices,
                                const int32_t* __restrict__ dcnt, const int32_t* __restrict__ kko,
                                const float* __restrict__ s1o, const double* __restrict__ part,
                                float* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int kk = kko[q];
  if (kk < 0) {
    out[q] = __int_as_float(0x7fc00000);
    return;
  }
  double s2 = 0.0;
  for (int sl = 0; sl < nslices; ++sl) s2 += part[q * nslices + sl];
  const int kept = m - dcnt[q];  // k' = n leaves every window entry in X_1
  const double nn = (double)n, s1 = (double)s1o[q];
  out[q] = (float)(kept > 0 ? (s1 + (nn - (double)kk) / (double)kept * s2) / nn : s1 / nn);
}

// ---------------------------------------------------------------------------
// Adjoint: d out / d y and d out / d log h with X_1 and S held fixed (the
// pathwise derivative of the estimator; the paper defines none).  With
// out = sum_i w_i K_h(x_i, y): dK/dy = K g, dK/dlog h = K s, where
//   Gaussian:    g = (x - y) / h^2,        s = r^2 / h^2
//   exponential: g = (x - y) / (h r),      s = r / h      (g = 0 at r = 0)
//   Laplacian:   g = sign(x - y) / h,      s = |x - y|_1 / h
// Rows are regathered from the saved ids and recomputed, never stored.
// Each lane group keeps its own copy of the d-vector (NV float4s per lane);
// the groups are combined through shared-memory atomics at the end.
// ---------------------------------------------------------------------------
template <int G, int NV>
__device__ void grad_rows(const float* __restrict__ X, int dp, const float* __restrict__ ys,
                          const int* ids, int cnt, int kern, float h, float w,
                          float4 (&gacc)[NV], float& est, float& sl) {
  const int tid = threadIdx.x;
  const int lig = tid & (G - 1);
  constexpr int kGpw = 32 / G;
  const int gw = (tid & 31) / G, warp = tid >> 5;
  const int dp4 = dp >> 2;
  const float4* y4 = reinterpret_cast<const float4*>(ys);
  const float inv = kernel_inv(kern, h);
  if (G == 32 && NV == 1) {
    // d <= 128: eight rows per warp in flight, one 16-byte piece per lane; a
    // reduce-scatter leaves row 4 b4 + 2 b3 + b2 (b_i the lane's bits) on a
    // 4-lane group, each lane evaluates its row's kernel value and factors,
    // and shuffles hand every row's coefficient back to all lanes
    const int lane = tid & 31;
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
    const int myrow = (h4 ? 4 : 0) + (h3 ? 2 : 0) + (h2 ? 1 : 0);
    const float4 yv = lane < dp4 ? y4[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4* X4 = reinterpret_cast<const float4*>(X);
    for (int wb = warp * 8; wb < cnt; wb += kNW * 8) {
      prefetch_next_rows(X, dp, ids, cnt, wb + kNW * 8);
      float4 diff[8];
      float acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int rid = wb + u < cnt ? ids[wb + u] : -1;
        const float4 xv = rid >= 0 && lane < dp4 ? __ldg(X4 + (size_t)rid * dp4 + lane) : yv;
        diff[u] = make_float4(xv.x - yv.x, xv.y - yv.y, xv.z - yv.z, xv.w - yv.w);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (kern == KDE_KERN_LAPLACIAN) {
          acc[u] = (fabsf(diff[u].x) + fabsf(diff[u].y)) + (fabsf(diff[u].z) + fabsf(diff[u].w));
        } else {
          float t = diff[u].x * diff[u].x;
          t = fmaf(diff[u].y, diff[u].y, t);
          t = fmaf(diff[u].z, diff[u].z, t);
          acc[u] = fmaf(diff[u].w, diff[u].w, t);
        }
      }
      float v4[4], v2[2], dist;
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
        dist = keep + __shfl_xor_sync(0xffffffffu, send, 4);
      }
      dist += __shfl_xor_sync(0xffffffffu, dist, 2);
      dist += __shfl_xor_sync(0xffffffffu, dist, 1);
      const float K = kernel_from_dist(kern, dist, inv);
      float gs, sv;
      if (kern == KDE_KERN_GAUSSIAN) {
        gs = 1.f / (h * h);
        sv = dist / (h * h);
      } else if (kern == KDE_KERN_EXPONENTIAL) {
        const float r = sqrtf(fmaxf(dist, 0.f));
        gs = r > 0.f ? 1.f / (h * r) : 0.f;
        sv = r / h;
      } else {
        gs = 1.f / h;
        sv = dist / h;
      }
      const float wk = wb + myrow < cnt ? w * K : 0.f;
      if ((lane & 3) == 0) {
        est += wk;
        sl += wk * sv;
      }
      const float coef = wk * gs;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float c = __shfl_sync(0xffffffffu, coef, ((u >> 2) << 4) | (((u >> 1) & 1) << 3) | ((u & 1) << 2));
        const float4 df = diff[u];
        if (kern == KDE_KERN_LAPLACIAN) {
          gacc[0].x += c * (df.x > 0.f ? 1.f : (df.x < 0.f ? -1.f : 0.f));
          gacc[0].y += c * (df.y > 0.f ? 1.f : (df.y < 0.f ? -1.f : 0.f));
          gacc[0].z += c * (df.z > 0.f ? 1.f : (df.z < 0.f ? -1.f : 0.f));
          gacc[0].w += c * (df.w > 0.f ? 1.f : (df.w < 0.f ? -1.f : 0.f));
        } else {
          gacc[0].x = fmaf(c, df.x, gacc[0].x);
          gacc[0].y = fmaf(c, df.y, gacc[0].y);
          gacc[0].z = fmaf(c, df.z, gacc[0].z);
          gacc[0].w = fmaf(c, df.w, gacc[0].w);
        }
      }
    }
    return;
  }
  // warp-uniform trip count (group reductions need all lanes)
  for (int wb = warp * kGpw; wb < cnt; wb += kNW * kGpw) {
    const int r = wb + gw;
    const bool valid = r < cnt;
    const float4* row =
        valid ? reinterpret_cast<const float4*>(X + (int64_t)ids[r] * dp) : nullptr;
    float4 diff[NV];
    float dist = 0.f;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int j4 = lig + v * G;
      if (valid && j4 < dp4) {
        const float4 xv = __ldg(row + j4), yv = y4[j4];
        diff[v] = make_float4(xv.x - yv.x, xv.y - yv.y, xv.z - yv.z, xv.w - yv.w);
      } else {
        diff[v] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (kern == KDE_KERN_LAPLACIAN) {
        dist += (fabsf(diff[v].x) + fabsf(diff[v].y)) + (fabsf(diff[v].z) + fabsf(diff[v].w));
      } else {
        dist = fmaf(diff[v].x, diff[v].x, dist);
        dist = fmaf(diff[v].y, diff[v].y, dist);
        dist = fmaf(diff[v].z, diff[v].z, dist);
        dist = fmaf(diff[v].w, diff[v].w, dist);
      }
    }
    dist = group_sum<G>(dist);
    const float K = kernel_from_dist(kern, dist, inv);
    float gs, s;  // per-component factor and d/dlog h factor
    if (kern == KDE_KERN_GAUSSIAN) {
      gs = 1.f / (h * h);
      s = dist / (h * h);
    } else if (kern == KDE_KERN_EXPONENTIAL) {
      const float r = sqrtf(fmaxf(dist, 0.f));
      gs = r > 0.f ? 1.f / (h * r) : 0.f;
      s = r / h;
    } else {
      gs = 1.f / h;
      s = dist / h;
    }
    const float wk = valid ? w * K : 0.f;
    if (lig == 0) {
      est += wk;
      sl += wk * s;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (kern == KDE_KERN_LAPLACIAN) {
        gacc[v].x += wk * gs * (diff[v].x > 0.f ? 1.f : (diff[v].x < 0.f ? -1.f : 0.f));
        gacc[v].y += wk * gs * (diff[v].y > 0.f ? 1.f : (diff[v].y < 0.f ? -1.f : 0.f));
        gacc[v].z += wk * gs * (diff[v].z > 0.f ? 1.f : (diff[v].z < 0.f ? -1.f : 0.f));
        gacc[v].w += wk * gs * (diff[v].w > 0.f ? 1.f : (diff[v].w < 0.f ? -1.f : 0.f));
      } else {
        gacc[v].x = fmaf(wk * gs, diff[v].x, gacc[v].x);
        gacc[v].y = fmaf(wk * gs, diff[v].y, gacc[v].y);
        gacc[v].z = fmaf(wk * gs, diff[v].z, gacc[v].z);
        gacc[v].w = fmaf(wk * gs, diff[v].w, gacc[v].w);
      }
    }
  }
}

template <int G, int NV>
__global__ void __launch_bounds__(kNT) k_estimate_grad(SampleArgs a) {
  __shared__ EstSmem sm;
  __shared__ int tmp[kMaxK];
  extern __shared__ float4 dyn4[];
  float* ys = reinterpret_cast<float*>(dyn4);
  float* gpart = ys + a.dp;  // [kNT / G][dp]: each lane group's partial gradient
  int* hs = reinterpret_cast<int*>(gpart + (size_t)(kNT / G) * a.dp);  // [kHashSlots]
  const int64_t q = blockIdx.x;
  const int tid = threadIdx.x;
  const uint64_t qid = a.qid_offset + (a.dev_qid != nullptr ? *a.dev_qid : 0ull) + (uint64_t)q;
  for (int j = tid; j < a.dp; j += kNT) ys[j] = a.Y[q * a.dp + j];
  const int k = a.rs ? 0 : a.k;
  // Rejection mode outside held-out fitting: X_1 in a hash set for the draws'
  // membership tests, and its rows taken in the row's own order (no sort) when
  // no id repeats; with a repeated id the sorted, deduplicated array is built
  // instead (the order of the X_1 rows fixes the gradient's summation order).
  bool use_hash = false;
  int k1h = 0;
  if (k > 0 && a.mode == 0 && !a.loo) {
    const int32_t* row = a.nbr + q * a.k;
    load_neighbours_hash(row, k, a.n, sm, hs);
    use_hash = sm.dup == 0;
    if (use_hash && !sm.status) {
      const int lane = tid & 31, warp = tid >> 5;
      for (int b0 = 0; b0 < k; b0 += kNT) {  // the valid ids in row order
        const int i = b0 + tid;
        const int32_t id = i < k ? row[i] : -1;
        const bool keep = id >= 0;
        const unsigned mk = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) sm.warp_cnt[warp] = __popc(mk);
        __syncthreads();
        int off = k1h, tot = 0;
        for (int w = 0; w < kNW; ++w) {
          if (w < warp) off += sm.warp_cnt[w];
          tot += sm.warp_cnt[w];
        }
        if (keep) tmp[off + __popc(mk & ((1u << lane) - 1u))] = id;
        k1h += tot;
        __syncthreads();
      }
    } else if (!sm.status) {
      load_neighbours(row, k, a.n, sm, tmp);
    }
  } else if (k > 0) {
    load_neighbours(a.nbr + q * a.k, k, a.n, sm, tmp);
  } else {
    if (tid == 0) {
      sm.kk = 0;
      sm.status = 0;
    }
    __syncthreads();
  }
  if (sm.status) {
    if (tid == 0) {
      atomicOr(a.err, KDE_ERRBIT_BADNBR);
      if (a.out) a.out[q] = __int_as_float(0x7fc00000);
    }
    return;
  }
  const int kk = sm.kk;
  const double nd = (double)a.n;
  const bool sampled = !((int64_t)kk == a.n || a.m == 0);
  float4 gacc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) gacc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  float est = 0.f, sl = 0.f;
  // Held-out mode: the row's first id z is the query point itself.  The
  // estimate is of KDE over X \ {z} at z: z stays in X_1 (never sampled) but
  // its own term is left out, and the weights use n - 1 points.
  const double nw = a.loo ? nd - 1.0 : nd;
  const int* rows1 = use_hash ? tmp : sm.nb;
  int k1 = use_hash ? k1h : kk;
  if (a.loo && k > 0) {
    const int32_t z = a.nbr[q * a.k];
    int w = 0;
    if (tid == 0) {
      for (int t = 0; t < kk; ++t)
        if (sm.nb[t] != z) tmp[w++] = sm.nb[t];
      sm.cnt = w;
    }
    __syncthreads();
    rows1 = tmp;
    k1 = sm.cnt;
    __syncthreads();
  }
  const float w1 = a.rs ? 0.f : (float)(1.0 / nw);
  if (k1 > 0) grad_rows<G, NV>(a.X, a.dp, ys, rows1, k1, a.kern, a.h, w1, gacc, est, sl);
  bool ok = true;
  if (sampled) {
    const float w2 = a.rs ? (float)(1.0 / (double)a.m)
                     : a.mode == 1 ? (float)(nd / (nw * (double)a.m))
                                   : (float)((nd - (double)kk) / (nw * (double)a.m));
    const int64_t cap = a.mode == 1 ? (int64_t)a.m : 64 * (int64_t)a.m + 4096;
    int64_t t0 = 0;
    int got = 0;
    while (got < a.m) {
      const int room = min(kChunk, a.m - got);
      if (!draw_chunk(a.seed, qid, (uint64_t)a.n, t0, cap, room, a.mode, sm, sm,
                      use_hash ? hs : nullptr)) {
        ok = false;
        break;
      }
      const int cnt = sm.cnt;
      t0 = sm.tnext;
      if (a.mode == 1) {
        __syncthreads();
        if (tid == 0) {
          int w = 0;
          for (int i = 0; i < cnt; ++i)
            if (!is_member(sm.nb, kk, sm.S[i])) sm.S[w++] = sm.S[i];
          sm.cnt = w;
        }
        __syncthreads();
      }
      grad_rows<G, NV>(a.X, a.dp, ys, sm.S, sm.cnt, a.kern, a.h, w2, gacc, est, sl);
      got += cnt;
      __syncthreads();
    }
  }
  // combine the groups' d-vectors in a fixed order (group 0 first), so that
  // the gradient is the same bits on every run
  const int lig = tid & (G - 1);
  const int dp4 = a.dp >> 2;
  float4* mine = reinterpret_cast<float4*>(gpart + (size_t)(tid / G) * a.dp);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int j4 = lig + v * G;
    if (j4 < dp4) mine[j4] = gacc[v];
  }
  const float est_t = block_sum(est, sm);
  const float sl_t = block_sum(sl, sm);
  __syncthreads();
  const float go = a.gout ? a.gout[q] : 1.f;
  if (!ok) {
    if (tid == 0) {
      atomicOr(a.err, KDE_ERRBIT_DRAWCAP);
      if (a.out) a.out[q] = __int_as_float(0x7fc00000);
      if (a.dlogh) a.dlogh[q] = __int_as_float(0x7fc00000);
    }
    for (int j = tid; j < a.d; j += kNT) a.dY[q * a.d + j] = __int_as_float(0x7fc00000);
    return;
  }
  for (int j = tid; j < a.d; j += kNT) {
    float g = 0.f;
    for (int grp = 0; grp < kNT / G; ++grp) g += gpart[(size_t)grp * a.dp + j];
    a.dY[q * a.d + j] = go * g;
  }
  if (tid == 0) {
    if (a.out) a.out[q] = est_t;
    if (a.dlogh) a.dlogh[q] = go * sl_t;
  }
}

// One Gaussian mean-shift step with the estimated density: the fixed point
// of y = sum_i w_i K_i x_i / sum_i w_i K_i is reached by
// y <- y + h^2 grad(est)(y) / est(y) (grad = sum_i w_i K_i (x_i - y) / h^2).
__global__ void k_mean_shift_update(float* __restrict__ Yp, int dp, int d,
                                    const float* __restrict__ dY, const float* __restrict__ est,
                                    int64_t nq, float h2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * d) return;
  const int64_t q = i / d;
  const int j = (int)(i - q * d);
  const float e = est[q];
  if (e > 0.f) Yp[q * dp + j] += h2 * dY[i] / e;
}

int group_lanes(int dp) {
  const int dp4 = dp / 4;
  if (dp4 <= 4) return 4;
  if (dp4 <= 8) return 8;
  if (dp4 <= 16) return 16;
  return 32;
}

}  // namespace

template <int G>
void launch_estimate_inst(const SampleArgs& a, size_t dyn, cudaStream_t s) {
  // the query row in dynamic shared memory: past 48 KB with the static part
  // (37 KB) for rows wider than 2,048 floats, which needs the opt-in
  if (dyn > 8192) set_dynamic_smem(reinterpret_cast<const void*>(&k_estimate<G>), dyn);
  k_estimate<G><<<(unsigned)a.nq, kNT, dyn, s>>>(a);
}

void launch_estimate(const SampleArgs& a, cudaStream_t s) {
  if (a.nq <= 0) return;
  const size_t dyn = sizeof(float) * a.dp;
  switch (group_lanes(a.dp)) {
    case 4: launch_estimate_inst<4>(a, dyn, s); break;
    case 8: launch_estimate_inst<8>(a, dyn, s); break;
    case 16: launch_estimate_inst<16>(a, dyn, s); break;
    default: launch_estimate_inst<32>(a, dyn, s); break;
  }
}

PhasePlan phase_plan(int64_t n, int dp, int m, int64_t nq, int64_t window_bytes) {
  PhasePlan pl;
  // the plan depends on the index and on m, not on the batch size (short of
  // the grid limit), so a query gets the same bits in any batch
  if (window_bytes <= 0 || n <= 0 || m <= 0 || m > kPhasedMaxM) return pl;
  // W: the largest power of two whose rows fit the window (a shift, not a
  // division, maps a row id to its window)
  const int64_t row_bytes = (int64_t)dp * (int64_t)sizeof(float);
  if (n * row_bytes <= window_bytes) return pl;  // X fits one window
  const int64_t rows = std::max<int64_t>(1, window_bytes / row_bytes);
  int sh = 0;
  while (sh < 30 && (int64_t(2) << sh) <= rows) ++sh;
  const int64_t P = (n + (int64_t(1) << sh) - 1) >> sh;
  // one window: every draw hits the same one, as in the per-query gathers
  if (P < 2 || P > kMaxPhases || P * nq > INT32_MAX) return pl;
  if ((int64_t)m < kMinPhaseRows * P) return pl;
  pl.P = (int)P;
  pl.shift = sh;
  return pl;
}

template <int G>
void launch_gather_phase(const SampleArgs& a, const PhaseArgs& ph, cudaStream_t s) {
  k_gather_phase<G><<<(unsigned)((int64_t)ph.P * a.nq), kNT, 0, s>>>(a, ph);
}

void launch_estimate_phased(const SampleArgs& a, const PhaseArgs& ph, cudaStream_t s) {
  if (a.nq <= 0) return;
  const size_t dyn = sizeof(int) * ((size_t)a.m + (size_t)kNW * ph.P);
  set_dynamic_smem(reinterpret_cast<const void*>(&k_draw_phased), dyn);
  k_draw_phased<<<(unsigned)a.nq, kNT, dyn, s>>>(a, ph);
  // the rows come from L2 and the gathers are issue-bound: 8 lanes a row
  // (four rows a warp instruction) reduce with a fifth of the shuffles and
  // id loads of 32 lanes a row
  if (group_lanes(a.dp) == 4) launch_gather_phase<4>(a, ph, s);
  else launch_gather_phase<8>(a, ph, s);
  k_phase_finish<<<(unsigned)((a.nq + 255) / 256), 256, 0, s>>>(a, ph);
}

void launch_window_prep(const SampleArgs& a, int32_t* drops, int dstride, int32_t* dcnt,
                        int32_t* kk, float* s1, cudaStream_t s) {
  if (a.nq <= 0) return;
  const size_t dyn = sizeof(float) * a.dp;
  const unsigned grid = (unsigned)a.nq;
  switch (group_lanes(a.dp)) {
    case 4: k_window_prep<4><<<grid, kNT, dyn, s>>>(a, drops, dstride, dcnt, kk, s1); break;
    case 8: k_window_prep<8><<<grid, kNT, dyn, s>>>(a, drops, dstride, dcnt, kk, s1); break;
    case 16: k_window_prep<16><<<grid, kNT, dyn, s>>>(a, drops, dstride, dcnt, kk, s1); break;
    default: k_window_prep<32><<<grid, kNT, dyn, s>>>(a, drops, dstride, dcnt, kk, s1); break;
  }
}

void launch_window_finish(const SampleArgs& a, const WindowPlan& p, const int32_t* dcnt,
                          const int32_t* kk, const float* s1, const double* part,
                          cudaStream_t s) {
  if (a.nq <= 0) return;
  k_window_finish<<<(unsigned)((a.nq + 255) / 256), 256, 0, s>>>(a.nq, a.n, a.m, p.nslices,
                                                                  dcnt, kk, s1, part, a.out);
}

namespace {
// Row j of X_1 for bandwidth fitting: the training point itself, then its k
// search neighbours (a repeat of the point counts once).
__global__ void k_prepend_self(const int32_t* __restrict__ zid, const int32_t* __restrict__ nbr,
                               int64_t nz, int k, int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t w = (int64_t)k + 1;
  if (i >= nz * w) return;
  const int64_t j = i / w, c = i % w;
  out[i] = c == 0 ? zid[j] : nbr[j * k + (c - 1)];
}

// Leave-one-out sums over the training points, in a fixed order (one CTA):
// red[0] = sum log KDE_{-z}, red[1] = sum dKDE_{-z}/dlog h / KDE_{-z},
// red[2] = points used; loo[j] is the held-out estimate at z_j, dloo[j] its
// derivative.  A point with no held-out density (loo <= 0: every other kernel
// value underflowed) is left out.
// out[0] = sum_i v[i], FP64 partial sums in a fixed order (thread t takes
// i = t, t + 1024, ...; then a tree over the 1024 partials), rounded once, so
// that the result does not depend on the launch or the device.
__global__ void __launch_bounds__(1024) k_sum_to_scalar(const float* __restrict__ v, int64_t n,
                                                        float* __restrict__ out) {
  __shared__ double part[1024];
  const int tid = threadIdx.x;
  double a = 0.0;
  for (int64_t i = tid; i < n; i += 1024) a += (double)v[i];
  part[tid] = a;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (tid < o) part[tid] += part[tid + o];
    __syncthreads();
  }
  if (tid == 0) out[0] = (float)part[0];
}

__global__ void __launch_bounds__(1024) k_loo_reduce(const float* __restrict__ loo,
                                                     const float* __restrict__ dloo, int64_t nz,
                                                     double* __restrict__ red) {
  __shared__ double s0[1024], s1[1024], s2[1024];
  const int tid = threadIdx.x;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int64_t j = tid; j < nz; j += 1024) {
    const double v = (double)loo[j];
    if (!(v > 0.0)) continue;
    a += log(v);
    b += (double)dloo[j] / v;
    c += 1.0;
  }
  s0[tid] = a;
  s1[tid] = b;
  s2[tid] = c;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (tid < o) {
      s0[tid] += s0[tid + o];
      s1[tid] += s1[tid + o];
      s2[tid] += s2[tid + o];
    }
    __syncthreads();
  }
  if (tid == 0) {
    red[0] = s0[0];
    red[1] = s1[0];
    red[2] = s2[0];
  }
}
}  // namespace

void launch_prepend_self(const int32_t* zid, const int32_t* nbr, int64_t nz, int k, int32_t* out,
                         cudaStream_t s) {
  const int64_t total = nz * ((int64_t)k + 1);
  if (total <= 0) return;
  k_prepend_self<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(zid, nbr, nz, k, out);
}

void launch_loo_reduce(const float* loo, const float* dloo, int64_t nz, double* red,
                       cudaStream_t s) {
  k_loo_reduce<<<1, 1024, 0, s>>>(loo, dloo, nz, red);
}

void launch_sum_to_scalar(const float* v, int64_t n, float* out, cudaStream_t s) {
  k_sum_to_scalar<<<1, 1024, 0, s>>>(v, n, out);
}

void launch_mean_shift_update(float* Yp, int dp, int d, const float* dY, const float* est,
                              int64_t nq, float h, cudaStream_t s) {
  const int64_t total = nq * d;
  if (total <= 0) return;
  k_mean_shift_update<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Yp, dp, d, dY, est, nq,
                                                                      h * h);
}

// static shared memory plus the partial gradients can pass the 48 KB default
// (d = 1024: 65 KB), so the limit is raised per launch
template <int G, int NV>
void launch_grad_inst(const SampleArgs& a, unsigned grid, size_t dyn, cudaStream_t s) {
  set_dynamic_smem(reinterpret_cast<const void*>(&k_estimate_grad<G, NV>), dyn);
  k_estimate_grad<G, NV><<<grid, kNT, dyn, s>>>(a);
}

void launch_estimate_grad(const SampleArgs& a, cudaStream_t s) {
  if (a.nq <= 0) return;
  const unsigned grid = (unsigned)a.nq;
  const int G = group_lanes(a.dp);
  // the staged query, one partial gradient per lane group (<= 36 KB at d = 1024)
  // and the hash set of X_1
  const size_t dyn = sizeof(float) * (size_t)a.dp * (1 + kNT / G) + sizeof(int) * kHashSlots;
  const int dp4 = a.dp / 4;
  if (G < 32) {  // d <= 64: shorter lane groups (measured faster than the warp-wide path)
    switch (G) {
      case 4: launch_grad_inst<4, 1>(a, grid, dyn, s); break;
      case 8: launch_grad_inst<8, 1>(a, grid, dyn, s); break;
      default: launch_grad_inst<16, 1>(a, grid, dyn, s); break;
    }
    return;
  }
  const int nv = (dp4 + 31) / 32;
  if (nv <= 1) launch_grad_inst<32, 1>(a, grid, dyn, s);
  else if (nv <= 2) launch_grad_inst<32, 2>(a, grid, dyn, s);
  else if (nv <= 4) launch_grad_inst<32, 4>(a, grid, dyn, s);
  else launch_grad_inst<32, 8>(a, grid, dyn, s);
}

}  // namespace deann
