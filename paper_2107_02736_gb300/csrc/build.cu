// Index build: row layout, norms, k-means (Lloyd iterations) and the
// list-contiguous IVF layout (paper Section 4: the inverted file runs k-means
// and stores every point in the list of its nearest centroid).
//
// Every step is deterministic: initial centroids are distinct points drawn
// from Philox stream 1, assignments break ties to the lower centroid id, the
// list layout is a stable counting sort (points keep their original order
// within a list), centroid sums run over the list in that order in FP64, and
// an empty list is reseeded with the point farthest from its centroid.
#include <cuda_bf16.h>

#include "common.cuh"

namespace deann {

namespace {

__global__ void k_pad_rows(const float* __restrict__ src, int64_t n, int d,
                           float* __restrict__ dst, int dp) {
  const int64_t total = n * dp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / dp;
    const int j = (int)(i - r * dp);
    dst[i] = j < d ? src[r * d + j] : 0.f;
  }
}

__global__ void k_row_norms(const float* __restrict__ X, int64_t n, int dp,
                            float* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  float s = 0.f;
  for (int j = lane; j < dp; j += 32) {
    const float v = X[r * dp + j];
    s = fmaf(v, v, s);
  }
  s = warp_sum(s);
  if (lane == 0) out[r] = s;
}

// One thread: L distinct points by rejection of repeats (stream 1, qid 0).
__global__ void k_kmeans_init(int64_t n, int L, uint64_t seed, uint32_t* __restrict__ bitmap,
                              int32_t* __restrict__ chosen, uint32_t* __restrict__ err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t t = 0;
  const uint32_t cap = 64u * (uint32_t)L + 4096u;
  for (int c = 0; c < L; ++c) {
    for (;;) {
      if (t >= cap) {
        atomicOr(err, KDE_ERRBIT_DRAWCAP);
        chosen[c] = c % (int)n;
        break;
      }
      const int64_t id = draw_index(seed, 0, t++, 1u, (uint64_t)n);
      const uint32_t w = bitmap[id >> 5], b = 1u << (id & 31);
      if (!(w & b)) {
        bitmap[id >> 5] = w | b;
        chosen[c] = (int32_t)id;
        break;
      }
    }
  }
}

__global__ void k_gather_rows(const float* __restrict__ X, int dp, const int32_t* __restrict__ ids,
                              int64_t count, float* __restrict__ dst) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (r >= count) return;
  const float4* s = reinterpret_cast<const float4*>(X + (int64_t)ids[r] * dp);
  float4* o = reinterpret_cast<float4*>(dst + r * dp);
  for (int j = lane; j < dp / 4; j += 32) o[j] = s[j];
}

__global__ void k_gather_f32(const float* __restrict__ v, const int32_t* __restrict__ ids,
                             int64_t count, float* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = v[ids[i]];
}

__global__ void k_list_hist(const int32_t* __restrict__ assign, int64_t n,
                            unsigned long long* __restrict__ counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(counts + assign[i], 1ull);
}

constexpr int kScatterChunk = 2048;

// chunk_hist[l * nchunks + c] = points of chunk c assigned to list l
__global__ void k_chunk_hist(const int32_t* __restrict__ assign, int64_t n, int L,
                             int64_t nchunks, int64_t* __restrict__ chunk_hist) {
  extern __shared__ int hist[];
  const int64_t c = blockIdx.x;
  for (int l = threadIdx.x; l < L; l += blockDim.x) hist[l] = 0;
  __syncthreads();
  const int64_t b = c * kScatterChunk, e = min(n, b + kScatterChunk);
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) atomicAdd(&hist[assign[i]], 1);
  __syncthreads();
  for (int l = threadIdx.x; l < L; l += blockDim.x) chunk_hist[(int64_t)l * nchunks + c] = hist[l];
}

// One warp per list: running offsets of each chunk's first point in the list.
__global__ void k_chunk_offsets(const int64_t* __restrict__ list_off, int L, int64_t nchunks,
                                int64_t* __restrict__ chunk_hist) {
  const int l = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (l >= L) return;
  int64_t base = list_off[l];
  int64_t* row = chunk_hist + (int64_t)l * nchunks;
  for (int64_t c0 = 0; c0 < nchunks; c0 += 32) {
    const int64_t c = c0 + lane;
    const int64_t v = c < nchunks ? row[c] : 0;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (c < nchunks) row[c] = base + incl - v;
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
}

// One warp per chunk, points in order, 32 at a time: stable positions.
__global__ void k_chunk_scatter(const int32_t* __restrict__ assign, int64_t n, int64_t nchunks,
                                int64_t* __restrict__ chunk_off, int32_t* __restrict__ perm) {
  const int64_t c = blockIdx.x;
  const int lane = threadIdx.x;
  const int64_t b = c * kScatterChunk, e = min(n, b + kScatterChunk);
  for (int64_t i0 = b; i0 < e; i0 += 32) {
    const int64_t i = i0 + lane;
    const bool valid = i < e;
    const int l = valid ? assign[i] : -1 - lane;  // invalid lanes never match
    const unsigned peers = __match_any_sync(0xffffffffu, l);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int64_t* slot = chunk_off + (int64_t)(valid ? l : 0) * nchunks + c;
    const int64_t start = valid ? *slot : 0;
    if (valid) perm[start + rank] = (int32_t)i;
    __syncwarp();
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) *slot = start + __popc(peers);
    __syncwarp();
  }
}

// Centroid = FP64 mean of the list's points in list order; empty -> flag.
__global__ void k_centroid_update(const float* __restrict__ X, int dp,
                                  const int32_t* __restrict__ perm,
                                  const int64_t* __restrict__ list_off, float* __restrict__ C,
                                  int32_t* __restrict__ empty_flags) {
  const int l = blockIdx.x;
  const int64_t b = list_off[l], e = list_off[l + 1];
  if (e == b) {
    if (threadIdx.x == 0) empty_flags[l] = 1;
    return;
  }
  if (threadIdx.x == 0) empty_flags[l] = 0;
  const double inv = 1.0 / (double)(e - b);
  for (int j = threadIdx.x; j < dp; j += blockDim.x) {
    double s = 0.0;
    for (int64_t p = b; p < e; ++p) s += (double)X[(int64_t)perm[p] * dp + j];
    C[(int64_t)l * dp + j] = (float)(s * inv);
  }
}

// Empty lists in increasing order each take the point farthest from its
// centroid (ties to the lower id); a taken point is not reused.
__global__ void __launch_bounds__(1024) k_reseed_empty(const float* __restrict__ X, int64_t n,
                                                       int dp, float* __restrict__ d2,
                                                       const int32_t* __restrict__ empty_flags,
                                                       int L, float* __restrict__ C) {
  __shared__ float sb[32];
  __shared__ int64_t si[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int any = 0;
  for (int l = tid; l < L; l += 1024) any |= empty_flags[l];
  if (!__syncthreads_or(any)) return;  // the usual case: no empty list
  for (int l = 0; l < L; ++l) {
    if (!empty_flags[l]) continue;
    float best = -1.f;
    int64_t arg = n;
    for (int64_t i = tid; i < n; i += 1024) {
      const float v = d2[i];
      if (v > best) {
        best = v;
        arg = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int64_t oa = __shfl_xor_sync(0xffffffffu, arg, o);
      if (ob > best || (ob == best && oa < arg)) {
        best = ob;
        arg = oa;
      }
    }
    if (lane == 0) {
      sb[warp] = best;
      si[warp] = arg;
    }
    __syncthreads();
    if (warp == 0) {
      best = sb[lane];
      arg = si[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int64_t oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa < arg)) {
          best = ob;
          arg = oa;
        }
      }
      if (lane == 0) si[0] = arg;
    }
    __syncthreads();
    const int64_t pick = si[0];
    if (pick < n) {
      for (int j = tid; j < dp; j += 1024) C[(int64_t)l * dp + j] = X[pick * dp + j];
      if (tid == 0) d2[pick] = -2.f;
    }
    __syncthreads();
  }
}

__global__ void k_to_bf16(const float* __restrict__ X, int64_t n, int dp,
                          __nv_bfloat16* __restrict__ dst, int dpb) {
  const int64_t total = n * dpb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / dpb;
    const int j = (int)(i - r * dpb);
    dst[i] = __float2bfloat16_rn(j < dp ? X[r * dp + j] : 0.f);
  }
}

// BF16 copy of the list-ordered rows centred on their list's centroid,
// x~ = x - c_l, with FP32 squared norms |x~|^2 and the list radius
// max |x~| (one block per list, one warp per row).
__global__ void k_center_bf16(const float* __restrict__ XL, int dp,
                              const int64_t* __restrict__ list_off, const float* __restrict__ C,
                              __nv_bfloat16* __restrict__ dst, int dpb, float* __restrict__ xcn,
                              float* __restrict__ rad) {
  const int l = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t b = list_off[l], e = list_off[l + 1];
  const float* c = C + (int64_t)l * dp;
  float rmax = 0.f;
  for (int64_t r = b + warp; r < e; r += nw) {
    float s = 0.f;
    for (int j = lane; j < dpb; j += 32) {
      const float v = j < dp ? XL[r * dp + j] - c[j] : 0.f;
      dst[r * dpb + j] = __float2bfloat16_rn(v);
      s = fmaf(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) {
      xcn[r] = s;
      rmax = fmaxf(rmax, sqrtf(s));
    }
  }
  __shared__ float red[32];
  if (lane == 0) red[warp] = rmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < nw; ++w) m = fmaxf(m, red[w]);
    rad[l] = m;
  }
}

// The centred rows x~ = x - c_l of each list split into three BF16 parts,
// x~ = p0 + p1 + p2 up to 2^-27 |x~| (p0 = bf16(x~), p1 = bf16(x~ - p0),
// p2 = bf16(x~ - p0 - p1); each difference is exact in FP32): part p of the
// list-order row r at dst[(p n + r) dpb + j].  |x~|^2 is summed in FP64 and
// rounded once.  One block per list, one warp per row.
__global__ void k_center_split3(const float* __restrict__ XL, int dp, int64_t n,
                                const int64_t* __restrict__ list_off, const float* __restrict__ C,
                                __nv_bfloat16* __restrict__ dst, int dpb,
                                float* __restrict__ xsn) {
  const int l = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t b = list_off[l], e = list_off[l + 1];
  const float* c = C + (int64_t)l * dp;
  for (int64_t r = b + warp; r < e; r += nw) {
    double s = 0.0;
    for (int j = lane; j < dpb; j += 32) {
      const float v = j < dp ? XL[r * dp + j] - c[j] : 0.f;
      const __nv_bfloat16 p0 = __float2bfloat16_rn(v);
      const float r1 = v - __bfloat162float(p0);
      const __nv_bfloat16 p1 = __float2bfloat16_rn(r1);
      const __nv_bfloat16 p2 = __float2bfloat16_rn(r1 - __bfloat162float(p1));
      dst[(0 * n + r) * dpb + j] = p0;
      dst[(1 * n + r) * dpb + j] = p1;
      dst[(2 * n + r) * dpb + j] = p2;
      s += (double)v * (double)v;
    }
    s = warp_sum_d(s);
    if (lane == 0) xsn[r] = (float)s;
  }
}

__global__ void k_fill_i32(int32_t* __restrict__ p, int64_t count, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

unsigned grid_for(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 152 * 64) g = 152 * 64;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

void launch_pad_rows(const float* src, int64_t n, int d, float* dst, int dp, cudaStream_t s) {
  k_pad_rows<<<grid_for(n * dp, 256), 256, 0, s>>>(src, n, d, dst, dp);
}

void launch_row_norms(const float* X, int64_t n, int dp, float* out, cudaStream_t s) {
  if (n <= 0) return;
  k_row_norms<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(X, n, dp, out);
}

void launch_kmeans_init(const float* X, int64_t n, int dp, int L, uint64_t seed,
                        uint32_t* bitmap, int32_t* chosen, float* C, uint32_t* err, cudaStream_t s) {
  cudaMemsetAsync(bitmap, 0, sizeof(uint32_t) * ((n + 31) / 32), s);
  k_kmeans_init<<<1, 32, 0, s>>>(n, L, seed, bitmap, chosen, err);
  k_gather_rows<<<(unsigned)((L + 7) / 8), 256, 0, s>>>(X, dp, chosen, L, C);
}

void launch_list_hist(const int32_t* assign, int64_t n, int L, int64_t* counts, cudaStream_t s) {
  cudaMemsetAsync(counts, 0, sizeof(int64_t) * L, s);
  k_list_hist<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      assign, n, reinterpret_cast<unsigned long long*>(counts));
}

void launch_stable_scatter(const int32_t* assign, int64_t n, int L, const int64_t* list_off,
                           int64_t* chunk_hist, int32_t* perm, cudaStream_t s) {
  const int64_t nchunks = (n + kScatterChunk - 1) / kScatterChunk;
  k_chunk_hist<<<(unsigned)nchunks, 256, sizeof(int) * L, s>>>(assign, n, L, nchunks, chunk_hist);
  k_chunk_offsets<<<(unsigned)((L + 7) / 8), 256, 0, s>>>(list_off, L, nchunks, chunk_hist);
  k_chunk_scatter<<<(unsigned)nchunks, 32, 0, s>>>(assign, n, nchunks, chunk_hist, perm);
}

void launch_centroid_update(const float* X, int dp, const int32_t* perm, const int64_t* list_off,
                            int L, float* C, int32_t* empty_flags, cudaStream_t s) {
  k_centroid_update<<<(unsigned)L, 128, 0, s>>>(X, dp, perm, list_off, C, empty_flags);
}

void launch_reseed_empty(const float* X, int64_t n, int dp, const float* best_d2,
                         int32_t* empty_flags, int L, float* C, float* tmp_d2, cudaStream_t s) {
  cudaMemcpyAsync(tmp_d2, best_d2, sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
  k_reseed_empty<<<1, 1024, 0, s>>>(X, n, dp, tmp_d2, empty_flags, L, C);
}

void launch_gather_rows(const float* X, int dp, const int32_t* ids, int64_t count, float* dst,
                        cudaStream_t s) {
  if (count <= 0) return;
  k_gather_rows<<<(unsigned)((count + 7) / 8), 256, 0, s>>>(X, dp, ids, count, dst);
}

void launch_gather_f32(const float* v, const int32_t* ids, int64_t count, float* dst,
                       cudaStream_t s) {
  if (count <= 0) return;
  k_gather_f32<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(v, ids, count, dst);
}

void launch_to_bf16(const float* X, int64_t n, int dp, void* dst, int dpb, cudaStream_t s) {
  k_to_bf16<<<grid_for(n * dpb, 256), 256, 0, s>>>(X, n, dp,
                                                   reinterpret_cast<__nv_bfloat16*>(dst), dpb);
}

void launch_center_bf16(const float* XL, int dp, const int64_t* list_off, int L, const float* C,
                        void* dst, int dpb, float* xcn, float* rad, cudaStream_t s) {
  k_center_bf16<<<(unsigned)L, 256, 0, s>>>(XL, dp, list_off, C,
                                            reinterpret_cast<__nv_bfloat16*>(dst), dpb, xcn, rad);
}

void launch_center_split3(const float* XL, int dp, int64_t n, const int64_t* list_off, int L,
                          const float* C, void* dst, int dpb, float* xsn, cudaStream_t s) {
  k_center_split3<<<(unsigned)L, 256, 0, s>>>(XL, dp, n, list_off, C,
                                              reinterpret_cast<__nv_bfloat16*>(dst), dpb, xsn);
}

void launch_fill_i32(int32_t* p, int64_t count, int32_t v, cudaStream_t s) {
  if (count <= 0) return;
  k_fill_i32<<<grid_for(count, 256), 256, 0, s>>>(p, count, v);
}

namespace {
// max of nonnegative floats through their order-preserving bit patterns
__global__ void k_max_f32(const float* __restrict__ v, int64_t n, unsigned* __restrict__ out) {
  unsigned best = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    best = max(best, dist_key(v[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}
}  // namespace

namespace {
// Algorithm 2's preprocessing permutation pi of [0, n): a 4-round balanced
// Feistel network on 2 hb bits (2^(2 hb) >= n) keyed by the index seed, its
// round function the word r0 of Philox4x32-10 at counter (R, round, 0, 3);
// values >= n are re-enciphered until they fall in [0, n) (cycle walking,
// Black and Rogaway, CT-RSA 2002).  The walk stays on the cycle of i under a
// bijection of [0, 2^(2 hb)), which contains i < n, so it ends after fewer
// than 2^(2 hb) - n + 2 passes (expected at most 4).
__device__ __forceinline__ uint32_t feistel_once(uint32_t x, int hb, uint32_t mask,
                                                 uint64_t seed) {
  uint32_t L = x >> hb, R = x & mask;
#pragma unroll
  for (uint32_t r = 0; r < 4; ++r) {
    const uint4 o = Philox::block(make_uint4(R, r, 0u, 3u), (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
    const uint32_t nR = L ^ (o.x & mask);
    L = R;
    R = nR;
  }
  return (L << hb) | R;
}

__global__ void k_feistel_perm(uint64_t seed, int64_t n, int hb, int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t mask = (1u << hb) - 1u;
  uint32_t x = (uint32_t)i;
  do {
    x = feistel_once(x, hb, mask, seed);
  } while ((int64_t)x >= n);
  out[i] = (int32_t)x;
}
}  // namespace

void launch_feistel_perm(uint64_t seed, int64_t n, int32_t* out, cudaStream_t s) {
  if (n <= 0) return;
  int bits = 1;
  while (((int64_t)1 << bits) < n) ++bits;  // n < 2^31, so bits <= 31 and 2 hb <= 32
  const int hb = (bits + 1) / 2;
  k_feistel_perm<<<grid_for(n, 256), 256, 0, s>>>(seed, n, hb, out);
}

namespace {
__global__ void k_invert_perm(const int32_t* __restrict__ perm, int64_t n,
                              int32_t* __restrict__ inv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) inv[perm[i]] = (int32_t)i;
}
}  // namespace

void launch_invert_perm(const int32_t* perm, int64_t n, int32_t* inv, cudaStream_t s) {
  if (n <= 0) return;
  k_invert_perm<<<grid_for(n, 256), 256, 0, s>>>(perm, n, inv);
}

void launch_max_f32(const float* v, int64_t n, float* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(float), s);
  k_max_f32<<<grid_for(n, 256), 256, 0, s>>>(v, n, reinterpret_cast<unsigned*>(out));
}

}  // namespace deann
