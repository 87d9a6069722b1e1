// SIMT distance tiles (CUDA cores, FP32): the exact-KDE baseline, the k-means
// assignment and the approximate distance matrices of the IVF coarse step and
// list scan.
//
// One CTA of 256 threads computes a 64 x 64 block of row-pair results; each
// thread owns a 4 x 4 sub-block.  Dimensions are consumed in chunks of 32,
// staged transposed in shared memory and prefetched into registers one chunk
// ahead.  Three accumulation modes:
//   DOT  : <a, b>            (Appendix D: D^2 = |a|^2 + |b|^2 - 2 <a, b>)
//   SQ   : sum (a_j - b_j)^2 (difference form, the FP32-accurate path)
//   ABS  : sum |a_j - b_j|   (L1 distance for the Laplacian kernel)
// Difference-form sums are two-level (a partial per 32-dim chunk, then added),
// which keeps the rounding error near sqrt(32) + sqrt(d/32) units of 2^-24.
#include "common.cuh"

namespace deann {

namespace {

constexpr int kKC = 32;        // dims per chunk
constexpr int kLd = kTile + 4; // shared row stride (floats), keeps float4 alignment

enum { MODE_DOT = 0, MODE_SQ = 1, MODE_ABS = 2 };

struct TileSmem {
  float A[kKC][kLd];
  float B[kKC][kLd];
};

__device__ __forceinline__ float4 ld4(const float* p, int k, int dp) {
  if (p != nullptr && k < dp) return *reinterpret_cast<const float4*>(p + k);
  return make_float4(0.f, 0.f, 0.f, 0.f);
}

// Computes acc[i][j] for A rows (ty*4+i) and B rows (tx*4+j) of the tile.
// aptr[s] / bptr[s] are the global rows this thread stages (slot s = 0, 1);
// a null pointer stages zeros.
template <int MODE>
__device__ __forceinline__ void tile_mainloop(const float* const (&aptr)[2],
                                              const float* const (&bptr)[2], int dp,
                                              TileSmem& sm, float (&acc)[4][4]) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  int srow[2], sc4[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int idx = tid + 256 * s;
    srow[s] = idx >> 3;
    sc4[s] = idx & 7;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  float4 ra[2], rb[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    ra[s] = ld4(aptr[s], 4 * sc4[s], dp);
    rb[s] = ld4(bptr[s], 4 * sc4[s], dp);
  }
  for (int k0 = 0; k0 < dp; k0 += kKC) {
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int r = srow[s], c = 4 * sc4[s];
      sm.A[c + 0][r] = ra[s].x;
      sm.A[c + 1][r] = ra[s].y;
      sm.A[c + 2][r] = ra[s].z;
      sm.A[c + 3][r] = ra[s].w;
      sm.B[c + 0][r] = rb[s].x;
      sm.B[c + 1][r] = rb[s].y;
      sm.B[c + 2][r] = rb[s].z;
      sm.B[c + 3][r] = rb[s].w;
    }
    __syncthreads();
    // prefetch the next chunk while this one is consumed
    const int kn = k0 + kKC;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      ra[s] = ld4(aptr[s], kn + 4 * sc4[s], dp);
      rb[s] = ld4(bptr[s], kn + 4 * sc4[s], dp);
    }
    float part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = 0.f;
#pragma unroll 8
    for (int kk = 0; kk < kKC; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&sm.A[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&sm.B[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (MODE == MODE_DOT) {
            part[i][j] = fmaf(av[i], bv[j], part[i][j]);
          } else if (MODE == MODE_SQ) {
            const float t = av[i] - bv[j];
            part[i][j] = fmaf(t, t, part[i][j]);
          } else {
            part[i][j] += fabsf(av[i] - bv[j]);
          }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += part[i][j];
  }
}

// --------------------------------------------------------------------------
// Exact KDE (paper Section 2 definition; Appendix D's "Naive" evaluation with
// the distance matrix never leaving the chip).  grid.x: 64-query tiles;
// grid.y: contiguous slices of X.  Per-row partial sums meet in FP64 atomics.
// --------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_exact_simt(const float* __restrict__ Y, int64_t nq,
                                                    const float* __restrict__ X, int64_t n,
                                                    int dp, int kern, float inv,
                                                    int64_t rows_per_slice,
                                                    double* __restrict__ acc_out) {
  __shared__ TileSmem sm;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t q0 = (int64_t)blockIdx.x * kTile;
  const int64_t x_begin = (int64_t)blockIdx.y * rows_per_slice;
  const int64_t x_end = min(n, x_begin + rows_per_slice);
  const float* aptr[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int64_t q = q0 + ((tid + 256 * s) >> 3);
    aptr[s] = q < nq ? Y + q * dp : nullptr;
  }
  // per-tile partials in FP32 (4 terms), running sums in FP64
  double rowsum[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t x0 = x_begin; x0 < x_end; x0 += kTile) {
    const float* bptr[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int64_t r = x0 + ((tid + 256 * s) >> 3);
      bptr[s] = r < x_end ? X + r * dp : nullptr;
    }
    float acc[4][4];
    tile_mainloop<MODE>(aptr, bptr, dp, sm, acc);
    float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (x0 + tx * 4 + j < x_end) {
#pragma unroll
        for (int i = 0; i < 4; ++i) part[i] += kernel_from_dist(kern, acc[i][j], inv);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) rowsum[i] += (double)part[i];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double v = rowsum[i];
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    const int64_t q = q0 + ty * 4 + i;
    if (tx == 0 && q < nq) atomicAdd(acc_out + q, v);
  }
}

__global__ void k_exact_finish(const double* __restrict__ acc, int64_t nq, double inv_n,
                               float* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nq) out[q] = (float)(acc[q] * inv_n);
}

// --------------------------------------------------------------------------
// k-means assignment: nearest centroid of each point (difference form), ties
// to the lower centroid id.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_assign_simt(const float* __restrict__ P, int64_t np,
                                                     const float* __restrict__ C, int L, int dp,
                                                     int32_t* __restrict__ assign,
                                                     float* __restrict__ best_d2) {
  __shared__ TileSmem sm;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t p0 = (int64_t)blockIdx.x * kTile;
  const float* aptr[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int64_t p = p0 + ((tid + 256 * s) >> 3);
    aptr[s] = p < np ? P + p * dp : nullptr;
  }
  float best[4];
  int arg[4];
  // arg starts at centroid 0 so that even non-finite distances give a valid id
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    best[i] = __int_as_float(0x7f800000);
    arg[i] = 0;
  }
  for (int c0 = 0; c0 < L; c0 += kTile) {
    const float* bptr[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int c = c0 + ((tid + 256 * s) >> 3);
      bptr[s] = c < L ? C + (int64_t)c * dp : nullptr;
    }
    float acc[4][4];
    tile_mainloop<MODE_SQ>(aptr, bptr, dp, sm, acc);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      if (c < L) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (acc[i][j] < best[i]) {  // increasing c: strict < keeps the lower id
            best[i] = acc[i][j];
            arg[i] = c;
          }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float b = best[i];
    int a = arg[i];
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, b, o);
      const int oa = __shfl_xor_sync(0xffffffffu, a, o);
      if (ob < b || (ob == b && oa < a)) {
        b = ob;
        a = oa;
      }
    }
    const int64_t p = p0 + ty * 4 + i;
    if (tx == 0 && p < np) {
      assign[p] = a;
      if (best_d2) best_d2[p] = b;
    }
  }
}

// --------------------------------------------------------------------------
// Approximate distance matrix D[q][c] = |y|^2 + |c|^2 - 2 <y, c> (IVF coarse
// quantiser; candidates are rescored exactly afterwards).
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dist_matrix(const float* __restrict__ Y,
                                                     const float* __restrict__ Yn, int64_t nq,
                                                     const float* __restrict__ C,
                                                     const float* __restrict__ Cn, int L, int dp,
                                                     float* __restrict__ D,
                                                     const int64_t* __restrict__ active,
                                                     int64_t row0) {
  __shared__ TileSmem sm;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t q0 = (int64_t)blockIdx.x * kTile;
  const int c0 = blockIdx.y * kTile;
  // rows at or past the device row count get no probes: no distances needed
  if (active != nullptr && row0 + q0 >= *active) return;
  const float* aptr[2];
  const float* bptr[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int64_t q = q0 + ((tid + 256 * s) >> 3);
    aptr[s] = q < nq ? Y + q * dp : nullptr;
    const int c = c0 + ((tid + 256 * s) >> 3);
    bptr[s] = c < L ? C + (int64_t)c * dp : nullptr;
  }
  float acc[4][4];
  tile_mainloop<MODE_DOT>(aptr, bptr, dp, sm, acc);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t q = q0 + ty * 4 + i;
    if (q >= nq) continue;
    const float yn = Yn[q];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      if (c < L) D[q * L + c] = fmaxf(yn + Cn[c] - 2.f * acc[i][j], 0.f);
    }
  }
}

// --------------------------------------------------------------------------
// IVF list scan, list-major: tile t covers up to 64 (query, probe) pairs that
// probe the same list; the CTA streams the list's points in 64-row tiles and
// writes the approximate squared distances into each pair's segment of the
// per-query candidate buffer.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scan_simt(
    const float* __restrict__ Y, const float* __restrict__ Yn, const float* __restrict__ XL,
    const float* __restrict__ XLn, const int64_t* __restrict__ list_off, int L, int dp,
    const int32_t* __restrict__ pair_q, const int64_t* __restrict__ pair_dst,
    const int64_t* __restrict__ bucket_off, const int64_t* __restrict__ tile_off,
    const int32_t* __restrict__ lorder, float* __restrict__ cand) {
  __shared__ TileSmem sm;
  __shared__ int s_list, s_pos;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t t = blockIdx.x;
  if (t >= tile_off[L]) return;
  if (tid == 0) {
    int lo = 0, hi = L - 1;  // last place i in the scan order with tile_off[i] <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    s_pos = lo;
    s_list = lorder[lo];
  }
  __syncthreads();
  const int l = s_list;
  const int64_t pb = bucket_off[l] + (t - tile_off[s_pos]) * kTile;
  const int64_t pe = min(bucket_off[l + 1], pb + kTile);
  const int64_t xb = list_off[l], xe = list_off[l + 1];
  const float* aptr[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int64_t p = pb + ((tid + 256 * s) >> 3);
    aptr[s] = p < pe ? Y + (int64_t)pair_q[p] * dp : nullptr;
  }
  float yn[4];
  int64_t dst[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t p = pb + ty * 4 + i;
    dst[i] = p < pe ? pair_dst[p] : -1;
    yn[i] = p < pe ? Yn[pair_q[p]] : 0.f;
  }
  for (int64_t x0 = xb; x0 < xe; x0 += kTile) {
    const float* bptr[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int64_t r = x0 + ((tid + 256 * s) >> 3);
      bptr[s] = r < xe ? XL + r * dp : nullptr;
    }
    float acc[4][4];
    tile_mainloop<MODE_DOT>(aptr, bptr, dp, sm, acc);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t r = x0 + tx * 4 + j;
      if (r >= xe) {
        // the segment's padding to 32 floats holds +inf
        if (r - xb < ((xe - xb + 31) & ~(int64_t)31)) {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (dst[i] >= 0) cand[dst[i] + (r - xb)] = __int_as_float(0x7f800000);
        }
        continue;
      }
      const float xn = XLn[r];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (dst[i] >= 0) cand[dst[i] + (r - xb)] = fmaxf(yn[i] + xn - 2.f * acc[i][j], 0.f);
    }
  }
}

}  // namespace

void launch_exact_simt(const float* Y, const float* Yn, int64_t nq, const float* X,
                       const float* Xn, int64_t n, int d, int dp, int kern, float h,
                       double* acc, float* out, cudaStream_t s) {
  (void)Yn;
  (void)Xn;
  (void)d;
  cudaMemsetAsync(acc, 0, sizeof(double) * nq, s);
  const int64_t qtiles = (nq + kTile - 1) / kTile;
  // enough CTAs to fill 152 SMs several times over; slices are multiples of 64 rows
  int64_t want = (152 * 8 + qtiles - 1) / qtiles;
  int64_t ntile_x = (n + kTile - 1) / kTile;
  int64_t slices = want < 1 ? 1 : (want > ntile_x ? ntile_x : want);
  if (slices > 65535) slices = 65535;
  const int64_t rows_per_slice = ((ntile_x + slices - 1) / slices) * kTile;
  slices = (n + rows_per_slice - 1) / rows_per_slice;
  dim3 grid((unsigned)qtiles, (unsigned)slices);
  const float inv = kernel_inv(kern, h);
  if (kern == KDE_KERN_LAPLACIAN)
    k_exact_simt<MODE_ABS><<<grid, 256, 0, s>>>(Y, nq, X, n, dp, kern, inv, rows_per_slice, acc);
  else
    k_exact_simt<MODE_SQ><<<grid, 256, 0, s>>>(Y, nq, X, n, dp, kern, inv, rows_per_slice, acc);
  k_exact_finish<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(acc, nq, 1.0 / (double)n, out);
}

void launch_assign_simt(const float* P, int64_t np, const float* C, int L, int d, int dp,
                        int32_t* assign, float* best_d2, cudaStream_t s) {
  (void)d;
  k_assign_simt<<<(unsigned)((np + kTile - 1) / kTile), 256, 0, s>>>(P, np, C, L, dp, assign,
                                                                     best_d2);
}

void launch_dist_matrix(const float* Y, const float* Yn, int64_t nq, const float* C,
                        const float* Cn, int L, int dp, float* D, const int64_t* active,
                        int64_t row0, cudaStream_t s) {
  dim3 grid((unsigned)((nq + kTile - 1) / kTile), (unsigned)((L + kTile - 1) / kTile));
  k_dist_matrix<<<grid, 256, 0, s>>>(Y, Yn, nq, C, Cn, L, dp, D, active, row0);
}

void launch_scan_simt(const float* Y, const float* Yn, const float* XL, const float* XLn,
                      const int64_t* list_off, int L, int dp, const ScanPlan& plan, float* cand,
                      cudaStream_t s) {
  if (plan.max_tiles <= 0) return;
  k_scan_simt<<<(unsigned)plan.max_tiles, 256, 0, s>>>(Y, Yn, XL, XLn, list_off, L, dp,
                                                       plan.pair_q, plan.pair_dst,
                                                       plan.bucket_off, plan.tile_off,
                                                       plan.lorder, cand);
}

}  // namespace deann
