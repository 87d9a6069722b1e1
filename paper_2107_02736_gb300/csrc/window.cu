// Permuted-window estimator (Algorithm 2) as dense tiles.
//
// The query with global id qid reads the window of m consecutive rows of the
// permuted dataset XP starting at (qid m) mod n.  Ids that agree mod
// P = n / gcd(n, m) give the same window, so a batch of nq queries holds
// about nq / P queries per window.  When that share is large the window sums
// form a dense (queries x window rows) block per residue class, and one CTA
// computes a 64-query x 64-row tile of it from shared memory: each window row
// is read from memory once per 64 queries instead of once per query.
//
// Distances are the FP32 difference form sum_j (y_j - x_j)^2 (L1 for the
// Laplacian kernel), with the same two-level chunked summation as the other
// SIMT tiles.  The squared form runs on Blackwell's packed FP32 pairs
// (sub.rn.f32x2 / fma.rn.f32x2: two round-to-nearest lanes, each result equal
// to the scalar instruction's).  Window entries that are members of X_1 are
// masked per (query, row) from each query's sorted list of their window
// positions; every CTA writes one FP64 partial per query and row slice, and a
// separate pass adds them in slice order, so results are deterministic.
#include "common.cuh"

namespace deann {

namespace {

constexpr int kKC = 32;            // dims per staged chunk of window rows
constexpr int kResMaxDp = 320;     // query tile resident in shared memory up to this width

enum { WMODE_SQ = 0, WMODE_ABS = 1 };

// Shared layouts, both XOR-swizzled on 16-byte groups so that the transposed
// staging stores and the fragment reads are free of bank conflicts:
//   queries A[dim][64]: query r of dim c at ((r >> 2) ^ sw(c)) * 4 + (r & 3);
//   rows B[dim][128]: every value twice; rows 4t, 4t + 1 of dim c fill group
//     t ^ sw(c) as (x, x, x', x'), rows 4t + 2, 4t + 3 group (16 + t) ^ sw(c).
__device__ __forceinline__ int sw(int c) { return (c >> 2) & 7; }
__device__ __forceinline__ int acol(int r, int c) { return (((r >> 2) ^ sw(c)) << 2) + (r & 3); }
__device__ __forceinline__ int bcol(int r, int c) {
  const int g = ((r & 2) ? 16 : 0) + (r >> 2);
  return ((g ^ sw(c)) << 2) + 2 * (r & 1);
}

struct alignas(16) WinSmem {
  float A[kKC][kTile];             // streamed query chunk (wide rows only)
  float B[kKC][2 * kTile];         // window rows of the current chunk
  uint64_t mask[2][kTile];         // per query slot: X_1 members among the tile's rows
};

__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

__device__ __forceinline__ float4 ld4(const float* p, int k, int dp) {
  if (p != nullptr && k < dp) return *reinterpret_cast<const float4*>(p + k);
  return make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ void store_a(float* A, int r, int c, float4 v) {
  A[(c + 0) * kTile + acol(r, c + 0)] = v.x;
  A[(c + 1) * kTile + acol(r, c + 1)] = v.y;
  A[(c + 2) * kTile + acol(r, c + 2)] = v.z;
  A[(c + 3) * kTile + acol(r, c + 3)] = v.w;
}

__device__ __forceinline__ void store_b(WinSmem& sm, int r, int c, float4 v) {
  *reinterpret_cast<float2*>(&sm.B[c + 0][bcol(r, c + 0)]) = make_float2(v.x, v.x);
  *reinterpret_cast<float2*>(&sm.B[c + 1][bcol(r, c + 1)]) = make_float2(v.y, v.y);
  *reinterpret_cast<float2*>(&sm.B[c + 2][bcol(r, c + 2)]) = make_float2(v.z, v.z);
  *reinterpret_cast<float2*>(&sm.B[c + 3][bcol(r, c + 3)]) = make_float2(v.w, v.w);
}

// acc[i][j]: distance between query slot ty*4+i and row slot tx*4+j.  RES:
// the queries sit in Ares[dp][64] for the CTA's lifetime; otherwise they are
// streamed chunk by chunk with the rows.
template <int MODE, bool RES>
__device__ __forceinline__ void win_mainloop(const float* const (&aptr)[2],
                                             const float* const (&bptr)[2], int dp,
                                             WinSmem& sm, const float* Ares,
                                             float (&acc)[4][4]) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  int srow[2], sc4[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int idx = tid + 256 * s;
    srow[s] = idx >> 3;
    sc4[s] = idx & 7;
  }
  uint64_t accp[2][4];  // packed (query 2p, query 2p + 1) x row j
  float accs[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    accp[0][j] = 0ull;
    accp[1][j] = 0ull;
#pragma unroll
    for (int i = 0; i < 4; ++i) accs[i][j] = 0.f;
  }
  float4 ra[2], rb[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    if (!RES) ra[s] = ld4(aptr[s], 4 * sc4[s], dp);
    rb[s] = ld4(bptr[s], 4 * sc4[s], dp);
  }
  for (int k0 = 0; k0 < dp; k0 += kKC) {
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (!RES) store_a(&sm.A[0][0], srow[s], 4 * sc4[s], ra[s]);
      store_b(sm, srow[s], 4 * sc4[s], rb[s]);
    }
    __syncthreads();
    const int kn = k0 + kKC;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (!RES) ra[s] = ld4(aptr[s], kn + 4 * sc4[s], dp);
      rb[s] = ld4(bptr[s], kn + 4 * sc4[s], dp);
    }
    const float* Ab = RES ? Ares + (size_t)k0 * kTile : &sm.A[0][0];
    if (MODE == WMODE_SQ) {
      uint64_t part[2][4];
#pragma unroll
      for (int j = 0; j < 4; ++j) part[0][j] = part[1][j] = 0ull;
#pragma unroll 8
      for (int kk = 0; kk < kKC; ++kk) {
        const int z = sw(kk);  // k0 is a multiple of 32: sw(k0 + kk) = sw(kk)
        const ulonglong2 a =
            *reinterpret_cast<const ulonglong2*>(Ab + kk * kTile + ((ty ^ z) << 2));
        const ulonglong2 b01 = *reinterpret_cast<const ulonglong2*>(&sm.B[kk][(tx ^ z) << 2]);
        const ulonglong2 b23 =
            *reinterpret_cast<const ulonglong2*>(&sm.B[kk][((16 + tx) ^ z) << 2]);
        const uint64_t av[2] = {a.x, a.y};
        const uint64_t bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint64_t t = f2_sub(av[p], bv[j]);
            part[p][j] = f2_fma(t, t, part[p][j]);
          }
      }
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int j = 0; j < 4; ++j) accp[p][j] = f2_add(accp[p][j], part[p][j]);
    } else {
      float part[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] = 0.f;
#pragma unroll 8
      for (int kk = 0; kk < kKC; ++kk) {
        const int z = sw(kk);
        const float4 a = *reinterpret_cast<const float4*>(Ab + kk * kTile + ((ty ^ z) << 2));
        const float4 b01 = *reinterpret_cast<const float4*>(&sm.B[kk][(tx ^ z) << 2]);
        const float4 b23 = *reinterpret_cast<const float4*>(&sm.B[kk][((16 + tx) ^ z) << 2]);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[4] = {b01.x, b01.z, b23.x, b23.z};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) part[i][j] += fabsf(av[i] - bv[j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) accs[i][j] += part[i][j];
    }
  }
  if (MODE == WMODE_SQ) {
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 v = f2_unpack(accp[p][j]);
        acc[2 * p][j] = v.x;
        acc[2 * p + 1][j] = v.y;
      }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = accs[i][j];
  }
}

// grid.x: (residue class s, 64-query tile of its queries); grid.y: slices of
// p.rs window positions.  Class s holds queries s, s + P, s + 2P, ... < nq.
template <int MODE, bool RES>
__global__ void __launch_bounds__(256, RES ? 3 : 2) k_window_tile(WindowTileArgs w) {
  __shared__ WinSmem sm;
  extern __shared__ float4 ares4[];  // RES: the query tile, [roundup(dp, 32)][64] swizzled
  float* Ares = reinterpret_cast<float*>(ares4);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const WindowPlan& p = w.p;
  const int64_t s = blockIdx.x / p.Tq;
  const int64_t j0 = (int64_t)(blockIdx.x % p.Tq) * kTile;
  const int64_t cs = s < p.B ? p.A + 1 : p.A;
  if (j0 >= cs) return;  // uniform over the CTA
  const uint64_t qid_s = w.qid_offset + (w.dev_qid != nullptr ? *w.dev_qid : 0ull) + (uint64_t)s;
  const int64_t w0 =
      (int64_t)(((qid_s % (uint64_t)w.n) * (uint64_t)w.m) % (uint64_t)w.n);
  const int64_t r0 = (int64_t)blockIdx.y * p.rs;
  const int64_t r1 = min((int64_t)w.m, r0 + (int64_t)p.rs);

  const float* aptr[2];
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
    const int64_t jj = j0 + ((tid + 256 * s2) >> 3);
    aptr[s2] = jj < cs ? w.Y + (s + jj * p.P) * w.dp : nullptr;
  }
  if (RES) {
    for (int k0 = 0; k0 < w.dp; k0 += kKC)
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2) {
        const int idx = tid + 256 * s2;
        const int c = k0 + 4 * (idx & 7);
        store_a(Ares, idx >> 3, c, ld4(aptr[s2], c, w.dp));
      }
  }
  // query slot tid (< 64): cursor into its sorted X_1 window positions
  const int32_t* dl = nullptr;
  int dc = 0, cur = 0;
  if (tid < kTile && j0 + tid < cs) {
    const int64_t q = s + (j0 + tid) * p.P;
    dl = w.drops + q * w.dstride;
    dc = w.dcnt[q];
    int lo = 0, hi = dc;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((int64_t)dl[mid] < r0) lo = mid + 1; else hi = mid;
    }
    cur = lo;
  }
  const float inv = kernel_inv(w.kern, w.h);
  double rowsum[4] = {0.0, 0.0, 0.0, 0.0};
  int buf = 0;
  for (int64_t x0 = r0; x0 < r1; x0 += kTile, buf ^= 1) {
    if (tid < kTile) {
      uint64_t mm = 0ull;
      while (cur < dc && (int64_t)dl[cur] < x0 + kTile) {
        mm |= 1ull << (int)((int64_t)dl[cur] - x0);
        ++cur;
      }
      sm.mask[buf][tid] = mm;
    }
    const float* bptr[2];
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const int64_t pos = x0 + ((tid + 256 * s2) >> 3);
      if (pos < r1) {
        int64_t j = w0 + pos;  // w0 < n and pos < m <= n
        if (j >= w.n) j -= w.n;
        bptr[s2] = w.XP + j * w.dp;
      } else {
        bptr[s2] = nullptr;
      }
    }
    float acc[4][4];
    win_mainloop<MODE, RES>(aptr, bptr, w.dp, sm, Ares, acc);  // starts with a barrier
    float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (x0 + tx * 4 + j < r1) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (((sm.mask[buf][ty * 4 + i] >> (tx * 4 + j)) & 1ull) == 0ull)
            part[i] += kernel_from_dist(w.kern, acc[i][j], inv);
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
    const int64_t jj = j0 + ty * 4 + i;
    if (tx == 0 && jj < cs) w.part[(s + jj * p.P) * p.nslices + blockIdx.y] = v;
  }
}

}  // namespace

int64_t window_period(int64_t n, int64_t m) {
  int64_t g = n, r = m;  // gcd(n, m); m = 0 gives n
  while (r != 0) {
    const int64_t t = g % r;
    g = r;
    r = t;
  }
  return n / g;
}

WindowPlan window_plan(int64_t nq, int64_t n, int m) {
  WindowPlan p;
  p.P = window_period(n, m);
  p.A = nq / p.P;
  p.B = nq % p.P;
  p.groups = std::min<int64_t>(p.P, nq);
  const int64_t biggest = p.A + (p.B > 0 ? 1 : 0);
  p.Tq = (int)((biggest + kTile - 1) / kTile);
  // about 2048 CTAs: several waves of 152 SMs with a few CTAs resident each
  const int64_t cols = std::max<int64_t>(1, p.groups * p.Tq);
  const int64_t tiles = std::max<int64_t>(1, ((int64_t)m + kTile - 1) / kTile);
  int64_t slices = std::min<int64_t>(tiles, std::max<int64_t>(1, (2048 + cols - 1) / cols));
  int64_t per = (tiles + slices - 1) / slices;
  while ((tiles + per - 1) / per > 65535) ++per;
  p.rs = (int)(per * kTile);
  p.nslices = (int)((tiles + per - 1) / per);
  return p;
}

bool window_tiled(const WindowPlan& p) { return p.A >= kWindowMinShare; }

void launch_window_tile(const WindowTileArgs& w, cudaStream_t s) {
  if (w.p.groups <= 0 || w.m <= 0) return;
  dim3 grid((unsigned)(w.p.groups * w.p.Tq), (unsigned)w.p.nslices);
  const bool res = w.dp <= kResMaxDp;
  // the resident tile is staged in whole 32-dim chunks: round its rows up
  const int dres = (w.dp + kKC - 1) / kKC * kKC;
  const size_t dyn = res ? sizeof(float) * (size_t)dres * kTile : 0;
  if (res) {
    // the resident query tile takes up to 80 KB beside the static 25 KB
    auto f0 = k_window_tile<WMODE_SQ, true>;
    auto f1 = k_window_tile<WMODE_ABS, true>;
    set_dynamic_smem(reinterpret_cast<const void*>(w.kern == KDE_KERN_LAPLACIAN ? f1 : f0), dyn);
    if (w.kern == KDE_KERN_LAPLACIAN)
      f1<<<grid, 256, dyn, s>>>(w);
    else
      f0<<<grid, 256, dyn, s>>>(w);
  } else if (w.kern == KDE_KERN_LAPLACIAN) {
    k_window_tile<WMODE_ABS, false><<<grid, 256, 0, s>>>(w);
  } else {
    k_window_tile<WMODE_SQ, false><<<grid, 256, 0, s>>>(w);
  }
}

}  // namespace deann
