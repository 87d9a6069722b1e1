// Device-side helpers shared by the DEANN kernels (sm_103a).
//
// Kernel functions (paper Section 1): Gaussian exp(-r^2 / (2 h^2)),
// exponential exp(-r / h), Laplacian exp(-|x - y|_1 / h); all map into [0, 1]
// with no normalising constant, so a KDE value lies in [0, 1].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace deann {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32
// multiplies whose high and low halves are permuted and XOR-ed with the other
// counter words and the round key; the key advances by the Weyl increments
// between rounds.
// ---------------------------------------------------------------------------
struct Philox {
  static constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
  static constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
  __device__ __forceinline__ static uint4 block(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      if (r) {
        k0 += kW0;
        k1 += kW1;
      }
      const uint32_t hi0 = __umulhi(kM0, c.x), lo0 = kM0 * c.x;
      const uint32_t hi1 = __umulhi(kM1, c.z), lo1 = kM1 * c.z;
      c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
  }
};

// Draw t of query qid's stream: counter (t, lo(qid), hi(qid), stream), key
// (lo(seed), hi(seed)); u = (r1 << 32) | r0; index = floor(u * n / 2^64).
__device__ __forceinline__ int64_t draw_index(uint64_t seed, uint64_t qid, uint32_t t,
                                              uint32_t stream, uint64_t n) {
  const uint4 r = Philox::block(make_uint4(t, (uint32_t)qid, (uint32_t)(qid >> 32), stream),
                                (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t u = ((uint64_t)r.y << 32) | (uint64_t)r.x;
  return (int64_t)__umul64hi(u, n);
}

// ---------------------------------------------------------------------------
// Kernel value from the squared Euclidean distance (Gaussian, exponential) or
// from the L1 distance (Laplacian).  `inv` is 1/(2h^2) for the Gaussian and
// 1/h otherwise.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float kernel_from_dist(int kern, float dist, float inv) {
  if (kern == KDE_KERN_GAUSSIAN) return expf(-fmaxf(dist, 0.f) * inv);
  if (kern == KDE_KERN_EXPONENTIAL) return expf(-sqrtf(fmaxf(dist, 0.f)) * inv);
  return expf(-fmaxf(dist, 0.f) * inv);
}

__host__ __device__ __forceinline__ float kernel_inv(int kern, float h) {
  return kern == KDE_KERN_GAUSSIAN ? 1.0f / (2.0f * h * h) : 1.0f / h;
}

// ---------------------------------------------------------------------------
// Warp / block reductions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over groups of G consecutive lanes (G a power of two <= 32).
template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Error-free sum a + b = s + e (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Requests the 128-byte line holding p into L2 (a hint: no register waits
// for it, and no fault is raised for it).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Nonnegative float -> order-preserving uint32 (NaN treated as +inf).
__device__ __forceinline__ uint32_t dist_key(float v) {
  if (!(v >= 0.f)) v = (v < 0.f) ? 0.f : __int_as_float(0x7f800000);
  return __float_as_uint(v);
}

// (distance, id) as one 64-bit key whose unsigned order is the (distance,
// id) lexicographic order.
__device__ __forceinline__ unsigned long long pack_key(float d2, int id) {
  return ((unsigned long long)dist_key(d2) << 32) | (unsigned)id;
}

// Distance of one row pair computed by G lanes cooperatively, in difference
// form with compensated summation: each lane splits x - y into an FP32 value
// and its exact rounding error (TwoSum), accumulates the squares with their
// FMA-exact error terms, and the lane partials are combined with TwoSum.
// Relative error ~ a few units of 2^-24, independent of d.
template <int G>
__device__ __forceinline__ float precise_sq_dist(const float* __restrict__ x,
                                                 const float* __restrict__ y, int d,
                                                 int lane_in_group) {
  float hi = 0.f, lo = 0.f;
#pragma unroll 4
  for (int j = lane_in_group; j < d; j += G) {
    float diff, derr;
    two_sum(x[j], -y[j], diff, derr);
    const float sq = diff * diff;
    const float sq_err = fmaf(diff, diff, -sq) + 2.f * diff * derr;
    float s, e;
    two_sum(hi, sq, s, e);
    hi = s;
    lo += e + sq_err;
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
    const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, ohi, s, e);
    hi = s;
    lo += olo + e;
  }
  return hi + lo;
}

// Plain FP32 difference-form squared distance by G lanes: each lane sums
// ceil(d/G) squares with FMA, then a log2(G)-level tree.  Relative error at
// most (ceil(d/G) + log2(G) + 2) units of 2^-24.
template <int G>
__device__ __forceinline__ float plain_sq_dist(const float* __restrict__ x,
                                               const float* __restrict__ y, int d,
                                               int lane_in_group) {
  float s = 0.f;
#pragma unroll 4
  for (int j = lane_in_group; j < d; j += G) {
    const float t = x[j] - y[j];
    s = fmaf(t, t, s);
  }
  return group_sum<G>(s);
}

// Same for the L1 distance (Laplacian kernel).
template <int G>
__device__ __forceinline__ float precise_l1_dist(const float* __restrict__ x,
                                                 const float* __restrict__ y, int d,
                                                 int lane_in_group) {
  float hi = 0.f, lo = 0.f;
  for (int j = lane_in_group; j < d; j += G) {
    float diff, derr;
    two_sum(x[j], -y[j], diff, derr);
    const float a = fabsf(diff);
    const float aerr = diff >= 0.f ? derr : -derr;
    float s, e;
    two_sum(hi, a, s, e);
    hi = s;
    lo += e + aerr;
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
    const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, ohi, s, e);
    hi = s;
    lo += olo + e;
  }
  return hi + lo;
}

}  // namespace deann
