/*
 * FP64 CPU oracle for the DEANN kernel-density estimator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may build, load or call it.  It shares
 * no code, header, table or helper with the CUDA library, and the CUDA library
 * never calls it.
 *
 * Paper: Karppa, Aumueller, Pagh, "DEANN: Speeding up Kernel-Density
 * Estimation using Approximate Nearest Neighbor Search" (arXiv 2107.02736).
 *
 * Every distance here is computed in difference form, sum_j (x_j - y_j)^2 (or
 * sum_j |x_j - y_j| for the Laplacian kernel), in FP64, from FP32 inputs
 * promoted to FP64.  Sums run in a fixed, documented order.  Parallelism is
 * over queries only (OpenMP when the compiler offers it); every query's
 * arithmetic is sequential, so the result does not depend on the thread count.
 *
 * Every function is pinned by tests/test_oracle_pins.py against values and
 * properties fixed outside this file (published known answers, closed forms,
 * library routines, brute force, invariants).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_GAUSSIAN 0
#define OR_EXPONENTIAL 1
#define OR_LAPLACIAN 2

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ELIMIT 4

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ------------------------------------------------------------------------
 * Philox4x32-10, written from its definition in Salmon, Moraes, Dror, Shaw,
 * "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11), Section 3.3:
 * a 4-word counter and a 2-word key; each of the 10 rounds multiplies words 0
 * and 2 by two fixed odd constants, swaps the halves of the 64-bit products
 * into place and XORs in the other counter words and the round key; the key
 * is advanced by the two Weyl increments between rounds.
 * ---------------------------------------------------------------------- */
static const uint32_t PHILOX_MUL0 = 0xD2511F53u;
static const uint32_t PHILOX_MUL1 = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL0 = 0x9E3779B9u;
static const uint32_t PHILOX_WEYL1 = 0xBB67AE85u;

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_WEYL0;
      k1 += PHILOX_WEYL1;
    }
    uint64_t p0 = (uint64_t)PHILOX_MUL0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)PHILOX_MUL1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Draw number t of query qid's stream: the uniform index in [0, n) that the
 * estimator's random sample uses (Algorithm 1; Lemma RS samples with
 * repetition).  key = (lo32(seed), hi32(seed)); counter = (t, lo32(qid),
 * hi32(qid), stream).  u = (r1 << 32) | r0 and index = floor(u * n / 2^64),
 * the exact high word of the 128-bit product. */
int64_t or_draw_index(uint64_t seed, uint64_t qid, uint32_t t, uint32_t stream,
                      int64_t n) {
  uint32_t ctr[4] = {t, (uint32_t)qid, (uint32_t)(qid >> 32), stream};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  or_philox4x32_10(ctr, key, r);
  uint64_t u = ((uint64_t)r[1] << 32) | (uint64_t)r[0];
  unsigned __int128 prod = (unsigned __int128)u * (unsigned __int128)(uint64_t)n;
  return (int64_t)(uint64_t)(prod >> 64);
}

/* ------------------------------------------------------------------------
 * Kernels (Section 1: Gaussian, Eq. "gaussiankernel"; exponential and
 * Laplacian named right after it).  K_h maps into [0, 1]: no normalising
 * constant.
 * ---------------------------------------------------------------------- */
static double sq_dist(const float* x, const float* y, int d) {
  double s = 0.0;
  for (int j = 0; j < d; ++j) {
    double t = (double)x[j] - (double)y[j];
    s += t * t;
  }
  return s;
}

static double l1_dist(const float* x, const float* y, int d) {
  double s = 0.0;
  for (int j = 0; j < d; ++j) s += fabs((double)x[j] - (double)y[j]);
  return s;
}

double or_kernel_value(int kern, const float* x, const float* y, int d,
                       double h) {
  if (kern == OR_GAUSSIAN) return exp(-sq_dist(x, y, d) / (2.0 * h * h));
  if (kern == OR_EXPONENTIAL) return exp(-sqrt(sq_dist(x, y, d)) / h);
  return exp(-l1_dist(x, y, d) / h);
}

/* Kernel value together with the two derivative factors used by the adjoint:
 * g (so that dK/dy = K * g) and s (so that dK/dlog h = K * s). */
static double kernel_and_derivs(int kern, const float* x, const float* y, int d,
                                double h, double* g /* d or NULL */,
                                double* s) {
  if (kern == OR_GAUSSIAN) {
    double r2 = sq_dist(x, y, d);
    double k = exp(-r2 / (2.0 * h * h));
    if (g)
      for (int j = 0; j < d; ++j) g[j] = ((double)x[j] - (double)y[j]) / (h * h);
    *s = r2 / (h * h);
    return k;
  }
  if (kern == OR_EXPONENTIAL) {
    double r = sqrt(sq_dist(x, y, d));
    double k = exp(-r / h);
    if (g)
      for (int j = 0; j < d; ++j)
        g[j] = (r > 0.0) ? ((double)x[j] - (double)y[j]) / (h * r) : 0.0;
    *s = r / h;
    return k;
  }
  double r1 = l1_dist(x, y, d);
  double k = exp(-r1 / h);
  if (g)
    for (int j = 0; j < d; ++j) {
      double t = (double)x[j] - (double)y[j];
      g[j] = (t > 0.0 ? 1.0 : (t < 0.0 ? -1.0 : 0.0)) / h;
    }
  *s = r1 / h;
  return k;
}

/* ------------------------------------------------------------------------
 * Exact KDE (Definition "Kernel Density Estimate", Section 2):
 * KDE_X(y) = (1/n) sum_{i<n} K_h(x_i, y), summed in index order.
 * ---------------------------------------------------------------------- */
void or_exact(const float* X, int64_t n, int d, const float* Y, int64_t nq,
              int kern, double h, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < nq; ++q) {
    const float* y = Y + q * (int64_t)d;
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
      s += or_kernel_value(kern, X + i * (int64_t)d, y, d, h);
    out[q] = s / (double)n;
  }
}

/* Gradient of the exact KDE with respect to the query and to log h. */
void or_exact_grad(const float* X, int64_t n, int d, const float* Y, int64_t nq,
                   int kern, double h, double* dY, double* dlogh_per_query) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < nq; ++q) {
    const float* y = Y + q * (int64_t)d;
    double* gq = dY + q * (int64_t)d;
    double* g = (double*)malloc(sizeof(double) * (size_t)d);
    for (int j = 0; j < d; ++j) gq[j] = 0.0;
    double sl = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double s;
      double k = kernel_and_derivs(kern, X + i * (int64_t)d, y, d, h, g, &s);
      for (int j = 0; j < d; ++j) gq[j] += k * g[j];
      sl += k * s;
    }
    for (int j = 0; j < d; ++j) gq[j] /= (double)n;
    dlogh_per_query[q] = sl / (double)n;
    free(g);
  }
}

/* ------------------------------------------------------------------------
 * Nearest neighbours.  Order: (squared distance, index) ascending.
 * ---------------------------------------------------------------------- */
typedef struct {
  double d2;
  int64_t id;
} or_pair;

static int pair_cmp(const void* a, const void* b) {
  const or_pair* p = (const or_pair*)a;
  const or_pair* r = (const or_pair*)b;
  if (p->d2 < r->d2) return -1;
  if (p->d2 > r->d2) return 1;
  if (p->id < r->id) return -1;
  if (p->id > r->id) return 1;
  return 0;
}

/* Brute-force k nearest neighbours of every query (the paper's exact
 * baseline ANN, scikit-learn NearestNeighbors, Section 4): sort all n points
 * by (squared Euclidean distance, index) and keep the first k.  Entries past
 * n are -1 with distance +inf. */
void or_knn(const float* X, int64_t n, int d, const float* Y, int64_t nq, int k,
            int32_t* nbr, double* d2) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < nq; ++q) {
    const float* y = Y + q * (int64_t)d;
    or_pair* all = (or_pair*)malloc(sizeof(or_pair) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
      all[i].d2 = sq_dist(X + i * (int64_t)d, y, d);
      all[i].id = i;
    }
    qsort(all, (size_t)n, sizeof(or_pair), pair_cmp);
    for (int j = 0; j < k; ++j) {
      nbr[q * k + j] = (j < n) ? (int32_t)all[j].id : -1;
      if (d2) d2[q * k + j] = (j < n) ? all[j].d2 : INFINITY;
    }
    free(all);
  }
}

/* Nearest centroid of each point (the assignment of an IVF index, Section 4:
 * "each dataset point is assigned to its closest centroid").  Ties go to the
 * lower centroid id. */
void or_nearest_centroid(const float* X, int64_t n, int d, const float* C,
                         int L, int32_t* assign, double* d2) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double best = INFINITY;
    int32_t arg = -1;
    for (int c = 0; c < L; ++c) {
      double t = sq_dist(X + i * (int64_t)d, C + (int64_t)c * d, d);
      if (t < best) {
        best = t;
        arg = c;
      }
    }
    assign[i] = arg;
    if (d2) d2[i] = best;
  }
}

/* k-means for the inverted file.  Section 4 builds the IVF index with FAISS's
 * k-means and gives no details; this is the reading taken for them:
 *  - initial centroids: the first L distinct points drawn from Philox stream 1
 *    of `seed` (query id 0, draws t = 0, 1, 2, ...; a point already chosen is
 *    skipped; after 64 L + 4096 draws centroid c falls back to point c mod n,
 *    and the function returns OR_ELIMIT);
 *  - `iters` Lloyd iterations, each (i) assigning every point to its nearest
 *    centroid (ties to the lower id), (ii) moving every centroid with points
 *    to their mean (summed in increasing point index), stored as float32 as
 *    the index stores it, and (iii) giving each empty list, in increasing
 *    list order, the point farthest from its centroid of step (i) (ties to the
 *    lower index; a point is given once);
 *  - a final assignment.
 * obj (nullable, iters + 1 entries) receives the mean squared distance of
 * each assignment. */
int or_kmeans(const float* X, int64_t n, int d, int L, uint64_t seed, int iters,
              float* C, int32_t* assign, double* obj) {
  if (n < 1 || L < 1 || L > n || d < 1 || iters < 0) return OR_EINVAL;
  int status = OR_OK;
  char* taken = (char*)calloc((size_t)n, 1);
  uint32_t t = 0;
  const uint32_t cap = 64u * (uint32_t)L + 4096u;
  for (int c = 0; c < L; ++c) {
    int64_t pick = -1;
    while (pick < 0) {
      if (t >= cap) {
        pick = c % n;
        status = OR_ELIMIT;
        break;
      }
      const int64_t id = or_draw_index(seed, 0, t++, 1u, n);
      if (!taken[id]) {
        taken[id] = 1;
        pick = id;
      }
    }
    memcpy(C + (int64_t)c * d, X + pick * (int64_t)d, sizeof(float) * (size_t)d);
  }
  double* d2 = (double*)malloc(sizeof(double) * (size_t)n);
  double* sum = (double*)malloc(sizeof(double) * (size_t)d);
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)L);
  for (int it = 0; it <= iters; ++it) {
    or_nearest_centroid(X, n, d, C, L, assign, d2);
    if (obj) {
      double tot = 0.0;
      for (int64_t i = 0; i < n; ++i) tot += d2[i];
      obj[it] = tot / (double)n;
    }
    if (it == iters) break;
    for (int c = 0; c < L; ++c) cnt[c] = 0;
    for (int64_t i = 0; i < n; ++i) ++cnt[assign[i]];
    for (int c = 0; c < L; ++c) {
      if (cnt[c] == 0) continue;
      for (int j = 0; j < d; ++j) sum[j] = 0.0;
      for (int64_t i = 0; i < n; ++i)
        if (assign[i] == c)
          for (int j = 0; j < d; ++j) sum[j] += (double)X[i * (int64_t)d + j];
      for (int j = 0; j < d; ++j) C[(int64_t)c * d + j] = (float)(sum[j] / (double)cnt[c]);
    }
    memset(taken, 0, (size_t)n);
    for (int c = 0; c < L; ++c) {
      if (cnt[c] != 0) continue;
      int64_t far = -1;
      for (int64_t i = 0; i < n; ++i)
        if (!taken[i] && (far < 0 || d2[i] > d2[far])) far = i;
      if (far < 0) continue;
      taken[far] = 1;
      memcpy(C + (int64_t)c * d, X + far * (int64_t)d, sizeof(float) * (size_t)d);
    }
  }
  free(cnt);
  free(sum);
  free(d2);
  free(taken);
  return status;
}

/* IVF search run from an exported index (Section 4, the FAISS inverted file:
 * "it inspects all points associated with the n_q closest centroids").
 * probes = the nprobe centroids with the smallest distance to y, ties to the
 * lower id; candidates = every i with assign[i] among the probes; result = the
 * k candidates with the smallest (distance, index).  Fewer than k candidates
 * leave -1 / +inf padding. */
void or_ivf_search(const float* X, int64_t n, int d, const float* C, int L,
                   const int32_t* assign, const float* Y, int64_t nq,
                   int nprobe, int k, int32_t* probes, int32_t* nbr,
                   double* d2) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < nq; ++q) {
    const float* y = Y + q * (int64_t)d;
    or_pair* cent = (or_pair*)malloc(sizeof(or_pair) * (size_t)L);
    for (int c = 0; c < L; ++c) {
      cent[c].d2 = sq_dist(C + (int64_t)c * d, y, d);
      cent[c].id = c;
    }
    qsort(cent, (size_t)L, sizeof(or_pair), pair_cmp);
    char* probed = (char*)calloc((size_t)L, 1);
    for (int p = 0; p < nprobe; ++p) {
      probed[cent[p].id] = 1;
      if (probes) probes[q * nprobe + p] = (int32_t)cent[p].id;
    }
    int64_t nc = 0;
    for (int64_t i = 0; i < n; ++i)
      if (probed[assign[i]]) ++nc;
    or_pair* cand = (or_pair*)malloc(sizeof(or_pair) * (size_t)(nc > 0 ? nc : 1));
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i)
      if (probed[assign[i]]) {
        cand[w].d2 = sq_dist(X + i * (int64_t)d, y, d);
        cand[w].id = i;
        ++w;
      }
    qsort(cand, (size_t)nc, sizeof(or_pair), pair_cmp);
    for (int j = 0; j < k; ++j) {
      nbr[q * k + j] = (j < nc) ? (int32_t)cand[j].id : -1;
      if (d2) d2[q * k + j] = (j < nc) ? cand[j].d2 : INFINITY;
    }
    free(cand);
    free(probed);
    free(cent);
  }
}

/* ------------------------------------------------------------------------
 * The estimators.
 * ---------------------------------------------------------------------- */

/* Distinct valid neighbour indices of one query, in first-occurrence order.
 * Negative entries are padding.  Returns k' or -1 if an entry is >= n. */
static int distinct_neighbours(const int32_t* row, int k, int64_t n,
                               int64_t* set) {
  int kk = 0;
  for (int j = 0; j < k; ++j) {
    int64_t id = row[j];
    if (id < 0) continue;
    if (id >= n) return -1;
    int seen = 0;
    for (int t = 0; t < kk; ++t)
      if (set[t] == id) {
        seen = 1;
        break;
      }
    if (!seen) set[kk++] = id;
  }
  return kk;
}

static int in_set(const int64_t* set, int kk, int64_t id) {
  for (int t = 0; t < kk; ++t)
    if (set[t] == id) return 1;
  return 0;
}

/* The sample S of Algorithm 1 for one query: the first m draws of
 * the query's Philox stream (stream 0) that are not in X_1; draws in X_1 are
 * rejected, so S is uniform on X \ X_1 with repetition (Lemma RS).  Returns
 * the number of draws used, or -1 when the draw cap 64 m + 4096 is hit. */
static int64_t draw_sample(uint64_t seed, uint64_t qid, int64_t n,
                           const int64_t* set, int kk, int m, int64_t* S) {
  const int64_t cap = 64 * (int64_t)m + 4096;
  int got = 0;
  int64_t t = 0;
  while (got < m) {
    if (t >= cap) return -1;
    int64_t id = or_draw_index(seed, qid, (uint32_t)t, 0u, n);
    ++t;
    if (in_set(set, kk, id)) continue;
    S[got++] = id;
  }
  return t;
}

/* DEANN, Algorithm 1, given the neighbour set X_1 of every query:
 *   Z_1 = (1/k') sum_{X_1} K,  S = m uniform draws from X \ X_1,
 *   Z_2 = (1/m) sum_S K,       out = (k'/n) Z_1 + ((n-k')/n) Z_2,
 * where k' = |X_1| counts distinct valid indices (negative entries are
 * padding).  Written as (1/n) [ s1 + ((n-k')/m) s2 ] with s1, s2 the plain
 * sums.  k' = n or m = 0 returns s1/n with no draws (Section 3.2: "discards
 * all far points"; with k' = n nothing is left to sample).
 * mode 0 = rejection sampling from X \ X_1 (above).
 * mode 1 = "drop": m draws from all of X, draws in X_1 contribute nothing,
 *          out = s1/n + (1/m) sum_{t<m, i_t not in X_1} K.  Also unbiased.
 * samples (nullable, nq x m) receives the sample indices (mode 0) or the raw
 * draws (mode 1); rows with no sampling hold -1. */
int or_deann(const float* X, int64_t n, int d, const float* Y, int64_t nq,
             int kern, double h, const int32_t* nbr, int k, int m,
             uint64_t seed, uint64_t qid_offset, int mode, double* out,
             int32_t* samples) {
  int status = OR_OK;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < nq; ++q) {
    const float* y = Y + q * (int64_t)d;
    int64_t* set = (int64_t*)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    int64_t* S = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int kk = distinct_neighbours(nbr ? nbr + q * (int64_t)k : NULL, nbr ? k : 0,
                                 n, set);
    if (samples)
      for (int t = 0; t < m; ++t) samples[q * (int64_t)m + t] = -1;
    if (kk < 0) {
#pragma omp atomic write
      status = OR_EINVAL;
      out[q] = NAN;
    } else {
      double s1 = 0.0;
      for (int t = 0; t < kk; ++t)
        s1 += or_kernel_value(kern, X + set[t] * (int64_t)d, y, d, h);
      if ((int64_t)kk == n || m == 0) {
        out[q] = s1 / (double)n;
      } else if (mode == 0) {
        int64_t used = draw_sample(seed, qid_offset + (uint64_t)q, n, set, kk, m, S);
        if (used < 0) {
#pragma omp atomic write
          status = OR_ELIMIT;
          out[q] = NAN;
        } else {
          double s2 = 0.0;
          for (int t = 0; t < m; ++t) {
            s2 += or_kernel_value(kern, X + S[t] * (int64_t)d, y, d, h);
            if (samples) samples[q * (int64_t)m + t] = (int32_t)S[t];
          }
          out[q] = (s1 + ((double)(n - kk) / (double)m) * s2) / (double)n;
        }
      } else {
        double s2 = 0.0;
        for (int t = 0; t < m; ++t) {
          int64_t id = or_draw_index(seed, qid_offset + (uint64_t)q, (uint32_t)t, 0u, n);
          if (samples) samples[q * (int64_t)m + t] = (int32_t)id;
          if (!in_set(set, kk, id))
            s2 += or_kernel_value(kern, X + id * (int64_t)d, y, d, h);
        }
        out[q] = s1 / (double)n + s2 / (double)m;
      }
    }
    free(S);
    free(set);
  }
  return status;
}

/* Plain random sampling (Lemma RS, Section 2): m uniform draws from X with
 * repetition, the first m draws of the query's stream, out = (1/m) sum K. */
int or_rs(const float* X, int64_t n, int d, const float* Y, int64_t nq, int kern,
          double h, int m, uint64_t seed, uint64_t qid_offset, double* out,
          int32_t* samples) {
  if (m <= 0) return OR_EINVAL;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < nq; ++q) {
    const float* y = Y + q * (int64_t)d;
    double s = 0.0;
    for (int t = 0; t < m; ++t) {
      int64_t id = or_draw_index(seed, qid_offset + (uint64_t)q, (uint32_t)t, 0u, n);
      if (samples) samples[q * (int64_t)m + t] = (int32_t)id;
      s += or_kernel_value(kern, X + id * (int64_t)d, y, d, h);
    }
    out[q] = s / (double)m;
  }
  return OR_OK;
}

/* Pathwise derivative of the DEANN estimate (mode 0) with the neighbour set
 * and the sample held fixed: every term of (1/n)[s1 + ((n-k')/m) s2] is a
 * weight w times K_h(x, y), so d/dy = sum w K g and d/dlog h = sum w K s
 * (g, s from kernel_and_derivs).  The paper defines no gradient; this is the
 * derivative of the estimator it defines.  Outputs are scaled by gout[q];
 * dlogh_per_query[q] receives gout[q] * d out[q] / d log h. */
int or_deann_grad(const float* X, int64_t n, int d, const float* Y, int64_t nq,
                  int kern, double h, const int32_t* nbr, int k, int m,
                  uint64_t seed, uint64_t qid_offset, const double* gout,
                  double* out, double* dY, double* dlogh_per_query) {
  int status = OR_OK;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < nq; ++q) {
    const float* y = Y + q * (int64_t)d;
    double* gq = dY + q * (int64_t)d;
    int64_t* set = (int64_t*)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    int64_t* S = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    double* g = (double*)malloc(sizeof(double) * (size_t)d);
    for (int j = 0; j < d; ++j) gq[j] = 0.0;
    dlogh_per_query[q] = 0.0;
    int kk = distinct_neighbours(nbr ? nbr + q * (int64_t)k : NULL, nbr ? k : 0,
                                 n, set);
    if (kk < 0) {
#pragma omp atomic write
      status = OR_EINVAL;
      out[q] = NAN;
    } else {
      int sampled = !((int64_t)kk == n || m == 0);
      int64_t used = 0;
      if (sampled) used = draw_sample(seed, qid_offset + (uint64_t)q, n, set, kk, m, S);
      if (used < 0) {
#pragma omp atomic write
        status = OR_ELIMIT;
        out[q] = NAN;
      } else {
        double w1 = 1.0 / (double)n;
        double w2 = sampled ? (double)(n - kk) / ((double)n * (double)m) : 0.0;
        double est = 0.0, sl = 0.0, sv;
        for (int t = 0; t < kk; ++t) {
          double kv = kernel_and_derivs(kern, X + set[t] * (int64_t)d, y, d, h, g, &sv);
          est += w1 * kv;
          sl += w1 * kv * sv;
          for (int j = 0; j < d; ++j) gq[j] += w1 * kv * g[j];
        }
        if (sampled)
          for (int t = 0; t < m; ++t) {
            double kv = kernel_and_derivs(kern, X + S[t] * (int64_t)d, y, d, h, g, &sv);
            est += w2 * kv;
            sl += w2 * kv * sv;
            for (int j = 0; j < d; ++j) gq[j] += w2 * kv * g[j];
          }
        out[q] = est;
        double go = gout ? gout[q] : 1.0;
        for (int j = 0; j < d; ++j) gq[j] *= go;
        dlogh_per_query[q] = go * sl;
      }
    }
    free(g);
    free(S);
    free(set);
  }
  return status;
}

/* ------------------------------------------------------------------------
 * Permuted random sampling (Algorithm 2, Appendix "Permuted Random
 * Sampling"): given the permutation pi and the running index ell, the sample
 * of a query is the window x'_{ell}, ..., x'_{ell+m-1} (indices mod n) of the
 * permuted dataset x'_i = x_{pi(i)}; ell then advances by m mod n.  Queries are
 * served in order, so query q's window starts at (ell0 + q m) mod n.
 * DEANNP combines it with the neighbour set: window entries that fall in X_1
 * are dropped and the window's sum is normalised by the m' entries of
 * X \ X_1 it holds, out = (1/n)[s1 + ((n - k')/m') s2] (s1/n when m' = 0).
 * Given m', the kept entries are a uniform m'-subset of X \ X_1 for a random
 * permutation, so the estimate is unbiased.  Requires m <= n.
 * ell_out (nullable) receives the running index after the last query.
 * ---------------------------------------------------------------------- */
int or_deannp(const float* X, int64_t n, int d, const float* Y, int64_t nq,
              int kern, double h, const int32_t* perm, const int32_t* nbr,
              int k, int m, int64_t ell0, double* out, int64_t* ell_out) {
  if (n <= 0) return OR_EINVAL;
  int64_t ell = ((ell0 % n) + n) % n;
  int64_t* set = (int64_t*)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
  int status = OR_OK;
  if (m < 0 || (int64_t)m > n) status = OR_EINVAL;
  for (int64_t q = 0; q < nq && status == OR_OK; ++q) {
    const float* y = Y + q * (int64_t)d;
    int kk = distinct_neighbours(nbr ? nbr + q * (int64_t)k : NULL, nbr ? k : 0,
                                 n, set);
    if (kk < 0) {
      status = OR_EINVAL;
      out[q] = NAN;
      break;
    }
    double s1 = 0.0;
    for (int t = 0; t < kk; ++t)
      s1 += or_kernel_value(kern, X + set[t] * (int64_t)d, y, d, h);
    double s2 = 0.0;
    int64_t kept = 0;
    if ((int64_t)kk < n) {
      for (int t = 0; t < m; ++t) {
        int64_t id = perm[(ell + t) % n];
        if (in_set(set, kk, id)) continue;
        s2 += or_kernel_value(kern, X + id * (int64_t)d, y, d, h);
        ++kept;
      }
    }
    out[q] = kept > 0 ? (s1 + ((double)(n - kk) / (double)kept) * s2) / (double)n
                      : s1 / (double)n;
    ell = (ell + m) % n;
  }
  free(set);
  if (ell_out) *ell_out = ell;
  return status;
}

/* Keyed pseudo-random permutation of [0, n) drawn for Algorithm 2's
 * preprocessing: a 4-round balanced Feistel network on 2h bits (h = half the
 * bit length of n - 1, rounded up) whose round function is Philox4x32-10
 * (counter (R, round, 0, 3), key (lo32(seed), hi32(seed)), output word r0),
 * made into a permutation of [0, n) by cycle walking (Black, Rogaway,
 * "Ciphers with Arbitrary Finite Domains", CT-RSA 2002): re-apply the network
 * until the value falls below n. */
int64_t or_feistel_perm(uint64_t seed, int64_t n, int64_t i) {
  int bits = 1;
  while (bits < 62 && ((int64_t)1 << bits) < n) ++bits;
  const int hb = (bits + 1) / 2;
  const uint64_t mask = ((uint64_t)1 << hb) - 1;
  uint64_t x = (uint64_t)i;
  do {
    uint64_t L = x >> hb, R = x & mask;
    for (uint32_t r = 0; r < 4; ++r) {
      uint32_t ctr[4] = {(uint32_t)R, r, 0u, 3u};
      uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
      uint32_t o[4];
      or_philox4x32_10(ctr, key, o);
      uint64_t F = (uint64_t)o[0] & mask;
      uint64_t nL = R, nR = L ^ F;
      L = nL;
      R = nR;
    }
    x = (L << hb) | R;
  } while ((int64_t)x >= n);
  return (int64_t)x;
}

/* ------------------------------------------------------------------------
 * Bandwidth fitting by the leave-one-out likelihood (gradient ascent on
 * log h with the estimator's derivative in log h; the paper tunes h by
 * bisection only, this is the fitting loop the adjoint serves).
 *
 * The kernels carry no normalising constant; each normalises as c h^d
 * (Gaussian (2 pi)^{d/2} h^d, exponential and Laplacian a constant times
 * h^d), so up to a constant the log-likelihood of a held-out point z under
 * the density built from X \ {z} is
 *     log KDE_{-z}(z) - d log h,   KDE_{-z}(z) = (n KDE(z) - 1) / (n - 1),
 * since K(z, z) = 1 for the three kernels.  Its derivative in log h is
 *     (n / (n - 1)) dKDE(z)/dlog h / KDE_{-z}(z) - d.
 * l(h) averages over training points z_j = x_{zid[j]}.  A point with no
 * held-out density (KDE_{-z}(z) <= 0: every other kernel value underflowed)
 * is left out of both averages.
 * ---------------------------------------------------------------------- */
static void loo_terms(int64_t n, int64_t nz, const double* out, const double* dlogh,
                      double* sum_log, double* sum_ratio, int64_t* used) {
  double sl = 0.0, sr = 0.0;
  int64_t u = 0;
  for (int64_t j = 0; j < nz; ++j) {
    const double nk = (double)n * out[j];
    if (!(nk - 1.0 > 0.0)) continue;
    const double loo = (nk - 1.0) / (double)(n - 1);
    const double dloo = (double)n * dlogh[j] / (double)(n - 1);
    sl += log(loo);
    sr += dloo / loo;
    ++u;
  }
  *sum_log = sl;
  *sum_ratio = sr;
  *used = u;
}

static float* gather_rows_f(const float* X, int d, const int32_t* zid, int64_t nz) {
  float* Y = (float*)malloc(sizeof(float) * (size_t)nz * (size_t)d);
  for (int64_t j = 0; j < nz; ++j)
    memcpy(Y + j * (int64_t)d, X + (int64_t)zid[j] * d, sizeof(float) * (size_t)d);
  return Y;
}

/* Exact l(h) and dl/dlog h (Section 2 definition for KDE(z)). */
int or_loo_exact(const float* X, int64_t n, int d, const int32_t* zid, int64_t nz, int kern,
                 double h, double* ll, double* dll, int64_t* used) {
  if (n < 2 || nz < 1) return OR_EINVAL;
  for (int64_t j = 0; j < nz; ++j)
    if (zid[j] < 0 || zid[j] >= n) return OR_EINVAL;
  float* Y = gather_rows_f(X, d, zid, nz);
  double* out = (double*)malloc(sizeof(double) * (size_t)nz);
  double* dl = (double*)malloc(sizeof(double) * (size_t)nz);
  double* dY = (double*)malloc(sizeof(double) * (size_t)nz * (size_t)d);
  or_exact(X, n, d, Y, nz, kern, h, out);
  or_exact_grad(X, n, d, Y, nz, kern, h, dY, dl);
  double sl, sr;
  int64_t u;
  loo_terms(n, nz, out, dl, &sl, &sr, &u);
  int status = OR_OK;
  if (u == 0) {
    status = OR_EINVAL;
  } else {
    *ll = sl / (double)u - (double)d * log(h);
    *dll = sr / (double)u - (double)d;
  }
  if (used) *used = u;
  free(Y);
  free(out);
  free(dl);
  free(dY);
  return status;
}

/* Gradient ascent on log h with the DEANN estimate: X_1 of z_j is row j of
 * nbr (nz x kw, -1 pads; it should contain z_j itself, so that KDE_{-z}
 * follows from the estimate); iteration t draws its samples with seed + t
 * and query ids j; log h <- log h + lr g_t.  h_trace[0..iters],
 * ll_trace[0..iters) (l at the h before each update). */
int or_fit_bandwidth(const float* X, int64_t n, int d, const int32_t* zid, int64_t nz, int kern,
                     double h0, const int32_t* nbr, int kw, int m, uint64_t seed, int iters,
                     double lr, double* h_trace, double* ll_trace) {
  if (n < 2 || nz < 1 || !(h0 > 0.0) || iters < 0) return OR_EINVAL;
  for (int64_t j = 0; j < nz; ++j)
    if (zid[j] < 0 || zid[j] >= n) return OR_EINVAL;
  float* Y = gather_rows_f(X, d, zid, nz);
  double* out = (double*)malloc(sizeof(double) * (size_t)nz);
  double* dl = (double*)malloc(sizeof(double) * (size_t)nz);
  double* dY = (double*)malloc(sizeof(double) * (size_t)nz * (size_t)d);
  double h = h0;
  int status = OR_OK;
  h_trace[0] = h;
  for (int t = 0; t < iters && status == OR_OK; ++t) {
    status = or_deann_grad(X, n, d, Y, nz, kern, h, nbr, kw, m, seed + (uint64_t)t, 0, NULL,
                           out, dY, dl);
    if (status != OR_OK) break;
    double sl, sr;
    int64_t u;
    loo_terms(n, nz, out, dl, &sl, &sr, &u);
    if (u == 0) {
      status = OR_EINVAL;
      break;
    }
    ll_trace[t] = sl / (double)u - (double)d * log(h);
    const double g = sr / (double)u - (double)d;
    h = exp(log(h) + lr * g);
    h_trace[t + 1] = h;
  }
  free(Y);
  free(out);
  free(dl);
  free(dY);
  return status;
}

/* ------------------------------------------------------------------------
 * Density-gradient flow with the DEANN estimate (Section 1 names gradient
 * lines of densities among the uses of KDE; the paper gives no algorithm).
 * Gaussian kernel only.  Each of `steps` steps moves every query by
 *     y <- y + h^2 grad KDE~(y) / KDE~(y),
 * the mean-shift step: since grad K_h(x, y) = K_h(x, y) (x - y) / h^2 for the
 * Gaussian kernel, the new y is the estimate-weighted mean of the points of
 * X_1 and S.  Step s takes X_1 from the IVF search of the current y (the
 * exported centroids C and list assignment, nprobe lists, k neighbours; no
 * search when k = 0) and draws S from the Philox stream of seed + s with query
 * id qid_offset + q; the gradient is the pathwise derivative of
 * or_deann_grad.  The iterate stays in FP32 between steps (a query is an FP32
 * vector); each update is computed in FP64 and rounded once.  A query whose
 * estimate is 0 does not move.  est (nullable) receives the estimate at the
 * start of the last step (0 when steps = 0).
 * ---------------------------------------------------------------------- */
int or_mean_shift(const float* X, int64_t n, int d, const float* C, int L,
                  const int32_t* assign, float* Y, int64_t nq, double h, int k,
                  int m, int nprobe, uint64_t seed, uint64_t qid_offset, int steps,
                  double* est) {
  if (n <= 0 || d <= 0 || nq < 0 || k < 0 || m < 0 || steps < 0 || !(h > 0.0))
    return OR_EINVAL;
  if (k > 0 && (nprobe < 1 || nprobe > L)) return OR_EINVAL;
  const size_t q1 = (size_t)(nq > 0 ? nq : 1);
  int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * q1 * (size_t)(k > 0 ? k : 1));
  int32_t* probes = (int32_t*)malloc(sizeof(int32_t) * q1 * (size_t)(nprobe > 0 ? nprobe : 1));
  double* out = (double*)malloc(sizeof(double) * q1);
  double* dY = (double*)malloc(sizeof(double) * q1 * (size_t)d);
  double* dl = (double*)malloc(sizeof(double) * q1);
  int status = OR_OK;
  if (est)
    for (int64_t q = 0; q < nq; ++q) est[q] = 0.0;
  for (int s = 0; s < steps && status == OR_OK; ++s) {
    if (k > 0)
      or_ivf_search(X, n, d, C, L, assign, Y, nq, nprobe, k, probes, nbr, NULL);
    status = or_deann_grad(X, n, d, Y, nq, OR_GAUSSIAN, h, k > 0 ? nbr : NULL, k, m,
                           seed + (uint64_t)s, qid_offset, NULL, out, dY, dl);
    if (status != OR_OK) break;
    for (int64_t q = 0; q < nq; ++q) {
      if (est) est[q] = out[q];
      if (!(out[q] > 0.0)) continue;
      float* y = Y + q * (int64_t)d;
      for (int j = 0; j < d; ++j)
        y[j] = (float)((double)y[j] + h * h * dY[q * (int64_t)d + j] / out[q]);
    }
  }
  free(dl);
  free(dY);
  free(out);
  free(probes);
  free(nbr);
  return status;
}
