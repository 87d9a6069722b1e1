// C-ABI entry points (include/deann_gb300.h): argument checks, pointer-space
// handling, scratch layout and the launch sequence of each call.  All
// arithmetic runs in the kernels of build.cu, tiles.cu, select.cu and
// sample.cu; this file only moves bytes and orders launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "deann_gb300.h"
#include "internal.h"

using namespace deann;

namespace {

thread_local std::string g_err;

kde_status fail(kde_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(KDE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

#define TRY(expr)                  \
  do {                             \
    kde_status s_ = (expr);        \
    if (s_ != KDE_OK) return s_;   \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      changed = cudaSetDevice(dev) == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

enum Space { SPACE_HOST = 0, SPACE_DEVICE = 1, SPACE_FOREIGN = 2 };

Space space_of(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return SPACE_HOST;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
    return a.device == device ? SPACE_DEVICE : SPACE_FOREIGN;
  return SPACE_HOST;
}

cudaStream_t stream_of(const kde_opts* o) {
  return (o != nullptr && o->stream != nullptr) ? reinterpret_cast<cudaStream_t>(o->stream)
                                                : cudaStream_t(0);
}

const kde_opts kDefaultOpts = {0, 0, 0, 0, 0, nullptr, nullptr, nullptr};

// Bump layout over the index's scratch buffer; with base == nullptr it only
// counts bytes, so the same carve code sizes and places the buffers.
struct Bump {
  char* base = nullptr;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    const size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += bytes;
    return p;
  }
};

kde_status ensure_scratch(kde_index* ix, size_t bytes) {
  if (bytes <= ix->scratch.cap) return KDE_OK;
  if (bytes > ix->scratch_limit)
    return fail(KDE_ENOMEM, "call needs %zu bytes of scratch, above the limit %zu", bytes,
                ix->scratch_limit);
  // The outgrown buffer is retired, not freed: CUDA graphs captured from
  // earlier calls hold its addresses and stay valid until kde_free.
  const size_t cap = std::max(bytes, size_t(64) << 20);
  void* p = nullptr;
  if (cudaMalloc(&p, cap) != cudaSuccess) {
    cudaGetLastError();
    return fail(KDE_ENOMEM, "cudaMalloc of %zu scratch bytes failed", cap);
  }
  if (ix->scratch.base) ix->retired.push_back(ix->scratch.base);
  ix->scratch.base = static_cast<char*>(p);
  ix->scratch.cap = cap;
  return KDE_OK;
}

template <class T>
kde_status dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(KDE_ENOMEM, "cudaMalloc of %zu bytes failed", count * sizeof(T));
  }
  return KDE_OK;
}

// Reads and clears the device error words; maps them to a status.
kde_status collect_errors(kde_index* ix, cudaStream_t st, int64_t* margin_out) {
  uint32_t h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, ix->err, sizeof h, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  CK(cudaMemsetAsync(ix->err, 0, 2 * sizeof(uint32_t), st));
  if (margin_out) *margin_out = h[1];
  if (h[0] & KDE_ERRBIT_DRAWCAP)
    return fail(KDE_ELIMIT, "a query needed more than 64 m + 4096 draws (k' close to n)");
  if (h[0] & KDE_ERRBIT_BADNBR) return fail(KDE_EINVAL, "a neighbour id was >= n");
  return KDE_OK;
}

void ix_margin_accumulate(kde_index* ix, int64_t m) { ix->margin_failures += m; }

// Stages of a call, for kde_profile_read.
enum { ST_STAGE = 0, ST_COARSE, ST_PLAN, ST_SCAN, ST_SELECT, ST_ESTIMATE, ST_EXACT, ST_GRAD };

// Counts the kernels a stage launches and, when profiling is on, brackets
// the stage with CUDA events on the call's stream.
struct StageTimer {
  kde_index* ix;
  cudaStream_t st;
  int stage;
  cudaEvent_t a = nullptr, b = nullptr;
  StageTimer(kde_index* ix_, int stage_, cudaStream_t st_, int nlaunch)
      : ix(ix_), st(st_), stage(stage_) {
    ix->launches[stage] += nlaunch;
    ix->calls[stage] += 1;
    if (ix->prof && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
      cudaEventRecord(a, st);
  }
  ~StageTimer() {
    if (a != nullptr && b != nullptr) {
      cudaEventRecord(b, st);
      ix->events.push_back({a, b, stage});
    }
  }
};

float scan_err_scale(int dp, int dpb, int precision) {
  const float u = 1.0f / 16777216.0f;  // 2^-24
  if (precision == 0) return 2.0f * ((float)dp / 32.0f + 40.0f) * u;
  if (precision == 2) {
    // three-way split, per unit of r^2 (r = |x~| + |y~|): the main
    // accumulator's FP32 additions, assuming only that each MMA accumulates at
    // FP32 precision (dpb / 16 MMAs of 16 products plus the accumulator,
    // each addition off by 2^-23 at most, on sums bounded by |x~||y~| <=
    // r^2 / 4), twice that in D^2, plus the dropped split terms, the norms'
    // rounding, the centring subtractions and the epilogue's FP32 sums
    return (1.1f * (float)dpb + 8.0f) * u;
  }
  // BF16 operands, each rounded to nearest with 8 significant bits: the dot
  // product is off by at most 2^-8 |x||y| <= 2^-10 (|x| + |y|)^2, twice that
  // in D^2, plus the FP32 accumulation and norm terms
  return 1.0f / 512.0f + 2.0f * ((float)dp / 32.0f + 40.0f) * u;
}

// ---- query scratch ---------------------------------------------------------
struct SearchBufs {
  int64_t qc = 0;  // queries per chunk
  float* D = nullptr;
  int32_t* probes = nullptr;
  float* probe_d2 = nullptr;  // |y - c_probe|^2, rescored
  int64_t *q_count = nullptr, *q_real = nullptr, *q_off = nullptr, *seg_off = nullptr;
  int64_t *list_cnt = nullptr, *bucket_off = nullptr, *bucket_fill = nullptr;
  int64_t *tile_cnt = nullptr, *tile_off = nullptr;
  int32_t* pair_q = nullptr;
  int64_t* pair_dst = nullptr;
  int64_t *ord_cnt = nullptr, *ord_off = nullptr, *ord_fill = nullptr;
  int32_t* order = nullptr;
  float* cand = nullptr;
  void* Ys = nullptr;     // the queries' BF16 parts [3][qc][dpb] (tensor-core coarse quantiser)
  float* ysn = nullptr;   // |y - mean|^2
};

constexpr size_t kCandCap = size_t(8) << 30;  // candidate buffer per chunk of queries

void carve_search(Bump& b, const kde_index* ix, int64_t nq, int P, SearchBufs& s) {
  const int L = ix->nlist;
  // each (query, probe) candidate segment is padded to a multiple of 32 floats
  const size_t per_q = ((size_t)P * ((size_t)std::max<int64_t>(ix->max_list, 1) + 32)) * sizeof(float);
  int64_t qc = (int64_t)std::max<size_t>(1, kCandCap / per_q);
  qc = std::min<int64_t>(qc, std::max<int64_t>(nq, 1));
  s.qc = qc;
  s.D = b.take<float>((size_t)qc * L);
  s.probes = b.take<int32_t>((size_t)qc * P);
  s.probe_d2 = b.take<float>((size_t)qc * P);
  s.q_count = b.take<int64_t>(qc);
  s.q_real = b.take<int64_t>(qc);
  s.q_off = b.take<int64_t>(qc + 1);
  s.seg_off = b.take<int64_t>((size_t)qc * P);
  s.list_cnt = b.take<int64_t>(L);
  s.bucket_off = b.take<int64_t>(L + 1);
  s.bucket_fill = b.take<int64_t>(L);
  s.tile_cnt = b.take<int64_t>(L);
  s.tile_off = b.take<int64_t>(L + 1);
  s.pair_q = b.take<int32_t>((size_t)qc * P);
  s.pair_dst = b.take<int64_t>((size_t)qc * P);
  s.ord_cnt = b.take<int64_t>(L);
  s.ord_off = b.take<int64_t>(L + 1);
  s.ord_fill = b.take<int64_t>(L);
  s.order = b.take<int32_t>(qc);
  s.Ys = b.take<uint16_t>((size_t)3 * qc * ix->dpb);
  s.ysn = b.take<float>(qc);
  s.cand = b.take<float>((size_t)qc * (size_t)P * ((size_t)std::max<int64_t>(ix->max_list, 1) + 32));
}

struct CallBufs {
  float* Yp = nullptr;     // nq x dp padded queries
  float* Yn = nullptr;     // nq norms
  float* out = nullptr;    // nq
  int32_t* nbr = nullptr;  // nq x k
  float* nd2 = nullptr;    // nq x k
  float* s1 = nullptr;     // nq
  int32_t* samples = nullptr;
  float* gout = nullptr;
  float* dY = nullptr;
  float* dlogh = nullptr;
  double* acc = nullptr;
  void* Ys = nullptr;      // [3][nq][dpb] BF16 parts of the centred queries
  float* ysn = nullptr;    // their squared norms
  // tiled permuted windows
  WindowPlan win;
  int32_t* win_drops = nullptr;  // nq x max(k, 1)
  int32_t* win_dcnt = nullptr;
  int32_t* win_kk = nullptr;
  float* win_s1 = nullptr;
  double* win_part = nullptr;    // nq x nslices
  // phased estimator (query calls)
  PhasePlan ph;
  int32_t* ph_ids = nullptr;     // nq x m
  int32_t* ph_off = nullptr;     // nq x (P + 1)
  int32_t* ph_info = nullptr;    // nq
  float* ph_part = nullptr;      // P x nq x kPhaseWarps
  // bandwidth fitting
  int32_t* fit_zid = nullptr;    // nq training point ids
  int32_t* fit_nbr = nullptr;    // nq x fit_k search neighbours
  double* fit_red = nullptr;     // leave-one-out sums
  SearchBufs search;
};

struct CallShape {
  int64_t nq = 0;
  int k = 0, m = 0, P = 0;
  bool search = false;     // runs the IVF search
  bool host = false;       // host-pointer call (needs device copies of outputs)
  bool need_nbr = false;   // neighbour ids on the device
  bool need_nd2 = false;
  bool need_out = false;
  bool need_s1 = false;
  bool need_samples = false;
  bool grad = false;
  bool exact = false;
  bool exact_tc = false;   // tensor-core exact: BF16 parts of the queries
  bool window = false;     // permuted-window estimator (sample_mode 2)
  int fit_k = -1;          // >= 0: bandwidth fitting with fit_k search neighbours
};

void carve_call(Bump& b, const kde_index* ix, const CallShape& c, CallBufs& cb) {
  const int64_t nq = std::max<int64_t>(c.nq, 1);
  cb.Yp = b.take<float>((size_t)nq * ix->dp);
  cb.Yn = b.take<float>(nq);
  if (c.need_out) cb.out = b.take<float>(nq);
  if (c.need_nbr) cb.nbr = b.take<int32_t>((size_t)nq * std::max(c.k, 1));
  if (c.need_nd2) cb.nd2 = b.take<float>((size_t)nq * std::max(c.k, 1));
  if (c.need_s1) cb.s1 = b.take<float>(nq);
  if (c.need_samples) cb.samples = b.take<int32_t>((size_t)nq * std::max(c.m, 1));
  if (c.grad) {
    cb.gout = b.take<float>(nq);
    cb.dY = b.take<float>((size_t)nq * ix->d);
    cb.dlogh = b.take<float>(nq);
  }
  if (c.exact) cb.acc = b.take<double>(nq);
  if (c.exact_tc) {
    cb.Ys = b.take<uint16_t>((size_t)3 * nq * ix->dpb);
    cb.ysn = b.take<float>(nq);
  }
  if (c.window && c.m > 0) {
    cb.win = window_plan(c.nq, ix->n, c.m);
    if (window_tiled(cb.win)) {
      cb.win_drops = b.take<int32_t>((size_t)nq * std::max(c.k, 1));
      cb.win_dcnt = b.take<int32_t>(nq);
      cb.win_kk = b.take<int32_t>(nq);
      cb.win_s1 = b.take<float>(nq);
      cb.win_part = b.take<double>((size_t)nq * cb.win.nslices);
    }
  }
  // the phased order's sorted draws are capped at kPhasedMaxDraws a call
  // (larger batches take the per-query order)
  if (c.search && c.k > 0 && c.m > 0 && (int64_t)c.nq * c.m <= kPhasedMaxDraws) {
    cb.ph = phase_plan(ix->n, ix->dp, c.m, c.nq, ix->phase_bytes);
    if (cb.ph.P > 0) {
      cb.ph_ids = b.take<int32_t>((size_t)nq * c.m);
      cb.ph_off = b.take<int32_t>((size_t)nq * (cb.ph.P + 1));
      cb.ph_info = b.take<int32_t>(nq);
      cb.ph_part = b.take<float>((size_t)nq * cb.ph.P * kPhaseWarps);
    }
  }
  if (c.fit_k >= 0) {
    cb.fit_zid = b.take<int32_t>(nq);
    cb.fit_nbr = b.take<int32_t>((size_t)nq * std::max(c.fit_k, 1));
    cb.fit_red = b.take<double>(4);
  }
  if (c.search) carve_search(b, ix, c.nq, c.P, cb.search);
}

kde_status prepare_call(kde_index* ix, const CallShape& c, CallBufs& cb) {
  Bump count;
  CallBufs dummy;
  carve_call(count, ix, c, dummy);
  TRY(ensure_scratch(ix, count.used));
  Bump real;
  real.base = ix->scratch.base;
  carve_call(real, ix, c, cb);
  return KDE_OK;
}

// Pads queries (nq x d, host or device) into cb.Yp (nq x dp) and computes norms.
kde_status stage_queries(kde_index* ix, const float* Y, int64_t nq, bool host, CallBufs& cb,
                         cudaStream_t st) {
  if (nq == 0) return KDE_OK;
  if (ix->dp != ix->d) CK(cudaMemsetAsync(cb.Yp, 0, sizeof(float) * nq * ix->dp, st));
  CK(cudaMemcpy2DAsync(cb.Yp, sizeof(float) * ix->dp, Y, sizeof(float) * ix->d,
                       sizeof(float) * ix->d, (size_t)nq,
                       host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
  StageTimer t(ix, ST_STAGE, st, 1);
  launch_query_norms(cb.Yp, nq, ix->dp, cb.Yn, st);
  return KDE_OK;
}

// IVF search on staged queries: neighbours, optional squared distances and s1.
// ids_only: the caller needs the neighbour set in any order (and s1), not
// the sorted list with distances; the selection then skips the full sort.
kde_status run_search(kde_index* ix, const CallBufs& cb, int64_t nq, int k, int P, int precision,
                      int32_t* nbr, float* nd2, float* s1, cudaStream_t st,
                      bool ids_only = false, const int64_t* active = nullptr) {
  const SearchBufs& s = cb.search;
  const int L = ix->nlist;
  for (int64_t q0 = 0; q0 < nq; q0 += s.qc) {
    const int64_t nc = std::min<int64_t>(s.qc, nq - q0);
    const float* Yc = cb.Yp + q0 * ix->dp;
    const float* Ync = cb.Yn + q0;
    {
      // with one list the probe is list 0; the step still yields |y - c_0|^2.
      // The tensor-core scans take the query-centroid distances from the
      // split-BF16 tensor-core GEMM, the FP32 scan from the SIMT tiles.
      const bool tc_coarse = (precision == KDE_PREC_BF16 || precision == KDE_PREC_BF16X3) &&
                             ix->cs_ok;
      StageTimer t(ix, ST_COARSE, st, tc_coarse ? 3 : 2);
      if (tc_coarse) {
        launch_split3(Yc, nc, ix->dp, ix->mean, s.Ys, nc, ix->dpb, s.ysn, st);
        if (!launch_coarse_tc(ix->tmap_cs, ix->csn, L, s.Ys, s.ysn, nc, ix->dpb, s.D, active, q0,
                              ix->err, st))
          return fail(KDE_ECUDA, "could not configure the tensor-core coarse quantiser");
      } else {
        launch_dist_matrix(Yc, Ync, nc, ix->C, ix->Cn, L, ix->dp, s.D, active, q0, st);
      }
      launch_select_probes(s.D, nc, L, Yc, ix->d, ix->dp, ix->C, P, std::max(8, P / 2),
                           s.probes, s.probe_d2, active, q0, st);
    }
    // the tensor-core scans group up to BN queries per list; the FP32 SIMT
    // scan groups 64
    const bool tcore = precision == KDE_PREC_BF16 || precision == KDE_PREC_BF16X3;
    const bool split = precision == KDE_PREC_BF16X3;
    if (split && ix->dpb > kMaxSplitDim)
      return fail(KDE_EINVAL, "the split BF16 scan needs d <= %d", kMaxSplitDim);
    if (tcore && !(split ? ix->xls_ok : ix->tmap_ok))
      return fail(KDE_ECUDA, "the BF16 tensor map could not be encoded on this driver");
    int qtile = tcore ? scan_tc_bn(ix->dpb, split) : kTile;
    if (tcore && ix->scan_tile[precision] > 0) qtile = std::min(qtile, ix->scan_tile[precision]);
    if (qtile <= 0)
      return fail(KDE_EINVAL, "the split BF16 scan needs d <= %d", kMaxSplitDim);
    {
      StageTimer t(ix, ST_PLAN, st, 9);
      launch_plan_pairs(s.probes, nc, P, ix->list_off, L, s.q_count, s.q_real, s.q_off, s.seg_off,
                        s.list_cnt, s.bucket_off, s.bucket_fill, s.pair_q, s.pair_dst,
                        s.tile_cnt, s.tile_off, ix->lorder, qtile, st);
      launch_select_order(s.probes, nc, P, L, s.ord_cnt, s.ord_off, s.ord_fill, s.order, st);
    }
    ScanPlan plan;
    plan.pair_q = s.pair_q;
    plan.pair_dst = s.pair_dst;
    plan.bucket_off = s.bucket_off;
    plan.tile_off = s.tile_off;
    plan.lorder = ix->lorder;
    plan.max_tiles = (nc * P + qtile - 1) / qtile + L;
    if (tcore) {
      StageTimer t(ix, ST_SCAN, st, 1);
      if (!launch_scan_tc(split, split ? ix->tmap_xls : ix->tmap_xlb, Yc, ix->C, ix->dp,
                          split ? ix->XLsn : ix->XLcn, ix->n, ix->list_off, L, ix->dpb, qtile,
                          plan, s.cand, ix->err, st))
        return fail(KDE_ECUDA, "could not configure the tensor-core scan kernel");
    } else {
      StageTimer t(ix, ST_SCAN, st, 1);
      launch_scan_simt(Yc, Ync, ix->XL, ix->XLn, ix->list_off, L, ix->dp, plan, s.cand, st);
    }
    StageTimer tsel(ix, ST_SELECT, st, 1);
    SelectArgs a;
    a.order = s.order;
    a.active = active;
    a.q0 = q0;
    a.cand = s.cand;
    a.q_off = s.q_off;
    a.q_count = s.q_count;
    a.q_real = s.q_real;
    a.seg_off = s.seg_off;
    a.probes = s.probes;
    a.P = P;
    a.list_off = ix->list_off;
    a.XL = ix->XL;
    a.XLn = ix->XLn;
    a.perm = ix->perm;
    a.X = ix->X;
    a.n = ix->n;
    a.xmax = ix->xmax;
    a.Y = Yc;
    a.Yn = Ync;
    a.nq = nc;
    a.d = ix->d;
    a.dp = ix->dp;
    a.k = k;
    a.kern = ix->kern;
    a.h = ix->h;
    a.err_scale = scan_err_scale(ix->dp, ix->dpb, precision);
    a.nbr = nbr + q0 * k;
    a.nd2 = nd2 ? nd2 + q0 * k : nullptr;
    a.s1 = s1 ? s1 + q0 : nullptr;
    a.kcount = nullptr;
    a.probe_d2 = s.probe_d2;
    a.rad = ix->rad;
    a.centered = tcore ? 1 : 0;
    a.rescore = split ? 0 : 1;
    // dpb / 16 units of 2^-24 per unit of (|x~| + |y~|)^2, one per MMA along a
    // row: 2 to 2.5 times the largest D^2 error measured for the split scan on
    // GB300 (1.9e-7 r^2 at d = 128, 6.1e-7 r^2 at d = 300), and s1 kept
    // unrescored up to a relative error of 8e-6
    a.XLsn = ix->XLsn;
    a.acc_scale = (float)ix->dpb / 16.0f / 16777216.0f;
    a.acc_tol = 8e-6f;
    a.ids_only = ids_only && nd2 == nullptr ? 1 : 0;
    a.err = ix->err;
    launch_select_neighbors(a, st);
  }
  CK(cudaGetLastError());
  return KDE_OK;
}

SampleArgs sample_args(kde_index* ix, const CallBufs& cb, int64_t nq, const int32_t* nbr, int k,
                       int m, uint64_t seed, const kde_opts* o) {
  SampleArgs a;
  a.X = ix->X;
  a.n = ix->n;
  a.d = ix->d;
  a.dp = ix->dp;
  a.kern = ix->kern;
  a.h = ix->h;
  a.Y = cb.Yp;
  a.nq = nq;
  a.nbr = nbr;
  a.k = k;
  a.m = m;
  a.seed = seed;
  a.qid_offset = o->query_id_offset;
  a.dev_qid = reinterpret_cast<const uint64_t*>(o->dev_query_id_offset);
  a.active = nullptr;
  a.mode = o->sample_mode;
  a.XP = ix->XP;
  a.wperm = ix->wperm;
  a.wpinv = ix->wpinv;
  a.nbr_distinct = 0;
  a.win_period = window_period(ix->n, m);
  a.s1_in = nullptr;
  a.kcount_in = nullptr;
  a.out = nullptr;
  a.samples = nullptr;
  a.rs = 0;
  a.loo = 0;
  a.gout = nullptr;
  a.dY = nullptr;
  a.dlogh = nullptr;
  a.err = ix->err;
  return a;
}

kde_status check_index(const kde_index* ix) {
  if (ix == nullptr) return fail(KDE_EINVAL, "index is NULL");
  return KDE_OK;
}

kde_status check_opts(const kde_opts* o) {
  if (o->precision < KDE_PREC_FP32 || o->precision > KDE_PREC_BF16X3)
    return fail(KDE_EINVAL, "precision must be 0 (FP32), 1 (BF16) or 2 (BF16 x3 split)");
  if (o->sample_mode < 0 || o->sample_mode > 2)
    return fail(KDE_EINVAL, "sample_mode must be 0 (reject), 1 (drop) or 2 (permuted window)");
  if (o->exact_path < 0 || o->exact_path > 2)
    return fail(KDE_EINVAL, "exact_path must be 0 (auto), 1 (CUDA cores) or 2 (tensor cores)");
  return KDE_OK;
}

// Decides the space of a call from Y and checks the other arrays agree.
kde_status call_space(const kde_index* ix, const void* Y, std::initializer_list<const void*> others,
                      bool* host) {
  const Space s = space_of(Y, ix->device);
  if (s == SPACE_FOREIGN) return fail(KDE_ESTATE, "Y lives on another device than the index");
  for (const void* p : others) {
    if (p == nullptr) continue;
    if (space_of(p, ix->device) != s)
      return fail(KDE_EINVAL, "all arrays of a call must be host or all device pointers");
  }
  *host = (s == SPACE_HOST);
  return KDE_OK;
}

kde_status copy_out(void* dst, const void* src, size_t bytes, bool host, cudaStream_t st) {
  if (bytes == 0) return KDE_OK;
  CK(cudaMemcpyAsync(dst, src, bytes, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     st));
  return KDE_OK;
}

kde_status finish_call(kde_index* ix, bool host, cudaStream_t st) {
  CK(cudaGetLastError());
  if (!host) return KDE_OK;
  int64_t margin = 0;
  kde_status s = collect_errors(ix, st, &margin);
  ix_margin_accumulate(ix, margin);
  return s;
}

// The estimator of a query call: per-query gathers (k_estimate); the phased
// order (draws, window-by-window gathers, finish) when X is several L2-sized
// windows; or, for permuted windows that many queries of the batch share, the
// tiled window path (prep, tiles, finish).
void run_estimate(kde_index* ix, const CallBufs& cb, const SampleArgs& a, cudaStream_t st) {
  if (a.mode == 0 && a.k > 0 && a.rs == 0 && a.loo == 0 && a.s1_in != nullptr &&
      a.out != nullptr && a.samples == nullptr && a.m > 0 && a.m <= kPhasedMaxM &&
      cb.ph.P > 0 && cb.ph_ids != nullptr) {
    StageTimer t(ix, ST_ESTIMATE, st, 3);
    PhaseArgs ph;
    ph.P = cb.ph.P;
    ph.shift = cb.ph.shift;
    ph.ids = cb.ph_ids;
    ph.off = cb.ph_off;
    ph.info = cb.ph_info;
    ph.part = cb.ph_part;
    launch_estimate_phased(a, ph, st);
    return;
  }
  if (a.mode == 2 && a.m > 0 && a.out != nullptr && a.samples == nullptr &&
      cb.win_part != nullptr) {
    StageTimer t(ix, ST_ESTIMATE, st, 3);
    const int dstride = std::max(a.k, 1);
    launch_window_prep(a, cb.win_drops, dstride, cb.win_dcnt, cb.win_kk, cb.win_s1, st);
    WindowTileArgs w;
    w.Y = a.Y;
    w.dp = a.dp;
    w.nq = a.nq;
    w.XP = a.XP;
    w.n = a.n;
    w.m = a.m;
    w.p = cb.win;
    w.qid_offset = a.qid_offset;
    w.dev_qid = a.dev_qid;
    w.drops = cb.win_drops;
    w.dstride = dstride;
    w.dcnt = cb.win_dcnt;
    w.kern = a.kern;
    w.h = a.h;
    w.part = cb.win_part;
    launch_window_tile(w, st);
    launch_window_finish(a, cb.win, cb.win_dcnt, cb.win_kk, cb.win_s1, cb.win_part, st);
    return;
  }
  StageTimer t(ix, ST_ESTIMATE, st, 1);
  launch_estimate(a, st);
}

}  // namespace

void deann::set_last_error(const char* msg) { g_err = msg; }

// ============================================================================
extern "C" {

const char* kde_strerror(kde_status s) {
  switch (s) {
    case KDE_OK: return "success";
    case KDE_EINVAL: return "invalid argument";
    case KDE_ENOMEM: return "out of device memory";
    case KDE_ECUDA: return "CUDA runtime error";
    case KDE_ELIMIT: return "draw cap reached";
    case KDE_ESTATE: return "invalid state";
  }
  return "unknown status";
}

const char* kde_last_error(void) { return g_err.c_str(); }

kde_status kde_build(const float* X, int64_t n, int32_t d, kde_kernel kernel, float h,
                     int32_t nlist, uint64_t seed, const kde_opts* opts, kde_index** out) {
  if (out == nullptr) return fail(KDE_EINVAL, "out is NULL");
  *out = nullptr;
  const kde_opts* o = opts ? opts : &kDefaultOpts;
  TRY(check_opts(o));
  if (X == nullptr) return fail(KDE_EINVAL, "X is NULL");
  if (n < 1 || n > INT32_MAX) return fail(KDE_EINVAL, "n must be in [1, 2^31 - 1]");
  if (d < 1 || d > kMaxDim) return fail(KDE_EINVAL, "d must be in [1, %d]", kMaxDim);
  if (!(h > 0.f) || !std::isfinite(h)) return fail(KDE_EINVAL, "h must be positive and finite");
  if (kernel != KDE_GAUSSIAN && kernel != KDE_EXPONENTIAL && kernel != KDE_LAPLACIAN)
    return fail(KDE_EINVAL, "unknown kernel");
  if (nlist < 1 || (int64_t)nlist > n || nlist > 8192)
    return fail(KDE_EINVAL, "nlist must be in [1, min(n, 8192)]");
  const int iters = o->kmeans_iters > 0 ? o->kmeans_iters : 20;
  cudaStream_t st = stream_of(o);

  kde_index* ix = new kde_index();
  CK(cudaGetDevice(&ix->device));
  const Space xs = space_of(X, ix->device);
  if (xs == SPACE_FOREIGN) {
    delete ix;
    return fail(KDE_ESTATE, "X lives on another device");
  }
  ix->n = n;
  ix->d = d;
  ix->dp = padded_dim(d);
  ix->dpb = (d + 63) & ~63;
  ix->nlist = nlist;
  ix->kern = (int)kernel;
  ix->h = h;
  ix->seed = seed;
  const int64_t L = nlist;
  kde_status s = KDE_OK;
  auto bail = [&](kde_status st2) {
    kde_free(ix);
    return st2;
  };
#define BTRY(expr)                      \
  do {                                  \
    kde_status s2_ = (expr);            \
    if (s2_ != KDE_OK) return bail(s2_); \
  } while (0)
#define BCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return bail(fail(KDE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)));    \
  } while (0)

  BTRY(dev_alloc(&ix->X, (size_t)n * ix->dp));
  BTRY(dev_alloc(&ix->Xn, (size_t)n));
  BTRY(dev_alloc(&ix->XL, (size_t)n * ix->dp));
  BTRY(dev_alloc(&ix->XLn, (size_t)n));
  BTRY(dev_alloc(&ix->perm, (size_t)n));
  BTRY(dev_alloc(&ix->assign, (size_t)n));
  BTRY(dev_alloc(&ix->list_off, (size_t)L + 1));
  BTRY(dev_alloc(&ix->C, (size_t)L * ix->dp));
  BTRY(dev_alloc(&ix->Cn, (size_t)L));
  BTRY(dev_alloc(&ix->XLcn, (size_t)n));
  BTRY(dev_alloc(&ix->rad, (size_t)L));
  BTRY(dev_alloc(&ix->err, 4));
  BTRY(dev_alloc(&ix->xmax_d, 2));
  BCK(cudaMemsetAsync(ix->xmax_d, 0, 2 * sizeof(float), st));
  {
    uint16_t* b = nullptr;
    BTRY(dev_alloc(&b, (size_t)n * ix->dpb));
    ix->XLb = b;
  }
  BCK(cudaMemsetAsync(ix->err, 0, 4 * sizeof(uint32_t), st));

  // build scratch
  const int64_t nchunks = (n + 2047) / 2048;
  Bump cnt;
  cnt.take<float>((size_t)n * d);  // staging copy of a host X
  cnt.take<float>(n);              // best_d2
  cnt.take<float>(n);              // tmp_d2
  cnt.take<int64_t>((size_t)L * nchunks);
  cnt.take<int32_t>(L);            // empty flags
  cnt.take<uint32_t>((n + 31) / 32 + 1);
  cnt.take<int32_t>(L);            // chosen
  cnt.take<int64_t>(L);            // counts
  cnt.take<double>((size_t)col_mean_slices(n) * ix->dp);  // column-mean partials
  const size_t amin_keys = (size_t)2 * n * (L > 1 ? assign_tc_slices(n, (int)L) : 1);
  cnt.take<unsigned long long>(amin_keys);                 // assignment keys
  BTRY(ensure_scratch(ix, cnt.used));
  Bump b;
  b.base = ix->scratch.base;
  float* stage = b.take<float>((size_t)n * d);
  float* best_d2 = b.take<float>(n);
  float* tmp_d2 = b.take<float>(n);
  int64_t* chunk_hist = b.take<int64_t>((size_t)L * nchunks);
  int32_t* empty = b.take<int32_t>(L);
  uint32_t* bitmap = b.take<uint32_t>((n + 31) / 32 + 1);
  int32_t* chosen = b.take<int32_t>(L);
  int64_t* counts = b.take<int64_t>(L);
  double* colpart = b.take<double>((size_t)col_mean_slices(n) * ix->dp);
  unsigned long long* amin = b.take<unsigned long long>(amin_keys);

  const float* src = X;
  if (xs == SPACE_HOST) {
    BCK(cudaMemcpyAsync(stage, X, sizeof(float) * n * d, cudaMemcpyHostToDevice, st));
    src = stage;
  }
  launch_pad_rows(src, n, d, ix->X, ix->dp, st);
  launch_row_norms(ix->X, n, ix->dp, ix->Xn, st);
  launch_max_f32(ix->Xn, n, ix->xmax_d, st);

  // the dataset mean: the centre of the tensor-core operands (coarse
  // quantiser, exact KDE, k-means assignment)
  BTRY(dev_alloc(&ix->mean, (size_t)ix->dp));
  launch_col_mean(ix->X, n, ix->dp, ix->mean, colpart, st);
  {
    uint16_t* cs = nullptr;
    BTRY(dev_alloc(&cs, (size_t)3 * L * ix->dpb));
    ix->Cs = cs;
    BTRY(dev_alloc(&ix->csn, (size_t)L));
    ix->cs_ok = make_parts_map(ix->tmap_cs, ix->Cs, 3 * L, ix->dpb);
  }
  if (kernel != KDE_LAPLACIAN) {
    // the rows minus the mean split into three BF16 parts: exact KDE and the
    // k-means assignment on the tensor cores
    BTRY(dev_alloc(&ix->xsn, (size_t)n));
    uint16_t* xs = nullptr;
    BTRY(dev_alloc(&xs, (size_t)3 * n * ix->dpb));
    ix->Xs = xs;
    launch_split3(ix->X, n, ix->dp, ix->mean, ix->Xs, n, ix->dpb, ix->xsn, st);
    ix->xs_ok = make_parts_map(ix->tmap_xs, ix->Xs, 3 * n, ix->dpb);
    launch_max_f32(ix->xsn, n, ix->xmax_d + 1, st);
  }
  // Lloyd's assignment step: nearest centroid by the split tensor-core
  // distances when the split rows exist, else by FP32 CUDA-core tiles
  const bool tc_assign = ix->xs_ok && ix->cs_ok;
  auto assign_step = [&]() -> bool {
    if (!tc_assign) {
      launch_assign_simt(ix->X, n, ix->C, (int)L, d, ix->dp, ix->assign, best_d2, st);
      return true;
    }
    launch_split3(ix->C, L, ix->dp, ix->mean, ix->Cs, L, ix->dpb, ix->csn, st);
    return launch_assign_tc(ix->tmap_xs, ix->xsn, n, ix->tmap_cs, ix->csn, (int)L, ix->dpb,
                            ix->X, ix->C, d, ix->dp, amin, ix->assign, best_d2, ix->err, st);
  };
  if (L == 1) {
    launch_fill_i32(ix->assign, n, 0, st);
  } else {
    launch_kmeans_init(ix->X, n, ix->dp, (int)L, seed, bitmap, chosen, ix->C, ix->err, st);
    for (int it = 0; it < iters; ++it) {
      if (!assign_step()) return bail(fail(KDE_ECUDA, "could not configure the k-means assignment"));
      launch_list_hist(ix->assign, n, (int)L, counts, st);
      launch_exclusive_scan_i64(counts, L, ix->list_off, st);
      launch_stable_scatter(ix->assign, n, (int)L, ix->list_off, chunk_hist, ix->perm, st);
      launch_centroid_update(ix->X, ix->dp, ix->perm, ix->list_off, (int)L, ix->C, empty, st);
      launch_reseed_empty(ix->X, n, ix->dp, best_d2, empty, (int)L, ix->C, tmp_d2, st);
    }
    if (!assign_step()) return bail(fail(KDE_ECUDA, "could not configure the k-means assignment"));
  }
  launch_list_hist(ix->assign, n, (int)L, counts, st);
  launch_exclusive_scan_i64(counts, L, ix->list_off, st);
  launch_stable_scatter(ix->assign, n, (int)L, ix->list_off, chunk_hist, ix->perm, st);
  if (L == 1) launch_centroid_update(ix->X, ix->dp, ix->perm, ix->list_off, 1, ix->C, empty, st);
  launch_row_norms(ix->C, L, ix->dp, ix->Cn, st);
  launch_gather_rows(ix->X, ix->dp, ix->perm, n, ix->XL, st);
  launch_gather_f32(ix->Xn, ix->perm, n, ix->XLn, st);
  launch_center_bf16(ix->XL, ix->dp, ix->list_off, (int)L, ix->C, ix->XLb, ix->dpb, ix->XLcn,
                     ix->rad, st);
  ix->tmap_ok = make_bf16_row_map(ix->tmap_xlb, ix->XLb, n, ix->dpb);
  if (ix->dpb <= kMaxSplitDim) {
    // the split copy of the centred rows for the FP32-accurate scan
    uint16_t* xls = nullptr;
    BTRY(dev_alloc(&xls, (size_t)3 * n * ix->dpb));
    ix->XLs = xls;
    BTRY(dev_alloc(&ix->XLsn, (size_t)n));
    launch_center_split3(ix->XL, ix->dp, n, ix->list_off, (int)L, ix->C, ix->XLs, ix->dpb,
                         ix->XLsn, st);
    ix->xls_ok = make_parts_map(ix->tmap_xls, ix->XLs, 3 * n, ix->dpb);
  }
  // the final centroids' split parts (the tensor-core coarse quantiser)
  launch_split3(ix->C, L, ix->dp, ix->mean, ix->Cs, L, ix->dpb, ix->csn, st);
  BCK(cudaGetLastError());

  ix->h_list_off = new int64_t[L + 1];
  BCK(cudaMemcpyAsync(ix->h_list_off, ix->list_off, sizeof(int64_t) * (L + 1),
                      cudaMemcpyDeviceToHost, st));
  float maxes[2] = {0.f, 0.f};  // max |x|^2, max |x - mean|^2
  BCK(cudaMemcpyAsync(maxes, ix->xmax_d, 2 * sizeof(float), cudaMemcpyDeviceToHost, st));
  const float xmax2 = maxes[0];
  ix->xs_max2 = maxes[1];
  BCK(cudaStreamSynchronize(st));
  ix->xmax = std::sqrt(xmax2);
  ix->max_list = 0;
  for (int64_t l = 0; l < L; ++l)
    ix->max_list = std::max(ix->max_list, ix->h_list_off[l + 1] - ix->h_list_off[l]);
  {
    // the scans take the lists longest first, so that the longest (the
    // slowest tiles) do not start last and leave a tail
    std::vector<int32_t> order(L);
    for (int l = 0; l < L; ++l) order[l] = l;
    const int64_t* lo = ix->h_list_off;
    std::stable_sort(order.begin(), order.end(), [lo](int32_t a, int32_t b) {
      return lo[a + 1] - lo[a] > lo[b + 1] - lo[b];
    });
    BTRY(dev_alloc(&ix->lorder, (size_t)L));
    BCK(cudaMemcpy(ix->lorder, order.data(), sizeof(int32_t) * L, cudaMemcpyHostToDevice));
  }
  int64_t margin = 0;
  s = collect_errors(ix, st, &margin);
  if (s == KDE_ELIMIT) s = KDE_OK;  // k-means init fell back to fixed points
  if (s != KDE_OK) return bail(s);
#undef BTRY
#undef BCK
  *out = ix;
  return KDE_OK;
}

kde_status kde_index_view(kde_index* ix, kde_index** out) {
  if (out == nullptr) return fail(KDE_EINVAL, "out must not be NULL");
  *out = nullptr;
  TRY(check_index(ix));
  if (ix->base != nullptr) return fail(KDE_EINVAL, "a view of a view: take the view of its base");
  DeviceGuard g(ix->device);
  kde_index* v = new kde_index(*ix);
  // shared: the dataset copies, the inverted file, tensor maps, the permuted
  // copy; the view's own: scratch, error words, statistics and profiling
  v->base = ix;
  v->scratch = deann::Arena();
  v->retired.clear();
  v->events.clear();
  v->prof = false;
  v->margin_failures = 0;
  for (int i = 0; i < kde_index::kStages; ++i) v->launches[i] = v->calls[i] = 0;
  v->err = nullptr;
  if (dev_alloc(&v->err, 4) != KDE_OK || cudaMemset(v->err, 0, 4 * sizeof(uint32_t)) !=
                                             cudaSuccess) {
    cudaFree(v->err);
    delete v;
    return fail(KDE_ENOMEM, "could not allocate the view's error words");
  }
  *out = v;
  return KDE_OK;
}

void kde_free(kde_index* ix) {
  if (ix == nullptr) return;
  DeviceGuard g(ix->device);
  cudaDeviceSynchronize();
  if (ix->base != nullptr) {  // a view frees only what is its own
    cudaFree(ix->err);
    if (ix->scratch.base) cudaFree(ix->scratch.base);
    for (char* p : ix->retired) cudaFree(p);
    for (const auto& e : ix->events) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    delete ix;
    return;
  }
  cudaFree(ix->X);
  cudaFree(ix->Xn);
  cudaFree(ix->XL);
  cudaFree(ix->XLn);
  cudaFree(ix->XLb);
  cudaFree(ix->XLs);
  cudaFree(ix->XLsn);
  cudaFree(ix->Cs);
  cudaFree(ix->csn);
  cudaFree(ix->perm);
  cudaFree(ix->assign);
  cudaFree(ix->lorder);
  cudaFree(ix->list_off);
  cudaFree(ix->C);
  cudaFree(ix->Cn);
  cudaFree(ix->XLcn);
  cudaFree(ix->rad);
  cudaFree(ix->mean);
  cudaFree(ix->Xs);
  cudaFree(ix->xsn);
  cudaFree(ix->err);
  cudaFree(ix->xmax_d);
  cudaFree(ix->wperm);
  cudaFree(ix->wpinv);
  cudaFree(ix->XP);
  if (ix->scratch.base) cudaFree(ix->scratch.base);
  for (char* p : ix->retired) cudaFree(p);
  for (const auto& e : ix->events) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  delete[] ix->h_list_off;
  delete ix;
}

kde_status kde_prepare_permuted(kde_index* ix, int32_t* perm_out, const kde_opts* opts) {
  if (ix != nullptr && ix->base != nullptr && ix->XP == nullptr)
    return fail(KDE_ESTATE, "prepare the permuted copy on the base index before taking views");
  TRY(check_index(ix));
  const kde_opts* o = opts ? opts : &kDefaultOpts;
  TRY(check_opts(o));
  DeviceGuard g(ix->device);
  cudaStream_t st = stream_of(o);
  if (ix->wperm == nullptr) {
    int32_t* wp = nullptr;
    int32_t* wi = nullptr;
    float* xp = nullptr;
    TRY(dev_alloc(&wp, (size_t)ix->n));
    if (dev_alloc(&wi, (size_t)ix->n) != KDE_OK || dev_alloc(&xp, (size_t)ix->n * ix->dp) != KDE_OK) {
      cudaFree(wp);
      cudaFree(wi);
      return fail(KDE_ENOMEM, "no room for the permuted dataset copy (%lld x %d floats)",
                  (long long)ix->n, ix->dp);
    }
    launch_feistel_perm(ix->seed, ix->n, wp, st);
    launch_invert_perm(wp, ix->n, wi, st);
    launch_gather_rows(ix->X, ix->dp, wp, ix->n, xp, st);
    CK(cudaGetLastError());
    ix->wperm = wp;
    ix->wpinv = wi;
    ix->XP = xp;
  }
  if (perm_out == nullptr) return KDE_OK;
  const Space sp = space_of(perm_out, ix->device);
  if (sp == SPACE_FOREIGN) return fail(KDE_ESTATE, "perm_out lives on another device");
  const bool host = sp == SPACE_HOST;
  TRY(copy_out(perm_out, ix->wperm, sizeof(int32_t) * ix->n, host, st));
  return finish_call(ix, host, st);
}

kde_status kde_set_bandwidth(kde_index* ix, float h) {
  TRY(check_index(ix));
  if (!(h > 0.f) || !std::isfinite(h)) return fail(KDE_EINVAL, "h must be positive and finite");
  ix->h = h;
  return KDE_OK;
}

kde_status kde_set_scan_tile(kde_index* ix, int32_t precision, int32_t tile) {
  TRY(check_index(ix));
  if (precision != KDE_PREC_BF16 && precision != KDE_PREC_BF16X3)
    return fail(KDE_EINVAL, "the scan tile is set for precision 1 (BF16) or 2 (BF16 x3 split)");
  if (tile != 0 && (tile < 16 || tile > 128 || tile % 16 != 0))
    return fail(KDE_EINVAL, "the scan tile must be 0 or a multiple of 16 in [16, 128]");
  ix->scan_tile[precision] = tile;
  return KDE_OK;
}

kde_status kde_set_phase_window(kde_index* ix, int64_t bytes) {
  TRY(check_index(ix));
  if (bytes < 0) return fail(KDE_EINVAL, "the phase window must be 0 (off) or a byte count");
  ix->phase_bytes = bytes;
  return KDE_OK;
}

kde_status kde_index_info(const kde_index* ix, int64_t* n, int32_t* d, int32_t* nlist,
                          int32_t* kernel, float* h, int64_t* max_list) {
  TRY(check_index(ix));
  if (n) *n = ix->n;
  if (d) *d = ix->d;
  if (nlist) *nlist = ix->nlist;
  if (kernel) *kernel = ix->kern;
  if (h) *h = ix->h;
  if (max_list) *max_list = ix->max_list;
  return KDE_OK;
}

kde_status kde_export_ivf(kde_index* ix, float* centroids, int32_t* assign) {
  TRY(check_index(ix));
  DeviceGuard g(ix->device);
  if (centroids)
    CK(cudaMemcpy2D(centroids, sizeof(float) * ix->d, ix->C, sizeof(float) * ix->dp,
                    sizeof(float) * ix->d, (size_t)ix->nlist, cudaMemcpyDeviceToHost));
  if (assign)
    CK(cudaMemcpy(assign, ix->assign, sizeof(int32_t) * ix->n, cudaMemcpyDeviceToHost));
  return KDE_OK;
}

static kde_status check_search_args(const kde_index* ix, int64_t nq, int32_t k, int32_t nprobe) {
  if (nq < 0 || nq > INT32_MAX) return fail(KDE_EINVAL, "nq must be in [0, 2^31 - 1]");
  if (k < 1 || k > kMaxK || (int64_t)k > ix->n)
    return fail(KDE_EINVAL, "k must be in [1, min(n, %d)]", kMaxK);
  if (nprobe < 1 || nprobe > ix->nlist || nprobe > kMaxProbe)
    return fail(KDE_EINVAL, "nprobe must be in [1, min(nlist, %d)]", kMaxProbe);
  return KDE_OK;
}

kde_status kde_search(kde_index* ix, const float* Y, int64_t nq, int32_t k, int32_t nprobe,
                      int32_t* nbr, float* d2, const kde_opts* opts) {
  TRY(check_index(ix));
  const kde_opts* o = opts ? opts : &kDefaultOpts;
  TRY(check_opts(o));
  TRY(check_search_args(ix, nq, k, nprobe));
  if (nq == 0) return KDE_OK;
  if (Y == nullptr || nbr == nullptr) return fail(KDE_EINVAL, "Y and nbr must not be NULL");
  DeviceGuard g(ix->device);
  bool host = false;
  TRY(call_space(ix, Y, {nbr, d2}, &host));
  cudaStream_t st = stream_of(o);
  CallShape c;
  c.nq = nq;
  c.k = k;
  c.P = nprobe;
  c.search = true;
  c.host = host;
  c.need_nbr = host;
  c.need_nd2 = host && d2 != nullptr;
  CallBufs cb;
  TRY(prepare_call(ix, c, cb));
  TRY(stage_queries(ix, Y, nq, host, cb, st));
  int32_t* nb = host ? cb.nbr : nbr;
  float* dd = host ? cb.nd2 : d2;
  TRY(run_search(ix, cb, nq, k, nprobe, o->precision, nb, dd, nullptr, st));
  if (host) {
    TRY(copy_out(nbr, nb, sizeof(int32_t) * nq * k, true, st));
    if (d2) TRY(copy_out(d2, dd, sizeof(float) * nq * k, true, st));
  }
  return finish_call(ix, host, st);
}

static kde_status check_est_args(const kde_index* ix, int64_t nq, int32_t k, int32_t m,
                                 const kde_opts* o) {
  if (nq < 0 || nq > INT32_MAX) return fail(KDE_EINVAL, "nq must be in [0, 2^31 - 1]");
  if (k < 0 || k > kMaxK) return fail(KDE_EINVAL, "k must be in [0, %d]", kMaxK);
  if (m < 0) return fail(KDE_EINVAL, "m must be >= 0");
  if ((int64_t)m * 64 + 4096 > INT32_MAX) return fail(KDE_EINVAL, "m too large");
  if (o->sample_mode == 2) {
    if (ix->wperm == nullptr || ix->XP == nullptr)
      return fail(KDE_ESTATE, "sample_mode 2 needs kde_prepare_permuted on the index first");
    if ((int64_t)m > ix->n) return fail(KDE_EINVAL, "sample_mode 2 needs m <= n");
  }
  return KDE_OK;
}

kde_status kde_query(kde_index* ix, const float* Y, int64_t nq, int32_t k, int32_t m,
                     int32_t nprobe, uint64_t seed, float* out, int32_t* nbr,
                     const kde_opts* opts) {
  TRY(check_index(ix));
  const kde_opts* o = opts ? opts : &kDefaultOpts;
  TRY(check_opts(o));
  TRY(check_est_args(ix, nq, k, m, o));
  if (k > 0) {
    TRY(check_search_args(ix, nq, k, nprobe));
  } else if (m < 1) {
    return fail(KDE_EINVAL, "k = 0 needs m >= 1");
  }
  if (nq == 0) return KDE_OK;
  if (Y == nullptr || out == nullptr) return fail(KDE_EINVAL, "Y and out must not be NULL");
  DeviceGuard g(ix->device);
  bool host = false;
  TRY(call_space(ix, Y, {out, nbr}, &host));
  cudaStream_t st = stream_of(o);
  CallShape c;
  c.nq = nq;
  c.k = k;
  c.m = m;
  c.P = nprobe;
  c.search = k > 0;
  c.host = host;
  c.need_out = host;
  c.need_nbr = k > 0 && (host || nbr == nullptr);
  c.need_s1 = k > 0;
  c.window = o->sample_mode == 2;
  CallBufs cb;
  TRY(prepare_call(ix, c, cb));
  TRY(stage_queries(ix, Y, nq, host, cb, st));
  int32_t* nb = (k > 0) ? ((host || nbr == nullptr) ? cb.nbr : nbr) : nullptr;
  const int64_t* active = reinterpret_cast<const int64_t*>(o->dev_active_rows);
  if (k > 0)
    TRY(run_search(ix, cb, nq, k, nprobe, o->precision, nb, nullptr, cb.s1, st, true, active));
  SampleArgs a = sample_args(ix, cb, nq, nb, k, m, seed, o);
  a.active = active;
  a.s1_in = k > 0 ? cb.s1 : nullptr;
  a.nbr_distinct = 1;
  a.out = host ? cb.out : out;
  a.rs = k == 0 ? 1 : 0;
  run_estimate(ix, cb, a, st);
  if (host) {
    TRY(copy_out(out, cb.out, sizeof(float) * nq, true, st));
    if (nbr && k > 0) TRY(copy_out(nbr, nb, sizeof(int32_t) * nq * k, true, st));
  }
  return finish_call(ix, host, st);
}

kde_status kde_query_with_neighbors(kde_index* ix, const float* Y, int64_t nq,
                                    const int32_t* nbr, int32_t k, int32_t m, uint64_t seed,
                                    float* out, const kde_opts* opts) {
  TRY(check_index(ix));
  const kde_opts* o = opts ? opts : &kDefaultOpts;
  TRY(check_opts(o));
  TRY(check_est_args(ix, nq, k, m, o));
  if (nq == 0) return KDE_OK;
  if (Y == nullptr || out == nullptr || (k > 0 && nbr == nullptr))
    return fail(KDE_EINVAL, "Y, out (and nbr when k > 0) must not be NULL");
  DeviceGuard g(ix->device);
  bool host = false;
  TRY(call_space(ix, Y, {out, k > 0 ? nbr : nullptr}, &host));
  cudaStream_t st = stream_of(o);
  CallShape c;
  c.nq = nq;
  c.k = k;
  c.m = m;
  c.host = host;
  c.need_out = host;
  c.need_nbr = host && k > 0;
  c.window = o->sample_mode == 2;
  CallBufs cb;
  TRY(prepare_call(ix, c, cb));
  TRY(stage_queries(ix, Y, nq, host, cb, st));
  const int32_t* nb = nbr;
  if (host && k > 0) {
    CK(cudaMemcpyAsync(cb.nbr, nbr, sizeof(int32_t) * nq * k, cudaMemcpyHostToDevice, st));
    nb = cb.nbr;
  }
  SampleArgs a = sample_args(ix, cb, nq, k > 0 ? nb : nullptr, k, m, seed, o);
  a.out = host ? cb.out : out;
  run_estimate(ix, cb, a, st);
  if (host) TRY(copy_out(out, cb.out, sizeof(float) * nq, true, st));
  return finish_call(ix, host, st);
}

kde_status kde_query_rs(kde_index* ix, const float* Y, int64_t nq, int32_t m, uint64_t seed,
                        float* out, const kde_opts* opts) {
  TRY(check_index(ix));
  if (m < 1) return fail(KDE_EINVAL, "m must be >= 1");
  TRY(check_opts(opts ? opts : &kDefaultOpts));
  kde_opts o2 = opts ? *opts : kDefaultOpts;
  if (o2.sample_mode != 2) o2.sample_mode = 0;  // with no X_1, reject = drop = plain RS
  return kde_query_with_neighbors(ix, Y, nq, nullptr, 0, m, seed, out, &o2);
}

kde_status kde_exact(kde_index* ix, const float* Y, int64_t nq, float* out,
                     const kde_opts* opts) {
  TRY(check_index(ix));
  const kde_opts* o = opts ? opts : &kDefaultOpts;
  TRY(check_opts(o));
  if (nq < 0 || nq > INT32_MAX) return fail(KDE_EINVAL, "nq must be in [0, 2^31 - 1]");
  if (nq == 0) return KDE_OK;
  if (Y == nullptr || out == nullptr) return fail(KDE_EINVAL, "Y and out must not be NULL");
  DeviceGuard g(ix->device);
  bool host = false;
  TRY(call_space(ix, Y, {out}, &host));
  cudaStream_t st = stream_of(o);
  CallShape c;
  c.nq = nq;
  c.host = host;
  c.need_out = host;
  c.exact = true;
  bool tcore = false;
  if (o->exact_path == 2) {
    if (!ix->xs_ok) return fail(KDE_EINVAL, "tensor-core exact KDE needs a Euclidean kernel");
    tcore = true;
  } else if (o->exact_path == 0) {
    // accuracy guard (see kde_exact in the header)
    tcore = ix->xs_ok && ix->kern == KDE_KERN_GAUSSIAN &&
            ix->xs_max2 <= 8.0f * 2.0f * ix->h * ix->h;
  }
  c.exact_tc = tcore;
  CallBufs cb;
  TRY(prepare_call(ix, c, cb));
  TRY(stage_queries(ix, Y, nq, host, cb, st));
  float* o_d = host ? cb.out : out;
  if (tcore) {
    StageTimer t(ix, ST_EXACT, st, 3);
    launch_split3(cb.Yp, nq, ix->dp, ix->mean, cb.Ys, nq, ix->dpb, cb.ysn, st);
    if (!launch_exact_tc(ix->tmap_xs, cb.Ys, cb.ysn, nq, nq, ix->xsn, ix->n, ix->dpb, ix->kern,
                         ix->h, cb.acc, o_d, ix->err, st))
      return fail(KDE_ECUDA, "could not configure the tensor-core exact kernel");
  } else {
    StageTimer t(ix, ST_EXACT, st, 2);
    launch_exact_simt(cb.Yp, cb.Yn, nq, ix->X, ix->Xn, ix->n, ix->d, ix->dp, ix->kern, ix->h,
                      cb.acc, o_d, st);
  }
  if (host) TRY(copy_out(out, cb.out, sizeof(float) * nq, true, st));
  return finish_call(ix, host, st);
}

kde_status kde_sample_indices(kde_index* ix, int64_t nq, const int32_t* nbr, int32_t k,
                              int32_t m, uint64_t seed, int32_t* samples, const kde_opts* opts) {
  TRY(check_index(ix));
  const kde_opts* o = opts ? opts : &kDefaultOpts;
  TRY(check_opts(o));
  TRY(check_est_args(ix, nq, k, m, o));
  if (nq == 0 || m == 0) return KDE_OK;
  if (samples == nullptr || (k > 0 && nbr == nullptr))
    return fail(KDE_EINVAL, "samples (and nbr when k > 0) must not be NULL");
  DeviceGuard g(ix->device);
  bool host = false;
  TRY(call_space(ix, samples, {k > 0 ? nbr : nullptr}, &host));
  cudaStream_t st = stream_of(o);
  CallShape c;
  c.nq = nq;
  c.k = k;
  c.m = m;
  c.host = host;
  c.need_nbr = host && k > 0;
  c.need_samples = host;
  CallBufs cb;
  TRY(prepare_call(ix, c, cb));
  const int32_t* nb = nbr;
  if (host && k > 0) {
    CK(cudaMemcpyAsync(cb.nbr, nbr, sizeof(int32_t) * nq * k, cudaMemcpyHostToDevice, st));
    nb = cb.nbr;
  }
  // the estimator kernel stages a query row; give it zeros
  CK(cudaMemsetAsync(cb.Yp, 0, sizeof(float) * nq * ix->dp, st));
  SampleArgs a = sample_args(ix, cb, nq, k > 0 ? nb : nullptr, k, m, seed, o);
  a.samples = host ? cb.samples : samples;
  {
    StageTimer t(ix, ST_ESTIMATE, st, 1);
    launch_estimate(a, st);
  }
  if (host) TRY(copy_out(samples, cb.samples, sizeof(int32_t) * nq * m, true, st));
  return finish_call(ix, host, st);
}

kde_status kde_grad_with_neighbors(kde_index* ix, const float* Y, int64_t nq,
                                   const int32_t* nbr, int32_t k, int32_t m, uint64_t seed,
                                   const float* gout, float* out, float* dY, float* dlogh,
                                   const kde_opts* opts) {
  TRY(check_index(ix));
  const kde_opts* o = opts ? opts : &kDefaultOpts;
  TRY(check_opts(o));
  TRY(check_est_args(ix, nq, k, m, o));
  if (ix->d > 1024) return fail(KDE_EINVAL, "the adjoint supports d <= 1024");
  if (o->sample_mode == 2) return fail(KDE_EINVAL, "the adjoint supports sample_mode 0 and 1");
  if (nq == 0) return KDE_OK;
  if (Y == nullptr || dY == nullptr || (k > 0 && nbr == nullptr))
    return fail(KDE_EINVAL, "Y, dY (and nbr when k > 0) must not be NULL");
  if (k == 0 && m == 0) return fail(KDE_EINVAL, "k = 0 needs m >= 1");
  DeviceGuard g(ix->device);
  bool host = false;
  TRY(call_space(ix, Y, {k > 0 ? nbr : nullptr, gout, out, dY, dlogh}, &host));
  cudaStream_t st = stream_of(o);
  CallShape c;
  c.nq = nq;
  c.k = k;
  c.m = m;
  c.host = host;
  c.need_out = host && out != nullptr;
  c.need_nbr = host && k > 0;
  c.grad = host;
  CallBufs cb;
  TRY(prepare_call(ix, c, cb));
  TRY(stage_queries(ix, Y, nq, host, cb, st));
  const int32_t* nb = nbr;
  const float* go = gout;
  if (host) {
    if (k > 0) {
      CK(cudaMemcpyAsync(cb.nbr, nbr, sizeof(int32_t) * nq * k, cudaMemcpyHostToDevice, st));
      nb = cb.nbr;
    }
    if (gout) {
      CK(cudaMemcpyAsync(cb.gout, gout, sizeof(float) * nq, cudaMemcpyHostToDevice, st));
      go = cb.gout;
    }
  }
  SampleArgs a = sample_args(ix, cb, nq, k > 0 ? nb : nullptr, k, m, seed, o);
  a.gout = go;
  a.out = host ? (out ? cb.out : nullptr) : out;
  a.dY = host ? cb.dY : dY;
  a.dlogh = host ? (dlogh ? cb.dlogh : nullptr) : dlogh;
  {
    StageTimer t(ix, ST_GRAD, st, 1);
    launch_estimate_grad(a, st);
  }
  if (host) {
    TRY(copy_out(dY, cb.dY, sizeof(float) * nq * ix->d, true, st));
    if (out) TRY(copy_out(out, cb.out, sizeof(float) * nq, true, st));
    if (dlogh) TRY(copy_out(dlogh, cb.dlogh, sizeof(float) * nq, true, st));
  }
  return finish_call(ix, host, st);
}

kde_status kde_grad(kde_index* ix, const float* Y, int64_t nq, int32_t k, int32_t m,
                    int32_t nprobe, uint64_t seed, const float* gout, float* dY, float* dlogh,
                    const kde_opts* opts) {
  TRY(check_index(ix));
  const kde_opts* o = opts ? opts : &kDefaultOpts;
  TRY(check_opts(o));
  TRY(check_est_args(ix, nq, k, m, o));
  if (ix->d > 1024) return fail(KDE_EINVAL, "the adjoint supports d <= 1024");
  if (o->sample_mode == 2) return fail(KDE_EINVAL, "the adjoint supports sample_mode 0 and 1");
  if (k > 0) {
    TRY(check_search_args(ix, nq, k, nprobe));
  } else if (m < 1) {
    return fail(KDE_EINVAL, "k = 0 needs m >= 1");
  }
  if (nq == 0) {
    if (dlogh == nullptr) return KDE_OK;
    // an empty batch: dlogh = 0 in the space of the pointer
    DeviceGuard g(ix->device);
    const Space sp = space_of(dlogh, ix->device);
    if (sp == SPACE_FOREIGN) return fail(KDE_ESTATE, "dlogh lives on another device");
    if (sp == SPACE_HOST) {
      *dlogh = 0.f;
      return KDE_OK;
    }
    CK(cudaMemsetAsync(dlogh, 0, sizeof(float), stream_of(o)));
    return KDE_OK;
  }
  if (Y == nullptr || dY == nullptr) return fail(KDE_EINVAL, "Y and dY must not be NULL");
  DeviceGuard g(ix->device);
  bool host = false;
  TRY(call_space(ix, Y, {gout, dY, dlogh}, &host));
  cudaStream_t st = stream_of(o);
  CallShape c;
  c.nq = nq;
  c.k = k;
  c.m = m;
  c.P = nprobe;
  c.search = k > 0;
  c.host = host;
  c.need_nbr = k > 0;
  c.need_out = true;
  c.grad = true;
  CallBufs cb;
  TRY(prepare_call(ix, c, cb));
  TRY(stage_queries(ix, Y, nq, host, cb, st));
  // X_1: the same search kde_query runs (a deterministic function of the
  // queries, the index, k, nprobe and the scan precision)
  if (k > 0)
    TRY(run_search(ix, cb, nq, k, nprobe, o->precision, cb.nbr, nullptr, nullptr, st, true));
  const float* go = gout;
  if (host && gout) {
    CK(cudaMemcpyAsync(cb.gout, gout, sizeof(float) * nq, cudaMemcpyHostToDevice, st));
    go = cb.gout;
  }
  SampleArgs a = sample_args(ix, cb, nq, k > 0 ? cb.nbr : nullptr, k, m, seed, o);
  a.rs = k == 0 ? 1 : 0;
  a.nbr_distinct = 1;
  a.gout = go;
  a.out = cb.out;
  a.dY = host ? cb.dY : dY;
  a.dlogh = cb.dlogh;
  {
    StageTimer t(ix, ST_GRAD, st, dlogh ? 2 : 1);
    launch_estimate_grad(a, st);
    // dlogh = sum over the queries of gout[q] d out[q] / d log h
    if (dlogh) launch_sum_to_scalar(cb.dlogh, nq, host ? cb.out : dlogh, st);
  }
  if (host) {
    TRY(copy_out(dY, cb.dY, sizeof(float) * nq * ix->d, true, st));
    if (dlogh) TRY(copy_out(dlogh, cb.out, sizeof(float), true, st));
  }
  return finish_call(ix, host, st);
}

kde_status kde_mean_shift(kde_index* ix, float* Y, int64_t nq, int32_t steps, int32_t k,
                          int32_t m, int32_t nprobe, uint64_t seed, float* est,
                          const kde_opts* opts) {
  TRY(check_index(ix));
  const kde_opts* o = opts ? opts : &kDefaultOpts;
  TRY(check_opts(o));
  TRY(check_est_args(ix, nq, k, m, o));
  if (ix->kern != KDE_KERN_GAUSSIAN)
    return fail(KDE_EINVAL, "mean shift is defined here for the Gaussian kernel");
  if (ix->d > 1024) return fail(KDE_EINVAL, "the adjoint supports d <= 1024");
  if (steps < 0) return fail(KDE_EINVAL, "steps must be >= 0");
  if (o->sample_mode == 2) return fail(KDE_EINVAL, "mean shift supports sample_mode 0 and 1");
  if (k > 0) {
    TRY(check_search_args(ix, nq, k, nprobe));
  } else if (m < 1) {
    return fail(KDE_EINVAL, "k = 0 needs m >= 1");
  }
  if (nq == 0) return KDE_OK;
  if (Y == nullptr) return fail(KDE_EINVAL, "Y must not be NULL");
  DeviceGuard g(ix->device);
  bool host = false;
  TRY(call_space(ix, Y, {est}, &host));
  cudaStream_t st = stream_of(o);
  CallShape c;
  c.nq = nq;
  c.k = k;
  c.m = m;
  c.P = nprobe;
  c.search = k > 0;
  c.host = host;
  c.need_out = true;
  c.need_nbr = k > 0;
  c.grad = true;
  CallBufs cb;
  TRY(prepare_call(ix, c, cb));
  TRY(stage_queries(ix, Y, nq, host, cb, st));
  if (steps == 0) CK(cudaMemsetAsync(cb.out, 0, sizeof(float) * nq, st));
  for (int s = 0; s < steps; ++s) {
    if (s > 0) {
      StageTimer t(ix, ST_STAGE, st, 1);
      launch_query_norms(cb.Yp, nq, ix->dp, cb.Yn, st);
    }
    // X_1 and S are redrawn at every step: the step's seed is seed + step
    if (k > 0)
      TRY(run_search(ix, cb, nq, k, nprobe, o->precision, cb.nbr, nullptr, nullptr, st, true));
    SampleArgs a = sample_args(ix, cb, nq, k > 0 ? cb.nbr : nullptr, k, m, seed + (uint64_t)s, o);
    a.rs = k == 0 ? 1 : 0;
    a.out = cb.out;
    a.dY = cb.dY;
    {
      StageTimer t(ix, ST_GRAD, st, 2);
      launch_estimate_grad(a, st);
      launch_mean_shift_update(cb.Yp, ix->dp, ix->d, cb.dY, cb.out, nq, ix->h, st);
    }
  }
  CK(cudaMemcpy2DAsync(Y, sizeof(float) * ix->d, cb.Yp, sizeof(float) * ix->dp,
                       sizeof(float) * ix->d, (size_t)nq,
                       host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  if (est) TRY(copy_out(est, cb.out, sizeof(float) * nq, host, st));
  return finish_call(ix, host, st);
}

kde_status kde_fit_bandwidth(kde_index* ix, const int32_t* zid, int64_t nz, int32_t k, int32_t m,
                             int32_t nprobe, uint64_t seed, int32_t iters, float lr,
                             float* h_trace, double* ll_trace, int32_t* nbr_out,
                             const kde_opts* opts) {
  TRY(check_index(ix));
  const kde_opts* o = opts ? opts : &kDefaultOpts;
  TRY(check_opts(o));
  if (o->sample_mode == 2)
    return fail(KDE_EINVAL, "bandwidth fitting supports sample_mode 0 and 1");
  if (nz < 1 || nz > INT32_MAX) return fail(KDE_EINVAL, "nz must be in [1, 2^31 - 1]");
  if (k < 0 || k > kMaxK - 1)
    return fail(KDE_EINVAL, "k must be in [0, %d] (X_1 holds the point and k neighbours)",
                kMaxK - 1);
  TRY(check_est_args(ix, nz, k + 1, m, o));
  if (k > 0) TRY(check_search_args(ix, nz, k, nprobe));
  if (ix->n < 2) return fail(KDE_EINVAL, "leave-one-out needs n >= 2");
  if (ix->d > 1024) return fail(KDE_EINVAL, "the adjoint supports d <= 1024");
  if (iters < 0) return fail(KDE_EINVAL, "iters must be >= 0");
  if (!std::isfinite(lr)) return fail(KDE_EINVAL, "lr must be finite");
  if (zid == nullptr || h_trace == nullptr) return fail(KDE_EINVAL, "zid and h_trace must not be NULL");
  DeviceGuard g(ix->device);
  const Space zs = space_of(zid, ix->device);
  if (zs == SPACE_FOREIGN) return fail(KDE_ESTATE, "zid lives on another device");
  cudaStream_t st = stream_of(o);
  std::vector<int32_t> hz((size_t)nz);
  if (zs == SPACE_HOST) {
    std::copy(zid, zid + nz, hz.begin());
  } else {
    CK(cudaMemcpyAsync(hz.data(), zid, sizeof(int32_t) * nz, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  for (int64_t j = 0; j < nz; ++j)
    if (hz[j] < 0 || (int64_t)hz[j] >= ix->n) return fail(KDE_EINVAL, "zid[%lld] out of range", (long long)j);
  CallShape c;
  c.nq = nz;
  c.k = k + 1;
  c.m = m;
  c.P = std::max(1, nprobe);
  c.search = k > 0;
  c.host = true;
  c.need_out = true;
  c.need_nbr = true;
  c.grad = true;
  c.fit_k = k;
  CallBufs cb;
  TRY(prepare_call(ix, c, cb));
  CK(cudaMemcpyAsync(cb.fit_zid, hz.data(), sizeof(int32_t) * nz, cudaMemcpyHostToDevice, st));
  {
    StageTimer t(ix, ST_STAGE, st, 2);
    launch_gather_rows(ix->X, ix->dp, cb.fit_zid, nz, cb.Yp, st);
    launch_query_norms(cb.Yp, nz, ix->dp, cb.Yn, st);
  }
  if (k > 0)
    TRY(run_search(ix, cb, nz, k, nprobe, o->precision, cb.fit_nbr, nullptr, nullptr, st, true));
  launch_prepend_self(cb.fit_zid, cb.fit_nbr, nz, k, cb.nbr, st);
  float h = ix->h;
  h_trace[0] = h;
  for (int t = 0; t < iters; ++t) {
    SampleArgs a = sample_args(ix, cb, nz, cb.nbr, k + 1, m, seed + (uint64_t)t, o);
    a.loo = 1;  // out, dlogh: the estimate over X \ {z} at z and its derivative
    a.out = cb.out;
    a.dY = cb.dY;
    a.dlogh = cb.dlogh;
    {
      StageTimer tm(ix, ST_GRAD, st, 2);
      launch_estimate_grad(a, st);
      launch_loo_reduce(cb.out, cb.dlogh, nz, cb.fit_red, st);
    }
    double red[3];
    CK(cudaMemcpyAsync(red, cb.fit_red, sizeof red, cudaMemcpyDeviceToHost, st));
    int64_t margin = 0;
    kde_status es = collect_errors(ix, st, &margin);  // synchronises the stream
    ix_margin_accumulate(ix, margin);
    if (es != KDE_OK) return es;
    if (red[2] < 1.0)
      return fail(KDE_EINVAL, "no training point keeps a held-out density at h = %g", (double)h);
    const double ll = red[0] / red[2] - (double)ix->d * std::log((double)h);
    const double gr = red[1] / red[2] - (double)ix->d;
    if (ll_trace) ll_trace[t] = ll;
    h = (float)std::exp(std::log((double)h) + (double)lr * gr);
    if (!(h > 0.f) || !std::isfinite(h)) return fail(KDE_EINVAL, "the step left h > 0 finite");
    ix->h = h;
    h_trace[t + 1] = h;
  }
  if (nbr_out) {
    const Space ns = space_of(nbr_out, ix->device);
    if (ns == SPACE_FOREIGN) return fail(KDE_ESTATE, "nbr_out lives on another device");
    TRY(copy_out(nbr_out, cb.nbr, sizeof(int32_t) * nz * (k + 1), ns == SPACE_HOST, st));
  }
  return finish_call(ix, true, st);
}

kde_status kde_sync(kde_index* ix, const kde_opts* opts) {
  TRY(check_index(ix));
  DeviceGuard g(ix->device);
  int64_t margin = 0;
  kde_status s = collect_errors(ix, stream_of(opts), &margin);
  ix_margin_accumulate(ix, margin);
  return s;
}

kde_status kde_stats(kde_index* ix, int64_t* margin_failures, const kde_opts* opts) {
  TRY(check_index(ix));
  DeviceGuard g(ix->device);
  int64_t margin = 0;
  kde_status s = collect_errors(ix, stream_of(opts), &margin);
  ix_margin_accumulate(ix, margin);
  if (margin_failures) *margin_failures = ix->margin_failures;
  return s;
}

kde_status kde_profile_enable(kde_index* ix, int32_t on) {
  TRY(check_index(ix));
  ix->prof = on != 0;
  return KDE_OK;
}

kde_status kde_profile_read(kde_index* ix, kde_profile* out, int32_t reset,
                            const kde_opts* opts) {
  TRY(check_index(ix));
  if (out == nullptr) return fail(KDE_EINVAL, "out is NULL");
  DeviceGuard g(ix->device);
  CK(cudaStreamSynchronize(stream_of(opts)));
  CK(cudaDeviceSynchronize());
  for (int s = 0; s < KDE_NUM_STAGES; ++s) {
    out->ms[s] = 0.0;
    out->timed[s] = 0;
    out->calls[s] = ix->calls[s];
    out->launches[s] = ix->launches[s];
  }
  for (const auto& e : ix->events) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
      out->ms[e.stage] += ms;
      out->timed[e.stage] += 1;
    }
  }
  if (reset) {
    for (const auto& e : ix->events) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    ix->events.clear();
    for (int s = 0; s < KDE_NUM_STAGES; ++s) ix->calls[s] = ix->launches[s] = 0;
  }
  return KDE_OK;
}

kde_status kde_reserve(kde_index* ix, int64_t nq, int32_t k, int32_t m, int32_t nprobe,
                       const kde_opts* opts) {
  TRY(check_index(ix));
  (void)opts;
  DeviceGuard g(ix->device);
  size_t need = 0;
  // variant 4: the largest batch whose sample sum still runs in the phased
  // order, whose sorted draws a smaller capture may need beyond nq's shapes
  for (int variant = 0; variant < 5; ++variant) {
    CallShape c;
    c.nq = variant == 4 ? std::min<int64_t>(nq, kPhasedMaxDraws / std::max(m, 1)) : nq;
    c.k = k;
    c.m = m;
    c.P = std::max(1, nprobe);
    c.search = k > 0;
    c.host = true;
    c.need_out = c.need_s1 = true;
    c.need_nbr = c.need_nd2 = k > 0;
    c.need_samples = variant == 1;
    c.grad = variant == 2;
    c.exact = variant == 3;
    c.exact_tc = variant == 3 && ix->xs_ok;
    c.window = variant == 0;  // sample_mode 2
    Bump cnt;
    CallBufs dummy;
    carve_call(cnt, ix, c, dummy);
    need = std::max(need, cnt.used);
  }
  return ensure_scratch(ix, need);
}

}  // extern "C"
