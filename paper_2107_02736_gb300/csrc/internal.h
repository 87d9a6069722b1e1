// Internal declarations of the DEANN GB300 library: the index layout in HBM
// and the launchers each translation unit provides.  Not part of the C-ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#define KDE_KERN_GAUSSIAN 0
#define KDE_KERN_EXPONENTIAL 1
#define KDE_KERN_LAPLACIAN 2

// Device error word bits (index->err[0]); index->err[1] counts queries whose
// candidate margin could not be certified.
#define KDE_ERRBIT_DRAWCAP 1u
#define KDE_ERRBIT_BADNBR 2u
#define KDE_ERRBIT_MARGIN 4u
#define KDE_ERRBIT_TMA 8u

namespace deann {

constexpr int kMaxDim = 4096;        // largest supported d
constexpr int kMaxK = 2048;          // largest neighbour count k
constexpr int kMaxProbe = 256;       // largest nprobe
constexpr int kSelectCap = 4096;     // largest candidate count kept for rescoring
constexpr int kTile = 64;            // SIMT distance tile edge
constexpr int kMaxSplitDim = 1152;   // widest padded row of the split BF16 scan

// Row stride (in floats) of every FP32 row-major matrix: d rounded up to a
// multiple of 4 so rows start on 16-byte boundaries; padding is zero.
inline int padded_dim(int d) { return (d + 3) & ~3; }

// Raises a kernel's dynamic shared-memory limit on the current device.  The
// limit is a per-device attribute, and the 48 KB default counts static and
// dynamic shared memory together, so it is set before every launch that takes
// dynamic shared memory (one cheap driver call per launch).
inline bool set_dynamic_smem(const void* kernel, size_t bytes) {
  if (bytes == 0) return true;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes) == cudaSuccess;
}

// Bump allocator over one device buffer owned by an index.  Calls on one
// index are stream-ordered, so scratch is reused call after call.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  void reset() { used = 0; }
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (used + bytes > cap) return nullptr;
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

}  // namespace deann

struct kde_index {
  const kde_index* base = nullptr;  // non-null: a view sharing base's device data
  int device = 0;
  int64_t n = 0;
  int d = 0;
  int dp = 0;                 // padded row stride (floats)
  int dpb = 0;                // padded row stride of the BF16 copy (elements)
  int nlist = 1;
  int kern = 0;
  float h = 1.f;
  uint64_t seed = 0;
  // dataset, original order: X[n x dp] FP32 and squared norms
  float* X = nullptr;
  float* Xn = nullptr;
  // dataset, IVF list order (list-contiguous): FP32, BF16 and norms
  float* XL = nullptr;
  float* XLn = nullptr;
  void* XLb = nullptr;        // __nv_bfloat16 [n x dpb], rows centred on their centroid
  float* XLcn = nullptr;      // |x - c_list|^2 of each list-ordered row (FP32)
  float* rad = nullptr;       // [nlist] max |x - c_list| over the list
  int32_t* perm = nullptr;    // list position -> original id
  int32_t* assign = nullptr;  // original id -> list id
  int32_t* lorder = nullptr;  // [nlist] list ids, longest list first (scan order)
  int64_t* list_off = nullptr;  // [nlist + 1] device
  int64_t* h_list_off = nullptr;  // host copy
  int64_t max_list = 0;
  float* C = nullptr;         // centroids [nlist x dp]
  float* Cn = nullptr;
  // TMA descriptor (CUtensorMap, 128 bytes) of XLb: 64 x 128 BF16 boxes,
  // 128-byte swizzle
  alignas(64) unsigned char tmap_xlb[128] = {0};
  bool tmap_ok = false;
  // the same centred rows split into three BF16 parts [3][n][dpb] (the
  // FP32-accurate tensor-core scan), their FP64-accurate squared norms, and
  // the TMA descriptor of the parts
  void* XLs = nullptr;
  float* XLsn = nullptr;
  alignas(64) unsigned char tmap_xls[128] = {0};
  bool xls_ok = false;
  // exact KDE on tensor cores (Euclidean kernels): dataset mean, the rows
  // minus the mean split into three BF16 parts [3][n][dpb], their squared
  // norms, and the TMA descriptor of the parts
  float* mean = nullptr;
  void* Xs = nullptr;
  float* xsn = nullptr;
  alignas(64) unsigned char tmap_xs[128] = {0};
  bool xs_ok = false;
  float xs_max2 = 0.f;        // max |x - mean|^2 (accuracy guard of the tensor-core path)
  // the centroids minus the mean split into three BF16 parts [3][nlist][dpb],
  // their squared norms and TMA descriptor (the tensor-core coarse quantiser)
  void* Cs = nullptr;
  float* csn = nullptr;
  alignas(64) unsigned char tmap_cs[128] = {0};
  bool cs_ok = false;
  // permuted sampling (Algorithm 2): pi and the dataset in pi order,
  // XP[i] = X[pi(i)]; built by kde_prepare_permuted
  int32_t* wperm = nullptr;   // [n] window position -> original id
  int32_t* wpinv = nullptr;   // [n] original id -> window position (pi^-1)
  float* XP = nullptr;        // [n x dp]
  uint32_t* err = nullptr;    // device error words [4]
  float* xmax_d = nullptr;    // device max |x|^2
  float xmax = 0.f;           // max |x| over the dataset
  int64_t margin_failures = 0;
  int scan_tile[3] = {0, 0, 0};  // per precision: the tensor-core scan's query tile, 0 = automatic
  // bytes of X one phase of the phased estimator reads (an L2-sized window);
  // 0 turns the phased order off
  int64_t phase_bytes = int64_t(64) << 20;
  deann::Arena scratch;
  std::vector<char*> retired;  // outgrown scratch buffers, freed by kde_free
  size_t scratch_limit = size_t(16) << 30;
  // per-stage profiling (CUDA events on the call's stream) and launch counts
  static constexpr int kStages = 8;
  bool prof = false;
  struct EvPair {
    cudaEvent_t a, b;
    int stage;
  };
  std::vector<EvPair> events;
  int64_t launches[kStages] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t calls[kStages] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace deann {

// Sets the calling thread's kde_last_error() message (capi.cu).
void set_last_error(const char* msg);

// ---- build.cu -------------------------------------------------------------
void launch_row_norms(const float* X, int64_t n, int dp, float* out, cudaStream_t s);
void launch_pad_rows(const float* src, int64_t n, int d, float* dst, int dp, cudaStream_t s);
void launch_kmeans_init(const float* X, int64_t n, int dp, int L, uint64_t seed,
                        uint32_t* bitmap, int32_t* chosen, float* C, uint32_t* err, cudaStream_t s);
void launch_max_f32(const float* v, int64_t n, float* out, cudaStream_t s);
void launch_list_hist(const int32_t* assign, int64_t n, int L, int64_t* counts, cudaStream_t s);
void launch_exclusive_scan_i64(const int64_t* in, int64_t count, int64_t* out, cudaStream_t s);
void launch_stable_scatter(const int32_t* assign, int64_t n, int L, const int64_t* list_off,
                           int64_t* chunk_hist, int32_t* perm, cudaStream_t s);
void launch_centroid_update(const float* X, int dp, const int32_t* perm, const int64_t* list_off,
                            int L, float* C, int32_t* empty_flags, cudaStream_t s);
void launch_reseed_empty(const float* X, int64_t n, int dp, const float* best_d2,
                         int32_t* empty_flags, int L, float* C, float* tmp_d2, cudaStream_t s);
void launch_gather_rows(const float* X, int dp, const int32_t* ids, int64_t count, float* dst,
                        cudaStream_t s);
void launch_gather_f32(const float* v, const int32_t* ids, int64_t count, float* dst,
                       cudaStream_t s);
void launch_to_bf16(const float* X, int64_t n, int dp, void* dst, int dpb, cudaStream_t s);
void launch_center_bf16(const float* XL, int dp, const int64_t* list_off, int L, const float* C,
                        void* dst, int dpb, float* xcn, float* rad, cudaStream_t s);
void launch_fill_i32(int32_t* p, int64_t count, int32_t v, cudaStream_t s);
// three-way BF16 split of the list-centred rows, [3][n][dpb], and FP64 norms
void launch_center_split3(const float* XL, int dp, int64_t n, const int64_t* list_off, int L,
                          const float* C, void* dst, int dpb, float* xsn, cudaStream_t s);
void launch_feistel_perm(uint64_t seed, int64_t n, int32_t* out, cudaStream_t s);
void launch_invert_perm(const int32_t* perm, int64_t n, int32_t* inv, cudaStream_t s);

// ---- tiles.cu (SIMT distance tiles) ---------------------------------------
void launch_exact_simt(const float* Y, const float* Yn, int64_t nq, const float* X,
                       const float* Xn, int64_t n, int d, int dp, int kern, float h,
                       double* acc, float* out, cudaStream_t s);
void launch_assign_simt(const float* P, int64_t np, const float* C, int L, int d, int dp,
                        int32_t* assign, float* best_d2, cudaStream_t s);
// active / row0: rows row0 + q >= *active (when active is not NULL) are skipped
void launch_dist_matrix(const float* Y, const float* Yn, int64_t nq, const float* C,
                        const float* Cn, int L, int dp, float* D, const int64_t* active,
                        int64_t row0, cudaStream_t s);
struct ScanPlan {
  const int32_t* pair_q;      // query of each (query, probe) pair, bucketed by list
  const int64_t* pair_dst;    // destination offset of the pair's segment in cand
  const int64_t* bucket_off;  // [L + 1] pairs of list l: [bucket_off[l], bucket_off[l+1])
  const int64_t* tile_off;    // [L + 1] query tiles of the i-th list of lorder
  const int32_t* lorder;      // [L] lists in scan order, longest first
  int64_t max_tiles;          // grid bound
};
void launch_scan_simt(const float* Y, const float* Yn, const float* XL, const float* XLn,
                      const int64_t* list_off, int L, int dp, const ScanPlan& plan, float* cand,
                      cudaStream_t s);

// ---- tc_scan.cu (tcgen05 BF16 scan) ----------------------------------------
// Queries per CTA for a row width (0: the operands do not fit); split = the
// three-way BF16 split of both operands (tmap over [3][n][dpb], xn the FP64-
// accurate norms), else plain BF16 (tmap over [n][dpb]).
int scan_tc_bn(int dpb, bool split);
bool make_bf16_row_map(void* map_out, const void* base, int64_t rows, int dpb);
bool launch_scan_tc(bool split, const void* tmap, const float* Yp, const float* C, int dp,
                    const float* xn, int64_t n, const int64_t* list_off, int L, int dpb, int BN,
                    const ScanPlan& plan, float* cand, uint32_t* err, cudaStream_t s);

// ---- tc_exact.cu (tcgen05 exact KDE, three-way BF16 split) -----------------
// column means in FP64 over fixed row slices; part holds col_mean_slices(n) x dp
int col_mean_slices(int64_t n);
void launch_col_mean(const float* X, int64_t n, int dp, float* mean, double* part,
                     cudaStream_t s);
// D[q][c] for the coarse quantiser on tensor cores (split BF16, FP32-level):
// tmap_c over the centroids' parts [3][L][dpb] (centred on the dataset mean),
// Ys the queries' parts [3][nq][dpb]; rows row0 + q >= *active skipped
bool launch_coarse_tc(const void* tmap_c, const float* cn, int L, const void* Ys, const float* yn,
                      int64_t nq, int dpb, float* D, const int64_t* active, int64_t row0,
                      uint32_t* err, cudaStream_t s);
void launch_split3(const float* V, int64_t rows, int dp, const float* mean, void* dst,
                   int64_t rows_pad, int dpb, float* norms, cudaStream_t s);
bool make_parts_map(void* map_out, const void* base, int64_t rows_total, int dpb);
// k-means assignment on the tensor cores: for each point (its three BF16
// parts centred on the dataset mean behind tmap_p, squared norms pn) the two
// nearest centroids (parts behind tmap_c, norms cn) by the split distances,
// then the nearer of the two by FP32 difference-form distances between the
// rows X and C, ties to the lower id; amin is 2 np assign_tc_slices(np, L)
// keys of scratch.
int assign_tc_slices(int64_t np, int L);
bool launch_assign_tc(const void* tmap_p, const float* pn, int64_t np, const void* tmap_c,
                      const float* cn, int L, int dpb, const float* X, const float* C, int d,
                      int dp, unsigned long long* amin, int32_t* assign, float* best_d2,
                      uint32_t* err, cudaStream_t s);
bool launch_exact_tc(const void* tmap_x, const void* Ys, const float* yn, int64_t nq, int64_t nqp,
                     const float* xn, int64_t n, int dpb, int kern, float h, double* acc,
                     float* out, uint32_t* err, cudaStream_t s);

// ---- select.cu -------------------------------------------------------------
void launch_query_norms(const float* Y, int64_t nq, int dp, float* out, cudaStream_t s);
// active / q0: rows q0 + q >= *active (when active is not NULL) get no probes
void launch_select_probes(const float* D, int64_t nq, int L, const float* Y, int d, int dp,
                          const float* C, int nprobe, int margin, int32_t* probes,
                          float* probe_d2, const int64_t* active, int64_t q0, cudaStream_t s);
void launch_plan_pairs(const int32_t* probes, int64_t nq, int P, const int64_t* list_off, int L,
                       int64_t* q_count, int64_t* q_real, int64_t* q_off, int64_t* seg_off,
                       int64_t* list_cnt,
                       int64_t* bucket_off, int64_t* bucket_fill, int32_t* pair_q,
                       int64_t* pair_dst, int64_t* tile_cnt, int64_t* tile_off,
                       const int32_t* lorder, int qtile,
                       cudaStream_t s);
void launch_select_order(const int32_t* probes, int64_t nq, int P, int L, int64_t* ord_cnt,
                         int64_t* ord_off, int64_t* ord_fill, int32_t* order, cudaStream_t s);
struct SelectArgs {
  const int32_t* order;      // [nq] processing order (nullable: row order)
  const int64_t* active;     // device row count A (nullable): rows q0 + q >= A are skipped
  int64_t q0;                // row of this chunk's first query within the call
  const float* cand;
  const int64_t* q_off;
  const int64_t* q_count;    // padded candidate slots per query (+inf in the padding)
  const int64_t* q_real;     // candidates per query
  const int64_t* seg_off;    // [nq x P]
  const int32_t* probes;     // [nq x P]
  int P;
  const int64_t* list_off;
  const float* XL;
  const float* XLn;
  const int32_t* perm;
  const float* X;            // original order (Laplacian neighbour sums)
  int64_t n;                 // rows of X
  float xmax;                // max |x| over the dataset
  const float* Y;
  const float* Yn;
  int64_t nq;
  int d, dp;
  int k;
  int kern;
  float h;
  float err_scale;           // approx-distance error bound per unit of (|x| + |y|)^2
  int32_t* nbr;              // [nq x k] original ids, -1 pad
  float* nd2;                // [nq x k] precise squared distances (nullable)
  float* s1;                 // [nq] sum of kernel values over the k' neighbours (nullable)
  int32_t* kcount;           // [nq] k' (nullable)
  // centred scan (BF16): the error bound uses |y - c_probe| and list radii
  const float* probe_d2;     // [nq x P]
  const float* rad;          // [nlist]
  int centered;
  int ids_only;              // 1: the neighbour set in any order (+ s1); no nd2
  int rescore;               // 1: rescore the band's rows in FP32 (plain BF16 / FP32 scans);
                             // 0: the scan's values are FP32-level (split scan)
  const float* XLsn;         // split scan: |x - c_list|^2 of each list-ordered row
  float acc_scale;           // split scan: D^2 error per unit of r^2 assumed for kernel values
  float acc_tol;             // split scan: largest relative error of s1 used unrescored
  uint32_t* err;
};
void launch_select_neighbors(const SelectArgs& a, cudaStream_t s);

// ---- sample.cu --------------------------------------------------------------
struct SampleArgs {
  const float* X;            // original order
  int64_t n;
  int d, dp;
  int kern;
  float h;
  const float* Y;
  int64_t nq;
  const int32_t* nbr;        // [nq x k] or null (k = 0)
  int k;
  int m;
  uint64_t seed;
  uint64_t qid_offset;
  const uint64_t* dev_qid;   // optional device-side addition to qid_offset
  const int64_t* active;     // device row count A (nullable): rows q >= A are skipped
  int mode;                  // 0 reject, 1 drop, 2 permuted window (Algorithm 2)
  const float* XP;           // mode 2: the dataset in pi order
  const int32_t* wperm;      // mode 2: pi
  const int32_t* wpinv;      // mode 2: pi^-1
  int nbr_distinct;          // 1: nbr rows hold distinct ids or -1 (the search's output)
  int64_t win_period;        // mode 2: n / gcd(n, m), queries this far apart share a window
  const float* s1_in;        // precomputed neighbour sums (nullable)
  const int32_t* kcount_in;  // matching k' (nullable)
  float* out;                // [nq] estimates (nullable)
  int32_t* samples;          // [nq x m] sample indices (nullable)
  int rs;                    // 1: plain random sampling (ignore nbr)
  int loo;                   // adjoint: estimate KDE over X minus the row's first id, at it
  // adjoint
  const float* gout;         // [nq] (grad only)
  float* dY;                 // [nq x d] (grad only)
  float* dlogh;              // [nq] (grad only)
  uint32_t* err;
};
void launch_estimate(const SampleArgs& a, cudaStream_t s);

// ---- sample.cu: the phased estimator ----------------------------------------
// The sampled rows of a batch are gathered in P phases, phase p reading only
// rows [p W, (p + 1) W) of X (W a power of two), so that the window a phase reads stays in L2
// while every query's draws inside it are summed.  One kernel draws each
// query's m accepted indices and sorts them stably by window; a phase-major
// grid sums each (window, query) run; a last kernel combines the P partial
// sums in window order into the estimate.
constexpr int kMaxPhases = 64;       // more windows leave too few rows per run
constexpr int kMinPhaseRows = 64;    // at least this many rows per run on average
constexpr int kPhasedMaxM = 8192;    // the draws of a query sit in shared memory
constexpr int64_t kPhasedMaxDraws = int64_t(1) << 30;  // nq x m sorted draws: 4 GiB of scratch
constexpr int kPhaseWarps = 8;        // warps of a gather block: one partial each
struct PhasePlan {
  int P = 0;                 // windows; 0 = the per-query gathers instead
  int shift = 0;             // rows per window W = 2^shift (the last may be shorter)
};
PhasePlan phase_plan(int64_t n, int dp, int m, int64_t nq, int64_t window_bytes);
struct PhaseArgs {
  int P = 0;
  int shift = 0;             // row id -> window: id >> shift
  int32_t* ids = nullptr;    // [nq x m] accepted draws, sorted stably by window
  int32_t* off = nullptr;    // [nq x (P + 1)] start of each window's run; off[P] = m
  int32_t* info = nullptr;   // [nq] k' of the query, or -1 when it failed
  float* part = nullptr;     // [P x nq x kPhaseWarps] per-window, per-warp sums
};
// Needs a.mode == 0, a.k > 0, a.s1_in, a.out, no a.samples, not a.rs, and
// 0 < a.m <= kPhasedMaxM.
void launch_estimate_phased(const SampleArgs& a, const PhaseArgs& ph, cudaStream_t s);

// ---- window.cu + sample.cu: permuted windows shared by many queries --------
// Queries whose ids agree mod P = n / gcd(n, m) read the same window; a batch
// with nq = A P + B holds A or A + 1 queries per residue class.  With
// A >= kWindowMinShare the estimator runs as dense (queries x window rows)
// tiles instead of per-query gathers.
constexpr int64_t kWindowMinShare = 16;
struct WindowPlan {
  int64_t P = 1, A = 0, B = 0;
  int64_t groups = 0;        // min(P, nq) residue classes
  int Tq = 0;                // 64-query tiles per class
  int rs = 64;               // window positions per row slice (multiple of 64)
  int nslices = 0;
};
int64_t window_period(int64_t n, int64_t m);
WindowPlan window_plan(int64_t nq, int64_t n, int m);
bool window_tiled(const WindowPlan& p);
struct WindowTileArgs {
  const float* Y;            // [nq x dp] staged queries
  int dp;
  int64_t nq;
  const float* XP;           // permuted dataset
  int64_t n;
  int m;
  WindowPlan p;
  uint64_t qid_offset;
  const uint64_t* dev_qid;
  const int32_t* drops;      // [nq x dstride] sorted window positions of X_1 members
  int dstride;
  const int32_t* dcnt;       // [nq]
  int kern;
  float h;
  double* part;              // [nq x p.nslices] partial window sums
};
void launch_window_tile(const WindowTileArgs& w, cudaStream_t s);
// Per query: X_1 (sorted, deduplicated), s1 (unless a.s1_in), and the sorted
// window positions of X_1's members; kk[q] = -1 flags a bad neighbour id.
void launch_window_prep(const SampleArgs& a, int32_t* drops, int dstride, int32_t* dcnt,
                        int32_t* kk, float* s1, cudaStream_t s);
// out[q] = (s1 + ((n - k') / m') s2) / n with s2 the slice partials' sum.
void launch_window_finish(const SampleArgs& a, const WindowPlan& p, const int32_t* dcnt,
                          const int32_t* kk, const float* s1, const double* part,
                          cudaStream_t s);
void launch_estimate_grad(const SampleArgs& a, cudaStream_t s);
void launch_mean_shift_update(float* Yp, int dp, int d, const float* dY, const float* est,
                              int64_t nq, float h, cudaStream_t s);
// bandwidth fitting: X_1 rows [z, its k neighbours], and the leave-one-out sums
void launch_prepend_self(const int32_t* zid, const int32_t* nbr, int64_t nz, int k, int32_t* out,
                         cudaStream_t s);
void launch_loo_reduce(const float* loo, const float* dloo, int64_t nz, double* red,
                       cudaStream_t s);
// out[0] = sum of v[0..n) (FP64 in a fixed order, rounded once); one block
void launch_sum_to_scalar(const float* v, int64_t n, float* out, cudaStream_t s);

}  // namespace deann
