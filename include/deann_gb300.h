/*
 * deann_gb300.h -- C-ABI of the GB300 (sm_103a) kernel-density estimation
 * library implementing DEANN: Karppa, Aumueller, Pagh, "DEANN: Speeding up
 * Kernel-Density Estimation using Approximate Nearest Neighbor Search"
 * (arXiv 2107.02736).
 *
 * Problem statement (Section 2, Definition "Kernel Density Estimate"): for a
 * dataset X = {x_0, ..., x_{n-1}} in R^d, a kernel K_h with values in [0, 1]
 * and a query y, KDE_X(y) = (1/n) sum_i K_h(x_i, y).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are row-major FP32 with rows of d contiguous floats (no padding).
 *  - Pointer spaces: the array arguments of one call are either all host
 *    pointers or all device pointers of the index's GPU; the space of Y (X for
 *    kde_build) decides, and outputs are written in that same space.
 *    Host-pointer calls copy in, compute, copy out and synchronise the stream
 *    before returning.  Device-pointer calls only enqueue work on the stream
 *    and return KDE_OK once it is enqueued; an error a kernel detects while
 *    running (the draw cap, an out-of-range neighbour id) writes NaN into the
 *    affected outputs and is reported by the next kde_sync().
 *  - Ownership: the caller keeps every array it passes.  kde_build copies X;
 *    the index owns all device memory it allocates until kde_free.  Scratch
 *    memory is owned by the index and reused by its calls, so calls on one
 *    index must be ordered on one stream (or synchronised by the caller).
 *  - Streams: kde_opts.stream is a cudaStream_t (NULL: the legacy default
 *    stream).  A NULL kde_opts pointer means all-default options.
 *  - Errors: every entry point returns a kde_status; no call aborts or throws.
 *    kde_last_error() gives a message for the calling thread's last failure.
 *  - Random numbers: the sample S of a query is drawn from Philox4x32-10
 *    (Salmon et al., SC'11) with key (lo32(seed), hi32(seed)) and counter
 *    (t, lo32(qid), hi32(qid), 0), where qid = opts.query_id_offset + row and
 *    t = 0, 1, 2, ... is the draw number; index = floor(u n / 2^64) with
 *    u = (r1 << 32) | r0.  The same (X, Y, neighbours, seed, qid) always gives
 *    the same sample.
 */
#ifndef DEANN_GB300_H
#define DEANN_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kde_index kde_index;

/* Kernels (Section 1): Gaussian exp(-|x-y|_2^2 / (2h^2)), exponential
 * exp(-|x-y|_2 / h), Laplacian exp(-|x-y|_1 / h).  No normalising constant. */
typedef enum {
  KDE_GAUSSIAN = 0,
  KDE_EXPONENTIAL = 1,
  KDE_LAPLACIAN = 2
} kde_kernel;

typedef enum {
  KDE_OK = 0,
  KDE_EINVAL = 1, /* invalid argument (message in kde_last_error) */
  KDE_ENOMEM = 2, /* device allocation failed */
  KDE_ECUDA = 3,  /* a CUDA runtime call failed */
  KDE_ELIMIT = 4, /* a query needed more than 64 m + 4096 draws */
  KDE_ESTATE = 5  /* wrong device, or an earlier asynchronous error pending */
} kde_status;

/* Precision of the IVF scan's distance tiles.  The returned neighbour
 * distances and estimates are FP32-level whatever the scan used: the FP32 and
 * BF16 scans only rank candidates, and the best (every one within the scan's
 * rigorous error band of the k-th) are rescored with FP32 difference-form
 * distances; the split scan's distances are FP32-level themselves (operands
 * split into three BF16 parts, six partial products), so only the candidates
 * within its error band of the k-th distance are rescored, with compensated
 * FP32 difference-form distances, to settle the order there.  With the split
 * scan the neighbours' kernel values come from its distances; a query whose
 * neighbour sum could be off by more than 8e-6 relative (a per-candidate
 * error of 2^-24 (d_pad / 16) (|x - c| + |y - c|)^2 assumed) has its
 * neighbours' rows rescored in FP32, unless the FP32 difference form's own
 * bound on that sum is no smaller. */
typedef enum {
  KDE_PREC_FP32 = 0,  /* FP32 operands */
  KDE_PREC_BF16 = 1,  /* BF16 operands, FP32 accumulation, FP32 rescoring */
  KDE_PREC_BF16X3 = 2 /* three-part BF16 split operands, FP32 accumulation; d <= 1152 */
} kde_precision;

typedef struct {
  int32_t precision;        /* kde_precision of the scan (kde_query, kde_search) */
  int32_t sample_mode;      /* 0: reject draws in X_1 (default); 1: "drop";
                               2: permuted window (Algorithm 2, DEANNP /
                               RSP): needs kde_prepare_permuted and m <= n;
                               not for the adjoint or mean shift */
  int32_t kmeans_iters;     /* kde_build: Lloyd iterations (0 = 20) */
  int32_t exact_path;       /* kde_exact: 0 = automatic (tensor cores when
                               the accuracy guard below allows, else CUDA
                               cores); 1 = CUDA cores; 2 = tensor cores
                               (Gaussian and exponential kernels only) */
  uint64_t query_id_offset; /* qid of row r is query_id_offset + r */
  void* stream;             /* cudaStream_t, NULL = legacy default stream */
  const void* dev_query_id_offset; /* NULL, or a DEVICE pointer to a uint64
                               added to query_id_offset when the estimator
                               runs: a call captured in a CUDA graph then
                               serves a new batch (new sample streams) per
                               replay by rewriting this value */
  const void* dev_active_rows; /* kde_query only: NULL, or a DEVICE pointer
                               to an int64 A.  Rows 0 .. A-1 are the queries;
                               rows at or past A get no probes, no neighbours
                               and no samples: their nbr entries are -1 and
                               their out entries unspecified.  A call
                               captured in a CUDA graph at a fixed capacity
                               then serves a smaller batch per replay by
                               rewriting A; rows past A cost at most the
                               query-centroid distances of their tile of 128
                               rows */
} kde_opts;

/* kde_build -- build an index over X (Section 4: FAISS-style inverted file).
 *   X       n x d, host or device.  Copied; the caller keeps X.
 *   n >= 1, 1 <= d <= 4096.
 *   kernel  kde_kernel; h > 0 and finite is the bandwidth.
 *   nlist   number of IVF lists, 1 <= nlist <= min(n, 8192).  nlist = 1 makes
 *           every query scan all n points (brute-force kNN as the ANN).
 *           Otherwise k-means with nlist centroids (initial centroids: distinct
 *           points drawn from Philox stream 1 of `seed`; opts.kmeans_iters
 *           Lloyd iterations; empty lists reseeded with the point farthest from
 *           its centroid), then every point goes to the list of its nearest
 *           centroid, lists stored contiguously.
 *   out     receives the new index (NULL on failure).
 * Synchronous.  Errors: EINVAL, ENOMEM, ECUDA. */
kde_status kde_build(const float* X, int64_t n, int32_t d, kde_kernel kernel, float h,
                     int32_t nlist, uint64_t seed, const kde_opts* opts, kde_index** out);

/* kde_free -- release the index and all device memory it owns (NULL is a
 * no-op).  Synchronises the device first.  For a view (kde_index_view) only
 * the view's own memory is released. */
void kde_free(kde_index* index);

/* kde_index_view -- a second handle on the same index for concurrent work:
 * it shares the dataset copies, the inverted file and (when prepared first on
 * the index) the permuted copy of Algorithm 2, and has its own scratch
 * memory, device error words, statistics and profiling state, so calls on
 * different views may run on different streams at the same time.  The view
 * starts with the index's bandwidth; kde_set_bandwidth on either changes only
 * that handle.  The index must outlive its views; free each with kde_free.
 * Views of a view are refused (take another view of the index).
 * Errors: EINVAL, ENOMEM. */
kde_status kde_index_view(kde_index* index, kde_index** out);

/* kde_prepare_permuted -- Algorithm 2's preprocessing: a random permutation
 * pi of [0, n) and the permuted copy XP[i] = X[pi(i)] (n x d FP32 more device
 * memory), which opts.sample_mode = 2 reads.  pi is a 4-round Feistel network
 * on 2 hb bits (hb = ceil(b / 2), b the bit length of n - 1, at least 1),
 * round r (0..3) mapping (L, R) to (R, L xor F_r(R)) with F_r(R) the low hb bits
 * of word r0 of Philox4x32-10 at counter (R, r, 0, 3) and key (lo32(seed),
 * hi32(seed)) of the build seed, x = (L << hb) | R; values >= n are enciphered
 * again until they fall below n (cycle walking).
 * Permuted mode: the query with global id qid (see kde_opts) reads the m
 * consecutive rows of XP from ell = (qid m) mod n, wrapping at n (the running
 * index of Algorithm 2, advanced by m per query); entries in X_1 are dropped
 * and the m' kept ones give out = (1/n) [ sum_{X_1} K + ((n - k')/m') sum K ]
 * (sum_{X_1} K / n when m' = 0); with k = 0 (kde_query_rs) it is RSP.
 *   perm_out  NULL, or n int32 (host or device) receiving pi(0..n-1).
 * Idempotent (the permutation is built once).  Errors: ENOMEM, ECUDA. */
kde_status kde_prepare_permuted(kde_index* index, int32_t* perm_out, const kde_opts* opts);

/* kde_set_bandwidth -- replace h (> 0, finite).  The IVF does not depend on h. */
kde_status kde_set_bandwidth(kde_index* index, float h);

/* kde_set_scan_tile -- the most queries one tensor-core list-scan tile takes
 * (the MMA's N; the scan reads a probed list once per tile of its queries).
 *   precision  KDE_PREC_BF16 or KDE_PREC_BF16X3 (the FP32 scan's tiles are
 *              fixed).
 *   tile       0 = automatic (the most that the operands' shared memory
 *              holds, at most 128), or a multiple of 16 in [16, 128]; a value
 *              above the automatic one is capped to it.
 * The estimates, neighbour sets and distances do not depend on the tile (each
 * distance is the same sum whatever the grouping); only the speed does.  The
 * binding's KDEIndex.tune_scan_tile measures a few tiles on sample queries and
 * keeps the fastest.  A view starts with its index's tiles.
 * Errors: EINVAL. */
kde_status kde_set_scan_tile(kde_index* index, int32_t precision, int32_t tile);

/* kde_set_phase_window -- the bytes of X one phase of kde_query's estimator
 * reads (Algorithm 1's sample sum s2 regrouped by where its rows lie).  When
 * X is larger than the window and splits into at most 64 windows of a power
 * of two of rows each (the most that fit the window), m <= 8192 and
 * m >= 64 x the window count, kde_query draws every
 * query's sample first, sorts each query's draws stably by window, and then
 * gathers the rows window by window, so that the window being read stays in
 * L2 while all queries' rows in it are summed.  The draws, the rejection of
 * X_1 and the estimate are those of Algorithm 1 as in the per-query gathers;
 * only the order in which s2's terms are added differs (FP32 rounding).  The
 * choice does not depend on the batch size, so a query gets the same bits in
 * any batch, up to nq x m = 2^30 draws a call (4 GiB of sorted draws in the
 * index's scratch); larger batches take the per-query order.
 *   bytes  0 = off (per-query gathers always), else the window size; the
 *          default is 64 MiB (half the GPU's L2).
 * A view starts with its index's window.  Errors: EINVAL. */
kde_status kde_set_phase_window(kde_index* index, int64_t bytes);

/* kde_index_info -- any output pointer may be NULL. */
kde_status kde_index_info(const kde_index* index, int64_t* n, int32_t* d, int32_t* nlist,
                          int32_t* kernel, float* h, int64_t* max_list);

/* kde_export_ivf -- copy the IVF state to HOST memory so that the search can
 * be re-run elsewhere: centroids (nlist x d FP32), assign (n int32: the list
 * of each point, in the original point order).  Either may be NULL. */
kde_status kde_export_ivf(kde_index* index, float* centroids, int32_t* assign);

/* kde_search -- the ANN subroutine of Algorithm 1: the k nearest
 * points (Euclidean) among the lists of the nprobe nearest centroids.
 *   Y      nq x d queries; nq >= 0.
 *   k      1 <= k <= 2048; 1 <= nprobe <= min(nlist, 256).
 *   nbr    nq x k original point ids sorted by (distance, id); -1 pads rows
 *          with fewer than k candidates.
 *   d2     nq x k squared distances (FP32, difference form) or NULL; +inf pads.
 *          (With the split scan, passing d2 makes the call rescore the
 *          candidates' rows as the BF16 scan does.)
 * Candidates are ranked first by approximate distances from the scan (see
 * opts.precision); every candidate within the scan's error band of the k-th
 * is then rescored in FP32 difference form, which makes the set the exact
 * top k (ties at the k-th distance excepted). */
kde_status kde_search(kde_index* index, const float* Y, int64_t nq, int32_t k, int32_t nprobe,
                      int32_t* nbr, float* d2, const kde_opts* opts);

/* kde_query -- DEANN (Algorithm 1): X_1 = kde_search(y, k, nprobe); the
 * neighbours' contribution is summed exactly; S = m draws uniform on X \ X_1
 * (with repetition, by rejection of draws in X_1; or opts.sample_mode = 1);
 * out = (1/n) [ sum_{X_1} K + ((n - k')/m) sum_S K ] with k' = |X_1|.
 *   k      0 <= k <= min(n, 2048) (k = 0 is plain random sampling);
 *   m      >= 0 (m = 0 keeps only the neighbours' exact contribution);
 *   nprobe 1 <= nprobe <= min(nlist, 256) (ignored when k = 0).
 *   out    nq estimates (FP32).
 *   nbr    NULL, or nq x k receiving the neighbour ids that were used (the
 *          set X_1, in no particular order; -1 pads).
 * With opts.dev_active_rows only the rows below the device count are served
 * (a CUDA graph captured at a fixed capacity serving a smaller batch).
 * With k > 0 and sample_mode 0 on an X larger than the index's phase window
 * (kde_set_phase_window) the sample sum runs in the phased order, whose
 * scratch holds nq x m int32 sorted draws besides the search's. */
kde_status kde_query(kde_index* index, const float* Y, int64_t nq, int32_t k, int32_t m,
                     int32_t nprobe, uint64_t seed, float* out, int32_t* nbr,
                     const kde_opts* opts);

/* kde_query_with_neighbors -- the estimate of Algorithm 1 with a caller-supplied
 * neighbour set per query (nq x k ids; negative entries are padding,
 * duplicates count once; an id >= n is an error).  Same estimate as
 * kde_query. */
kde_status kde_query_with_neighbors(kde_index* index, const float* Y, int64_t nq,
                                    const int32_t* nbr, int32_t k, int32_t m, uint64_t seed,
                                    float* out, const kde_opts* opts);

/* kde_query_rs -- random sampling (Lemma RS): m >= 1 draws uniform on X with
 * repetition (the first m draws of each query's stream), out = mean kernel
 * value; with opts.sample_mode = 2, RSP (Algorithm 2): the mean over the
 * query's permuted window. */
kde_status kde_query_rs(kde_index* index, const float* Y, int64_t nq, int32_t m, uint64_t seed,
                        float* out, const kde_opts* opts);

/* kde_exact -- the exact KDE (Section 2 definition; the "Naive" evaluation of
 * Appendix D), out[q] = (1/n) sum_i K_h(x_i, y_q), FP64 accumulation across
 * the dataset.  Two implementations:
 *   CUDA cores: FP32 difference-form distances, any kernel;
 *   tensor cores (Gaussian, exponential): D^2 = |x|^2 + |y|^2 - 2<x, y> with
 *     both sides centred on the dataset mean and every operand split into
 *     three BF16 parts (six partial products, FP32 accumulation in TMEM).
 *     Its D^2 carries an absolute error near 2^-22 (|x - mean|^2 +
 *     |y - mean|^2) from the FP32 accumulator, so a kernel value's relative
 *     error is about that divided by 2h^2.
 * opts.exact_path 0 picks the tensor cores for the Gaussian kernel when
 * max_i |x_i - mean|^2 <= 8 (2 h^2) (in-distribution queries then stay near
 * 1e-6 relative error) and the CUDA cores otherwise, including for the
 * exponential kernel, whose derivative is unbounded at distance 0. */
kde_status kde_exact(kde_index* index, const float* Y, int64_t nq, float* out,
                     const kde_opts* opts);

/* kde_sample_indices -- the sample S that kde_query_with_neighbors uses for
 * each query (nq x m original ids): the accepted draws in draw order
 * (sample_mode 0), the raw draws (sample_mode 1), or the window's ids in
 * window order with -1 for the dropped members of X_1 (sample_mode 2).  Rows
 * with no sampling (k' = n or m = 0) are filled with -1. */
kde_status kde_sample_indices(kde_index* index, int64_t nq, const int32_t* nbr, int32_t k,
                              int32_t m, uint64_t seed, int32_t* samples, const kde_opts* opts);

/* kde_grad_with_neighbors -- adjoint of kde_query_with_neighbors with X_1 and
 * S held fixed (the pathwise derivative; the paper defines no gradient):
 *   out[q]   the estimate (as kde_query_with_neighbors), or NULL;
 *   dY[q]    gout[q] * d out[q] / d y_q (nq x d);
 *   dlogh[q] gout[q] * d out[q] / d log h, or NULL.
 * gout may be NULL (all ones).  Kernel values are recomputed from the
 * neighbour ids and the regenerated sample, never stored.  d <= 1024. */
kde_status kde_grad_with_neighbors(kde_index* index, const float* Y, int64_t nq,
                                   const int32_t* nbr, int32_t k, int32_t m, uint64_t seed,
                                   const float* gout, float* out, float* dY, float* dlogh,
                                   const kde_opts* opts);

/* kde_grad -- the adjoint of kde_query: runs the same IVF search for X_1
 * (k nearest among nprobe lists; none when k = 0) and the same sample S (seed,
 * query ids as in kde_query), then the pathwise derivative of Algorithm 1's
 * estimate with X_1 and S held fixed (the paper defines no gradient; X_1 is
 * piecewise constant in y and E_S[estimate | X_1] is the exact KDE, so the
 * derivative is unbiased for the KDE's almost everywhere):
 *   dY[q]   gout[q] * d out[q] / d y_q (nq x d);
 *   dlogh   NULL, or ONE float: sum_q gout[q] * d out[q] / d log h, summed on
 *           the device in FP64 in a fixed order and rounded once.
 * gout may be NULL (all ones).  The search is a deterministic function of
 * (Y, index, k, nprobe, opts.precision), so after kde_query with the same
 * arguments the sets are the ones that call used.  Limits as kde_query
 * (sample_mode 0 or 1), d <= 1024.  Errors: EINVAL, ELIMIT, ECUDA. */
kde_status kde_grad(kde_index* index, const float* Y, int64_t nq, int32_t k, int32_t m,
                    int32_t nprobe, uint64_t seed, const float* gout, float* dY, float* dlogh,
                    const kde_opts* opts);

/* kde_mean_shift -- density-gradient flow with the DEANN estimate (Gaussian
 * kernel only; the paper names gradient lines of densities as a use of KDE,
 * Section 1): `steps` updates y <- y + h^2 grad(KDE~)(y) / KDE~(y), which for
 * the Gaussian kernel move y to the estimate-weighted mean of its neighbour
 * and sample points.  Step s draws X_1 and S afresh with seed + s; the
 * gradient is the adjoint of kde_grad_with_neighbors.
 *   Y    nq x d, updated in place (host or device).
 *   est  NULL or nq: the estimate at the start of the last step.
 * Same argument limits as kde_query; d <= 1024. */
kde_status kde_mean_shift(kde_index* index, float* Y, int64_t nq, int32_t steps, int32_t k,
                          int32_t m, int32_t nprobe, uint64_t seed, float* est,
                          const kde_opts* opts);

/* kde_fit_bandwidth -- fit h by gradient ascent on the leave-one-out
 * log-likelihood of the normalised KDE (the paper sets h by bisection on a
 * target KDE value; this is the fitting loop that the estimator's derivative
 * in log h serves).  All three kernels normalise as a constant times h^d, so
 * up to a constant
 *   l(h) = mean_j log KDE_{-z_j}(z_j) - d log h,
 *   KDE_{-z}(z) = (n KDE(z) - 1) / (n - 1)            (K(z, z) = 1),
 *   dl/dlog h = mean_j (n / (n - 1)) dKDE(z_j)/dlog h / KDE_{-z_j}(z_j) - d,
 * with KDE and its derivative the DEANN estimate and its adjoint, X_1 of z_j =
 * {z_j} and its k nearest points from kde_search (so that the point's own
 * term is exact and the held-out value follows), samples drawn with
 * seed + t at iteration t and query ids j.  The library evaluates the
 * held-out estimate directly (the point's own term left out of the neighbour
 * sum, weights over n - 1 points), which is the same value without the
 * cancellation of n KDE - 1.  A point with no held-out density (every other
 * kernel value underflowed) is left out of the means.  Step:
 * log h <- log h + lr dl/dlog h (dl/dlog h grows with d: lr of order 1/d
 * keeps the steps stable); the index keeps the final h.
 *   zid       nz training point ids (rows of the indexed X), host or device.
 *   k         0 <= k <= 2047 search neighbours (nprobe as in kde_search).
 *   m         samples per training point (sample_mode 0 or 1).
 *   h_trace   HOST, iters + 1 floats: h before the first and after each step.
 *   ll_trace  HOST or NULL, iters doubles: l(h) before each step.
 *   nbr_out   NULL, or nz x (k + 1) ids (host or device): the X_1 rows used.
 * Synchronous.  Errors: EINVAL (arguments, no usable training point, a step
 * leaving h > 0 finite), ELIMIT, ECUDA. */
kde_status kde_fit_bandwidth(kde_index* index, const int32_t* zid, int64_t nz, int32_t k,
                             int32_t m, int32_t nprobe, uint64_t seed, int32_t iters, float lr,
                             float* h_trace, double* ll_trace, int32_t* nbr_out,
                             const kde_opts* opts);

/* kde_sync -- wait for the index's work on opts->stream and report (then
 * clear) errors raised by kernels of earlier device-pointer calls:
 * KDE_ELIMIT (draw cap), KDE_EINVAL (neighbour id >= n). */
kde_status kde_sync(kde_index* index, const kde_opts* opts);

/* kde_stats -- counters kept since the index was built: margin_failures =
 * queries whose rescored top-k could not be certified against the scan's
 * error bound (the neighbours returned are still valid points, possibly not
 * the exact top k).  Synchronises opts->stream. */
kde_status kde_stats(kde_index* index, int64_t* margin_failures, const kde_opts* opts);

/* kde_reserve -- pre-allocate scratch for calls with up to nq queries and the
 * given k, m, nprobe at opts->precision, so that later calls allocate nothing
 * (required before capturing calls into a CUDA graph).  A later call that
 * needs more scratch allocates a larger buffer; the outgrown one is kept
 * until kde_free, so graphs captured before stay valid. */
kde_status kde_reserve(kde_index* index, int64_t nq, int32_t k, int32_t m, int32_t nprobe,
                       const kde_opts* opts);

/* kde_exact_noalloc -- kde_exact for callers that may not allocate device
 * memory while they call (the paper has no counterpart; it is a deployment
 * aid).  A cudaMalloc inside a call is not an option while a CUDA graph is
 * being captured, when an application has reserved all device memory for its
 * own allocator, or in loops that cannot afford an allocation's implicit
 * synchronisation.  This variant allocates nothing: its FP64 accumulators live
 * in a fixed array of 65,536 doubles (512 KiB) inside the library, present on
 * every GPU that loads it for the life of the process.
 *   Y, out  DEVICE pointers of the index's GPU, which must be current; Y is
 *           nq x d with d a multiple of 4 and 16-byte aligned; out is nq.
 *   nq      0 <= nq <= 65536; larger batches are rejected with KDE_EINVAL.
 *   opts    only opts->stream is read (NULL: the legacy default stream).
 * It runs the CUDA-core path of kde_exact (FP32 difference-form distances,
 * any kernel), so it agrees with kde_exact(opts.exact_path = 1) and with the
 * default path within the FP32 tolerance.  The first call on a device looks
 * up the array's address (make it before any stream capture); the address is
 * kept for the process, so the call is not valid after cudaDeviceReset.
 * Calls share the array and clear it at their start, so calls that overlap on
 * the GPU race: order them on one stream.  Asynchronous like every
 * device-pointer call. */
kde_status kde_exact_noalloc(kde_index* index, const float* Y, int64_t nq, float* out,
                             const kde_opts* opts);

/* Per-stage device timing of an index's calls.  Stages: 0 query staging
 * (padding, norms), 1 coarse quantiser (probe selection), 2 scan work plan,
 * 3 IVF list scan, 4 candidate selection and rescoring, 5 estimator (sample
 * draws, gathers, combination), 6 exact KDE, 7 adjoint.  launches counts the
 * kernels each stage launched (always on); ms / timed are filled from CUDA
 * events recorded on the call's stream around every stage while profiling is
 * enabled. */
#define KDE_NUM_STAGES 8
typedef struct {
  double ms[KDE_NUM_STAGES];      /* total device time per stage */
  int64_t timed[KDE_NUM_STAGES];  /* timed stage executions */
  int64_t calls[KDE_NUM_STAGES];  /* stage executions */
  int64_t launches[KDE_NUM_STAGES];
} kde_profile;

/* kde_profile_enable -- on != 0 starts recording events for later calls. */
kde_status kde_profile_enable(kde_index* index, int32_t on);

/* kde_profile_read -- synchronises, sums the recorded times into *out and,
 * when reset != 0, clears the counters and events. */
kde_status kde_profile_read(kde_index* index, kde_profile* out, int32_t reset,
                            const kde_opts* opts);

/* kde_strerror -- static description of a status. */
const char* kde_strerror(kde_status status);

/* kde_last_error -- message of the calling thread's last failed call. */
const char* kde_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DEANN_GB300_H */
