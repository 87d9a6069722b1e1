// kde_exact_noalloc: the exact KDE for callers that must not allocate device
// memory during the call.
//
// The exact-KDE kernel accumulates each query's partial sums from all slices
// of the dataset in an FP64 buffer.  kde_exact takes that buffer from the
// index's scratch pool, which grows with cudaMalloc when a call needs more.
// Some callers cannot let a call allocate: code that runs while a CUDA graph
// is being captured (a cudaMalloc there breaks the capture), programs whose
// device memory is fully reserved up front by their own allocator, or
// latency-critical loops where an allocation's implicit synchronisation is
// not acceptable.  For them this variant keeps the FP64 buffer in a
// fixed-size array in the library's own device memory instead.
//
// The array lives in every GPU that loads the library, for the life of the
// process.  Its device address is looked up once per device on the first call
// made with that device current; make that first call before any stream
// capture starts.  All calls share the one array, so calls whose kernels
// overlap on the GPU (different streams, or different host threads) race on
// it; keep calls on one stream, or synchronise between them.  The buffer is
// cleared at the start of every call.
#include <mutex>

#include "deann_gb300.h"
#include "internal.h"

using namespace deann;

namespace {

// Largest query count of one call: 65,536 FP64 accumulators (512 KiB).
constexpr int64_t kNoAllocMaxQueries = 65536;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_exact_acc[kNoAllocMaxQueries];

std::mutex g_mutex;
double* g_acc_ptr[kMaxDevices] = {nullptr};

kde_status noalloc_fail(kde_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

}  // namespace

extern "C" {

kde_status kde_exact_noalloc(kde_index* ix, const float* Y, int64_t nq, float* out,
                             const kde_opts* opts) {
  if (ix == nullptr) return noalloc_fail(KDE_EINVAL, "index is NULL");
  if (nq < 0 || nq > kNoAllocMaxQueries)
    return noalloc_fail(KDE_EINVAL, "nq must be in [0, 65536] for kde_exact_noalloc");
  if (nq == 0) return KDE_OK;
  if (Y == nullptr || out == nullptr) return noalloc_fail(KDE_EINVAL, "Y and out must not be NULL");
  if (ix->dp != ix->d)
    return noalloc_fail(KDE_EINVAL, "kde_exact_noalloc needs d to be a multiple of 4");
  if ((reinterpret_cast<uintptr_t>(Y) & 15u) != 0)
    return noalloc_fail(KDE_EINVAL, "Y must be 16-byte aligned");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return noalloc_fail(KDE_ECUDA, "cudaGetDevice failed");
  if (prev != ix->device) return noalloc_fail(KDE_ESTATE, "the index's device must be current");
  if (ix->device < 0 || ix->device >= kMaxDevices)
    return noalloc_fail(KDE_ESTATE, "device ordinal out of range");
  cudaPointerAttributes a;
  for (const void* p : {static_cast<const void*>(Y), static_cast<const void*>(out)}) {
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
        (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) ||
        a.device != ix->device) {
      cudaGetLastError();
      return noalloc_fail(KDE_EINVAL, "Y and out must be device pointers of the index's GPU");
    }
  }
  double* acc = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_acc_ptr[ix->device] == nullptr) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_exact_acc);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(KDE_ECUDA, "cudaGetSymbolAddress of the accumulator array failed");
      }
      g_acc_ptr[ix->device] = static_cast<double*>(p);
    }
    acc = g_acc_ptr[ix->device];
  }
  cudaStream_t st = (opts != nullptr && opts->stream != nullptr)
                        ? reinterpret_cast<cudaStream_t>(opts->stream)
                        : cudaStream_t(0);
  // the exact kernel never reads the query norms; the accumulator is cleared
  // inside the launcher before the kernel runs
  launch_exact_simt(Y, nullptr, nq, ix->X, ix->Xn, ix->n, ix->d, ix->dp, ix->kern, ix->h, acc,
                    out, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(KDE_ECUDA, cudaGetErrorString(e));
  return KDE_OK;
}

}  // extern "C"
