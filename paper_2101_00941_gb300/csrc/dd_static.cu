// dd_sps_static: the single pulse search over caller-provided device series, with its scratch
// (the per-trial moments) in a fixed device array instead of memory the library allocates.
//
// Some callers cannot let a library allocate device memory at run time: a real-time beam
// pipeline that reserves its whole GPU memory budget at start-up and must never pay the
// implicit device synchronisation of cudaMalloc/cudaFree in its processing loop, or a plug-in
// whose host framework owns every device allocation. This entry point serves them: it
// allocates nothing, and the caller passes the inputs and the outputs.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "dd_internal.h"

namespace {

constexpr int32_t kStaticMaxTrials = 16384;

// Scratch shared by every call on a device: one moments record per trial (512 KB). Every
// GPU that loads the library holds it until the process exits.
static __device__ __align__(256) ddk::Moments g_static_moments[kStaticMaxTrials];

// Device address of the scratch array, cached per CUDA context: a context that is destroyed
// and created again (cudaDeviceReset, or a primary context released by its last user) may load
// the module at another address, so the cache is keyed by the context handle, not the ordinal.
constexpr int kMaxContexts = 64;
struct ScratchEntry {
  CUcontext ctx;
  ddk::Moments* ptr;
};
ScratchEntry g_scratch[kMaxContexts] = {};
int g_nscratch = 0;
std::mutex g_scratch_mu;

// errors go to the library's per-thread message (dd_last_error)
int static_fail(int code, const char* msg) { return ddk::report_error(code, msg); }

PFN_cuCtxGetCurrent_v4000 ctx_get_current() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
  });
  return fn;
}

// Device address of the scratch array in the current context, looked up the first time a
// context is seen (in host code the array's name is only a host-side stand-in, not a device
// address). cudaSetDevice makes the device's primary context current if no context is yet.
int scratch_for_current_context(ddk::Moments** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || cudaSetDevice(dev) != cudaSuccess)
    return static_fail(DD_ERR_CUDA, "dd_sps_static: no usable current CUDA device");
  PFN_cuCtxGetCurrent_v4000 get = ctx_get_current();
  CUcontext ctx = nullptr;
  if (!get || get(&ctx) != CUDA_SUCCESS || !ctx)
    return static_fail(DD_ERR_CUDA, "dd_sps_static: no current CUDA context");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  for (int k = 0; k < g_nscratch; ++k)
    if (g_scratch[k].ctx == ctx) {
      *out = g_scratch[k].ptr;
      return DD_OK;
    }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_moments);
  if (e != cudaSuccess || !p)
    return static_fail(DD_ERR_CUDA, "dd_sps_static: cudaGetSymbolAddress of the scratch failed");
  // a full cache forgets its oldest entry (contexts come and go rarely)
  if (g_nscratch == kMaxContexts) {
    for (int k = 1; k < kMaxContexts; ++k) g_scratch[k - 1] = g_scratch[k];
    --g_nscratch;
  }
  g_scratch[g_nscratch++] = {ctx, static_cast<ddk::Moments*>(p)};
  *out = static_cast<ddk::Moments*>(p);
  return DD_OK;
}

}  // namespace

extern "C" {

int dd_sps_static(const int32_t* series, int32_t n_trials, int64_t n, int64_t stride,
                  int32_t range, int32_t decimation, int64_t j0, const int32_t* widths,
                  int32_t nwidths, float threshold, int32_t peak_block, dd_cand_t* cands,
                  int64_t cap, unsigned long long* count, void* cuda_stream) {
  if (!series || !cands || !count || !widths)
    return static_fail(DD_ERR_ARG, "dd_sps_static: NULL argument");
  if (n_trials < 1 || n_trials > kStaticMaxTrials)
    return static_fail(DD_ERR_ARG,
                       "dd_sps_static: n_trials must be 1..16384 (the size of the fixed scratch)");
  if (n < 1 || stride < n || cap < 0)
    return static_fail(DD_ERR_ARG, "dd_sps_static: need n >= 1, stride >= n, cap >= 0");
  if (decimation < 1 || (decimation & (decimation - 1)) || decimation > 256)
    return static_fail(DD_ERR_ARG, "dd_sps_static: decimation must be a power of two <= 256");
  if (peak_block < 1 || peak_block > 32 || (peak_block & (peak_block - 1)))
    return static_fail(DD_ERR_ARG, "dd_sps_static: peak_block must be a power of two <= 32");
  if (nwidths < 1 || nwidths > ddk::kMaxWidths)
    return static_fail(DD_ERR_ARG, "dd_sps_static: nwidths must be 1..16");
  if (!std::isfinite(threshold))
    return static_fail(DD_ERR_ARG, "dd_sps_static: threshold must be finite");
  ddk::SpsArgs a;
  memset(&a, 0, sizeof a);
  int maxw = 0;
  for (int k = 0; k < nwidths; ++k) {
    if (widths[k] < 1 || widths[k] > 1024 || (k > 0 && widths[k] <= widths[k - 1]))
      return static_fail(DD_ERR_ARG,
                         "dd_sps_static: widths must be strictly increasing within 1..1024");
    if (widths[k] >= decimation && widths[k] % decimation == 0) {
      a.wd[a.nw++] = widths[k] / decimation;
      maxw = widths[k] / decimation;
    }
  }
  ddk::Moments* scratch = nullptr;
  int rc = scratch_for_current_context(&scratch);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the caller's counter must start at zero; the moments are overwritten in full, so the
  // previous call's contents need no clearing
  if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess)
    return static_fail(DD_ERR_CUDA, "dd_sps_static: clearing the candidate counter failed");
  if (ddk::launch_moments(series, n_trials, n, stride, scratch, st) != cudaSuccess)
    return static_fail(DD_ERR_CUDA, "dd_sps_static: moments launch failed");
  if (a.nw == 0) return DD_OK;
  a.y = series;
  a.stride = stride;
  a.n = n;
  a.mom = scratch;
  a.n_trials = n_trials;
  a.range = range;
  a.d = decimation;
  a.block = peak_block;
  a.J0 = j0;
  a.hist = (int32_t)(((maxw - 1 > 0 ? maxw - 1 : 0) + 255) / 256 * 256);
  a.threshold = threshold;
  a.cands = cands;
  a.count = count;
  a.cap = cap;
  if (ddk::launch_sps(a, st) != cudaSuccess)
    return static_fail(DD_ERR_CUDA, "dd_sps_static: search launch failed");
  return DD_OK;
}

}  // extern "C"
