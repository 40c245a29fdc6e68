// Allocation-free variant of the row-pointer scan (K4).
//
// Some callers cannot allocate device memory when they need this step: a
// process whose device memory is entirely owned by another allocator (for
// example a framework's caching pool that reserved the GPU), or a
// latency-critical loop that must not pay for cudaMalloc's implicit device
// synchronisation.  This entry point needs no context (creating one
// allocates) and keeps its scratch, the per-tile partial sums, in the
// file-scope device array below.
#include <cuda.h>

#include <mutex>

#include "../../include/cb.h"
#include "cb_kernels.h"

namespace {

constexpr int64_t kMaxTiles = 65536;
constexpr int64_t kMaxN = kMaxTiles * cb::kScanTileItems;  // 268,435,456 entries

// One partial sum per tile plus one spare entry, as the scan launcher lays
// them out: 65,537 x 8 bytes = 512 KiB + 8 bytes.  Every GPU that loads the
// library holds this array until the process exits.
static __device__ __align__(256) int64_t g_scan_scratch[kMaxTiles + 1];

// The host-side name g_scan_scratch is only a stand-in, not a device address.
// The array's device address belongs to a CUDA context (a new context after
// cudaDeviceReset, or a driver-API context of the caller's own, has it
// elsewhere), so it is looked up once per context and cached under the
// context's unique id.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

struct Cached {
  unsigned long long ctx_id;
  int64_t* addr;
};
constexpr int kCacheSlots = 16;

std::mutex g_mu;
Cached g_cache[kCacheSlots] = {};
int g_next = 0;
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;

// Id of the context current on this thread (0 if none), through driver
// entry points fetched from the runtime (the library does not link libcuda).
bool current_ctx_id(unsigned long long* id) {
  if (!g_get_current || !g_get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return false;
    g_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext c = nullptr;
  if (g_get_current(&c) != CUDA_SUCCESS) return false;
  if (!c) {
    *id = 0;
    return true;
  }
  return g_get_id(c, id) == CUDA_SUCCESS;
}

// Device address of g_scan_scratch in the current context.  The first call
// in a context looks it up (cudaGetSymbolAddress, which also makes the
// device's primary context current when the thread has none).
int scratch_for_current_context(int64_t** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  if (!current_ctx_id(&id)) return CB_ERR_CUDA;
  if (id != 0) {
    for (const Cached& c : g_cache)
      if (c.ctx_id == id && c.addr) {
        *out = c.addr;
        return CB_OK;
      }
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scan_scratch) != cudaSuccess || !p) return CB_ERR_CUDA;
  if (id == 0 && (!current_ctx_id(&id) || id == 0)) return CB_ERR_CUDA;
  g_cache[g_next] = Cached{id, static_cast<int64_t*>(p)};
  g_next = (g_next + 1) % kCacheSlots;
  *out = static_cast<int64_t*>(p);
  return CB_OK;
}

}  // namespace

extern "C" int cb_exclusive_scan_noalloc(const int64_t* in, int64_t n, int64_t* out,
                                         void* cuda_stream) {
  if (n < 0 || !out || (n > 0 && !in)) return CB_ERR_ARG;
  if (n > kMaxN) return CB_ERR_SCRATCH;
  int64_t* scratch = nullptr;
  const int rc = scratch_for_current_context(&scratch);
  if (rc != CB_OK) return rc;
  // Every scratch entry the kernels read is written earlier in the same
  // call, so nothing has to be cleared between calls.  The launcher returns
  // the error of its own launches only.
  const cudaError_t e =
      cb::launch_exclusive_scan(in, n, out, scratch, static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? CB_OK : CB_ERR_CUDA;
}
