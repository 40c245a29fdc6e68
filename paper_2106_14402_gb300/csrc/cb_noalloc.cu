// Allocation-free variant of the row-pointer scan (K4).
//
// Some callers cannot allocate device memory when they need this step: a
// process whose device memory is entirely owned by another allocator (for
// example a framework's caching pool that reserved the GPU), or a
// latency-critical loop that must not pay for cudaMalloc's implicit device
// synchronisation.  This entry point needs no context (creating one
// allocates) and keeps its scratch, the per-tile partial sums, in the
// file-scope device array below.
#include <mutex>

#include "../../include/cb.h"
#include "cb_kernels.h"

namespace {

constexpr int64_t kScanTileItems = 4096;     // entries per scan tile (K4's layout)
constexpr int64_t kMaxTiles = 65536;
constexpr int64_t kMaxN = kMaxTiles * kScanTileItems;  // 268,435,456 entries

// One partial sum per tile plus one spare entry, as the scan launcher lays
// them out: 65,537 x 8 bytes = 512 KiB + 8 bytes.  Every GPU that loads the
// library holds this array until the process exits.
static __device__ __align__(256) int64_t g_scan_scratch[kMaxTiles + 1];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int64_t* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scan_scratch on the current device, looked up once per
// device (the host-side symbol is only a stand-in, not a device address).
int scratch_for_current_device(int64_t** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CB_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scan_scratch) != cudaSuccess || !p) return CB_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<int64_t*>(p);
  }
  *out = g_scratch_addr[dev];
  return CB_OK;
}

}  // namespace

extern "C" int cb_exclusive_scan_noalloc(const int64_t* in, int64_t n, int64_t* out,
                                         void* cuda_stream) {
  if (n < 0 || !out || (n > 0 && !in)) return CB_ERR_ARG;
  if (n > kMaxN) return CB_ERR_SCRATCH;
  int64_t* scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != CB_OK) return rc;
  // Every scratch entry the kernels read is written earlier in the same
  // call, so nothing has to be cleared between calls.
  cb::launch_exclusive_scan(in, n, out, scratch, static_cast<cudaStream_t>(cuda_stream));
  return cudaGetLastError() == cudaSuccess ? CB_OK : CB_ERR_CUDA;
}
