// C ABI of the semiring SpGEMM (include/cb.h): argument checks, workspace
// management and the host-side plan that orders the kernels of the path on
// one stream:
//   validate? -> K1 flops + tiers -> K2 scatter -> [sync: tier sizes]
//   -> K3 symbolic (hash tiers + heavy bitmap slices) -> K4 scan -> numeric
//   binning + heavy units -> [sync: nnz(C)] -> allocate C -> K5-K7 numeric.
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <deque>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/cb.h"
#include "cb_common.cuh"
#include "cb_kernels.h"

struct cb_ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 0;
  void* ws = nullptr;   // workspace for per-row arrays
  size_t ws_cap = 0;
  void* ws2 = nullptr;  // workspace for heavy-row slice arrays
  size_t ws2_cap = 0;
  int64_t* host = nullptr;  // pinned read-back buffer
  cudaEvent_t ev[6] = {};   // phase boundaries (CB_FLAG_TIMING)
  nvtxRangeId_t nvtx = 0;   // the open NVTX range of the current phase (0: none)
  cb::Tune tune;            // tier bounds (cb_ctx_set_tune / cb_autotune)
  unsigned long long* fstat = nullptr;  // tile status words of the one-launch path
  int64_t fstat_cap = 0;
  unsigned* fsync = nullptr;  // [0] launch epoch, [1] finished CTAs, [4] status word
  void* spa = nullptr;        // SpMSpV dense accumulator (spa_n values of spa_sr's type)
  unsigned* spa_bits = nullptr;  // its touched bitmap, all zero between calls
  int64_t spa_n = 0;
  int spa_sr = 0;
  std::string err;
  cb_stats stats{};
  // fault injection (cb_ctx_set_fault)
  int64_t fault_alloc = 0;    // the fault_alloc-th device allocation fails (0: off)
  int64_t allocs_seen = 0;    // device allocations since the fault was set
  unsigned fused_spin = cb::kFusedSpinDefault;  // polls per look-back wait
  int64_t fused_silent = -1;  // tile of the one-launch kernel that never publishes
  int64_t fault_short_row = -1;  // row whose exact size is made one short (-1: off)
};

namespace {

using cb::DevCSR;

struct Fail {
  int code;
};

#define CB_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
      throw Fail{e_ == cudaErrorMemoryAllocation ? CB_ERR_OOM : CB_ERR_CUDA};         \
    }                                                                                 \
  } while (0)

#define CB_LAUNCHED()                                                                 \
  do {                                                                                \
    cudaError_t e_ = cudaGetLastError();                                              \
    if (e_ != cudaSuccess) {                                                          \
      ctx->err = std::string("kernel launch: ") + cudaGetErrorString(e_);             \
      throw Fail{CB_ERR_CUDA};                                                        \
    }                                                                                 \
  } while (0)

// Every device allocation of the context goes through these, so that
// CB_FAULT_ALLOC can fail the k-th one as an out-of-memory would.
bool injected_alloc_failure(cb_ctx* ctx) {
  if (ctx->fault_alloc <= 0) return false;
  if (++ctx->allocs_seen < ctx->fault_alloc) return false;
  ctx->fault_alloc = 0;
  return true;
}

template <class T>
cudaError_t dev_alloc(cb_ctx* ctx, T** p, size_t bytes) {
  if (injected_alloc_failure(ctx)) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, ctx->stream);
}

template <class T>
cudaError_t dev_alloc_sync(cb_ctx* ctx, T** p, size_t bytes) {
  if (injected_alloc_failure(ctx)) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

void fail(cb_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  throw Fail{code};
}

// Internal semiring id of the merge form of CB_MAXW_LABEL (Sem<7>): the
// selector product of cb_merge; never accepted from callers.
constexpr int kMergeMaxwLabel = 7;

// Value sizes of A's, B's and C's arrays under a semiring (0: unknown).
size_t a_value_size(int sr) {
  switch (sr) {
    case CB_PLUS_TIMES_I64: return 8;
    case CB_PLUS_TIMES_F64: return 8;
    case CB_MIN_PLUS_U32: return 4;
    case CB_OR_AND_BOOL: return 1;
    case CB_SEL2ND_MIN_I32: return 4;
    case CB_MAXW_LABEL: return sizeof(float);
    case kMergeMaxwLabel: return 1;
  }
  return 0;
}
size_t b_value_size(int sr) {
  if (sr == CB_MAXW_LABEL) return sizeof(int32_t);
  if (sr == kMergeMaxwLabel) return sizeof(cb_wlabel);
  return a_value_size(sr);
}
size_t value_size(int sr) {
  return sr == CB_MAXW_LABEL || sr == kMergeMaxwLabel ? sizeof(cb_wlabel) : a_value_size(sr);
}
// A semiring a caller may name (the internal merge form is not one).
bool public_semiring(int sr) { return sr >= CB_PLUS_TIMES_I64 && sr <= CB_MAXW_LABEL; }

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Bump allocator over a workspace buffer.
struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    T* p = reinterpret_cast<T*>(base + off);
    off += align_up(n * sizeof(T));
    return p;
  }
};

void ensure(cb_ctx* ctx, void** buf, size_t* cap, size_t need) {
  if (need <= *cap) return;
  size_t want = need + need / 4 + (1 << 20);
  if (*buf) CB_CUDA(cudaFreeAsync(*buf, ctx->stream));
  *buf = nullptr;
  *cap = 0;
  CB_CUDA(dev_alloc(ctx, buf, want));
  *cap = want;
}

// Stream-ordered device buffer released when it goes out of scope.
struct DevBuf {
  cb_ctx* ctx;
  void* p = nullptr;
  explicit DevBuf(cb_ctx* c) : ctx(c) {}
  void alloc(size_t bytes) {
    CB_CUDA(dev_alloc(ctx, &p, bytes ? bytes : 1));
  }
  ~DevBuf() {
    if (p) cudaFreeAsync(p, ctx->stream);
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

void check_operand(cb_ctx* ctx, const cb_csr* M, const char* name) {
  if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0)
    fail(ctx, CB_ERR_ARG, std::string(name) + ": negative size");
  if (!M->row_ptr) fail(ctx, CB_ERR_ARG, std::string(name) + ": null row_ptr");
  if (M->nnz > 0 && (!M->col || !M->val))
    fail(ctx, CB_ERR_ARG, std::string(name) + ": null col/val with nnz > 0");
  if (M->ncols > INT32_MAX || M->nrows >= INT32_MAX)
    fail(ctx, CB_ERR_INDEX, std::string(name) + ": dimension beyond int32 indices");
}

DevCSR dev(const cb_csr* M) { return DevCSR{M->nrows, M->ncols, M->row_ptr, M->col, M->val}; }

void read_counters(cb_ctx* ctx, const int64_t* counters, const int64_t* extra, int n_extra) {
  CB_CUDA(cudaMemcpyAsync(ctx->host, counters, sizeof(int64_t) * cb::kCounters,
                          cudaMemcpyDeviceToHost, ctx->stream));
  if (n_extra)
    CB_CUDA(cudaMemcpyAsync(ctx->host + cb::kCounters, extra, sizeof(int64_t) * n_extra,
                            cudaMemcpyDeviceToHost, ctx->stream));
  CB_CUDA(cudaStreamSynchronize(ctx->stream));
}

void run_validation(cb_ctx* ctx, const cb_csr* A, const cb_csr* B) {
  ensure(ctx, &ctx->ws, &ctx->ws_cap, align_up(sizeof(int64_t) * cb::kCounters));
  int64_t* counters = static_cast<int64_t*>(ctx->ws);
  CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
  cb::launch_validate(dev(A), A->nnz, 0, counters, ctx->stream, ctx->sms);
  cb::launch_validate(dev(B), B->nnz, 10, counters, ctx->stream, ctx->sms);
  CB_LAUNCHED();
  ctx->stats.kernels += 2;
  read_counters(ctx, counters, nullptr, 0);
  const int64_t e = ctx->host[cb::kError];
  if (e) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "%s: %s invalid at index %lld", e >= 10 ? "B" : "A",
                  (e % 10) == 1 ? "row_ptr" : "column index",
                  (long long)ctx->host[cb::kErrDetail]);
    fail(ctx, CB_ERR_INDEX, msg);
  }
}

// Debug build: fail the call when a kernel recorded a failed bounds check
// (synchronises; nothing happens in the normal build).
void check_words(cb_ctx* ctx) {
  if constexpr (!cb::kChecked) return;
  struct {
    const char* file;
    int64_t (*take)(cudaStream_t, int64_t*);
  } const readers[] = {{"numeric", cb::check_take_numeric},   {"symbolic", cb::check_take_symbolic},
                       {"queue", cb::check_take_queue},       {"rows", cb::check_take_rows},
                       {"fused", cb::check_take_fused}};
  for (const auto& r : readers) {
    int64_t index = 0;
    const int64_t code = r.take(ctx->stream, &index);
    if (code == 0) continue;
    char msg[160];
    if (code < 0) std::snprintf(msg, sizeof msg, "bounds check word of %s unreadable", r.file);
    else std::snprintf(msg, sizeof msg, "bounds check %lld failed at index %lld (%s kernels)",
                       (long long)code, (long long)index, r.file);
    fail(ctx, CB_ERR_CUDA, msg);
  }
}

// Phase boundary k of a product: 0 before the flop count (K1), 1 before the
// symbolic phase, 2 before the scan, 3 after it (C allocated next), 4 before
// the numeric phase, 5 after it.  Each phase is an NVTX range on the host
// thread ("cb.stats" ... "cb.numeric", free without a profiler attached);
// with CB_FLAG_TIMING an event is also recorded on ctx's stream.
void mark(cb_ctx* ctx, const cb_opts& opt, int k) {
  static const char* const kPhase[5] = {"cb.stats", "cb.symbolic", "cb.scan", "cb.alloc",
                                        "cb.numeric"};
  if (ctx->nvtx) nvtxRangeEnd(ctx->nvtx);
  ctx->nvtx = k < 5 ? nvtxRangeStartA(kPhase[k]) : 0;
  if (!(opt.flags & CB_FLAG_TIMING)) return;
  if (!ctx->ev[k]) CB_CUDA(cudaEventCreate(&ctx->ev[k]));
  CB_CUDA(cudaEventRecord(ctx->ev[k], ctx->stream));
}

void collect_times(cb_ctx* ctx, const cb_opts& opt, bool numeric_ran) {
  if (ctx->nvtx) {  // the product is done: close its last phase's range
    nvtxRangeEnd(ctx->nvtx);
    ctx->nvtx = 0;
  }
  if (!(opt.flags & CB_FLAG_TIMING)) return;
  CB_CUDA(cudaEventSynchronize(ctx->ev[numeric_ran ? 5 : 3]));
  float t = 0.f;
  CB_CUDA(cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[1]));
  ctx->stats.ms_stats = t;
  CB_CUDA(cudaEventElapsedTime(&t, ctx->ev[1], ctx->ev[2]));
  ctx->stats.ms_symbolic = t;
  CB_CUDA(cudaEventElapsedTime(&t, ctx->ev[2], ctx->ev[3]));
  ctx->stats.ms_scan = t;
  if (numeric_ran) {
    CB_CUDA(cudaEventElapsedTime(&t, ctx->ev[4], ctx->ev[5]));
    ctx->stats.ms_numeric = t;
  }
}

// Scratch of the one-launch path: tile status words (zeroed once; launch
// epochs keep them valid across calls) and the epoch / finished-CTA words.
void ensure_fused(cb_ctx* ctx, int64_t tiles) {
  if (!ctx->fsync) {
    CB_CUDA(dev_alloc_sync(ctx, &ctx->fsync, 64));
    CB_CUDA(cudaMemsetAsync(ctx->fsync, 0, 64, ctx->stream));
  }
  if (tiles <= ctx->fstat_cap) return;
  const int64_t want = std::max<int64_t>(tiles + tiles / 4, 4096);
  if (ctx->fstat) {
    CB_CUDA(cudaStreamSynchronize(ctx->stream));
    CB_CUDA(cudaFree(ctx->fstat));
    ctx->fstat = nullptr;
    ctx->fstat_cap = 0;
  }
  CB_CUDA(dev_alloc_sync(ctx, &ctx->fstat, sizeof(unsigned long long) * (size_t)want));
  CB_CUDA(cudaMemsetAsync(ctx->fstat, 0, sizeof(unsigned long long) * (size_t)want, ctx->stream));
  ctx->fstat_cap = want;
}

// Smallest lane count whose bounds hold for every row, 0 if none.
int fused_fit(int64_t max_arow, int64_t max_flops, int64_t ncols) {
  for (int lanes : {8, 16, 32})
    if (max_arow <= lanes && max_flops <= 8 * lanes && ncols <= cb::fused_max_cols(lanes))
      return lanes;
  return 0;
}

void run_fused(cb_ctx* ctx, int sr, int lanes, const DevCSR& dA, const DevCSR& dB, int64_t* rp,
               int32_t* col, void* val, int64_t cap, int* status) {
  if (dA.nrows == 0) {
    CB_CUDA(cudaMemsetAsync(rp, 0, sizeof(int64_t), ctx->stream));
    return;
  }
  ensure_fused(ctx, cb::fused_tiles(lanes, dA.nrows));
  const cudaError_t e = cb::launch_fused(sr, lanes, dA, dB, rp, col, val, cap, ctx->fstat,
                                         ctx->fstat_cap, ctx->fsync, status, ctx->stream, ctx->sms,
                                         ctx->fused_spin, ctx->fused_silent);
  if (e != cudaSuccess) {
    ctx->err = std::string("fused launch: ") + cudaGetErrorString(e);
    throw Fail{CB_ERR_CUDA};
  }
  CB_LAUNCHED();
  ctx->stats.kernels += 1;
}

// One launch of the one-launch kernel into C (capacity cap) with the
// context's status word, then one read-back of nnz(C), the status bits and
// the product count (synchronises).  Returns the status bits.
int fused_pass(cb_ctx* ctx, int sr, int lanes, const DevCSR& dA, const DevCSR& dB, cb_csr* C,
               int64_t cap, const cb_opts& opt) {
  ensure_fused(ctx, 0);
  int* st = reinterpret_cast<int*>(ctx->fsync + 4);
  CB_CUDA(cudaMemsetAsync(st, 0, sizeof(int), ctx->stream));
  mark(ctx, opt, 4);
  run_fused(ctx, sr, lanes, dA, dB, C->row_ptr, C->col, C->val, cap, st);
  mark(ctx, opt, 5);
  // words 2..7 of the sync area: nnz(C), status, product count
  CB_CUDA(cudaMemcpyAsync(ctx->host, ctx->fsync + 2, 6 * sizeof(unsigned), cudaMemcpyDeviceToHost,
                          ctx->stream));
  CB_CUDA(cudaStreamSynchronize(ctx->stream));
  return (int)(ctx->host[1] & 0xFFFFFFFF);
}

// One launch of the work-queue kernel over the m rows of A.B into C
// (capacity cap), then one read-back of nnz(C) and the status bits
// (synchronises).  Returns the status bits.
int queue_pass(cb_ctx* ctx, int sr, const DevCSR& dA, const DevCSR& dB, int64_t m, cb_csr* C,
               int64_t cap, const cb_opts& opt) {
  ensure_fused(ctx, m);
  int* st = reinterpret_cast<int*>(ctx->fsync + 4);
  CB_CUDA(cudaMemsetAsync(st, 0, sizeof(int), ctx->stream));
  mark(ctx, opt, 4);
  const cudaError_t e = cb::launch_queue_rows(sr, dA, dB, m, C->row_ptr, C->col, C->val, cap,
                                              ctx->fstat, ctx->fstat_cap, ctx->fsync, st, ctx->stream,
                                              ctx->sms, ctx->fused_spin, ctx->fused_silent);
  if (e != cudaSuccess) {
    ctx->err = std::string("queued SpGEMM launch: ") + cudaGetErrorString(e);
    throw Fail{CB_ERR_CUDA};
  }
  ctx->stats.kernels += 1;
  mark(ctx, opt, 5);
  CB_CUDA(cudaMemcpyAsync(ctx->host, ctx->fsync + 2, 6 * sizeof(unsigned), cudaMemcpyDeviceToHost,
                          ctx->stream));
  CB_CUDA(cudaStreamSynchronize(ctx->stream));
  return (int)(ctx->host[1] & 0xFFFFFFFF);
}

// Results of a fused pass that had no row beyond its bounds.
void finish_fused(cb_ctx* ctx, cb_csr* C, int bits, int64_t cap, const cb_opts& opt) {
  const int64_t total = ctx->host[0];
  C->nnz = total;
  ctx->stats.nnz = total;
  ctx->stats.flops = ctx->host[2];
  if (bits & CB_FUSED_STALLED) fail(ctx, CB_ERR_TIMEOUT, "fused SpGEMM: a tile wait expired");
  if (bits & CB_FUSED_CAPACITY) {
    char msg[128];
    std::snprintf(msg, sizeof msg, "output needs %lld entries, capacity %lld", (long long)total,
                  (long long)cap);
    ctx->err = msg;
    throw Fail{CB_ERR_CAPACITY};
  }
  collect_times(ctx, opt, true);
}

// Largest C the speculative path allocates itself (entries): 8 * lanes per
// row is its bound of nnz(C) before any row has been counted.
constexpr int64_t kSpeculativeMaxEntries = int64_t(1) << 24;

// The speculative one-launch pass (see spgemm_plain).  Lanes come from the
// mean row lengths of A and B (every row must fit them; the kernel checks).
// Returns true when the product is complete, false to take the classified
// path (nothing of C kept).
bool try_fused_speculatively(cb_ctx* ctx, int sr, const cb_csr* A, const DevCSR& dB, int64_t b_nnz,
                             cb_csr* C, const cb_opts& opt, bool caller_buf, size_t vsz) {
  const int64_t m = A->nrows;
  if (m == 0 || dB.nrows == 0) return false;
  const double mean_a = (double)A->nnz / (double)m, mean_b = (double)b_nnz / (double)dB.nrows;
  int lanes = 0;
  for (int g : {8, 16, 32})
    if (mean_a <= g && mean_a * mean_b <= 8.0 * g && dB.ncols <= cb::fused_max_cols(g)) {
      lanes = g;
      break;
    }
  if (!lanes) return false;
  const int64_t bound = 8 * (int64_t)lanes * m;  // nnz(C) when every row fits
  const int64_t cap = caller_buf ? opt.out_capacity : bound;
  if (!caller_buf && bound > kSpeculativeMaxEntries) return false;
  if (!caller_buf) {
    CB_CUDA(dev_alloc(ctx, &C->col, sizeof(int32_t) * (size_t)cap));
    CB_CUDA(dev_alloc(ctx, &C->val, vsz * (size_t)cap));
  }
  mark(ctx, opt, 0);
  mark(ctx, opt, 1);
  mark(ctx, opt, 2);
  mark(ctx, opt, 3);
  const int bits = fused_pass(ctx, sr, lanes, dev(A), dB, C, cap, opt);
  if (bits & CB_FUSED_ROW_TOO_LARGE) {  // a row beyond the lanes' bounds: classify first
    if (!caller_buf) {
      CB_CUDA(cudaFreeAsync(C->col, ctx->stream));
      CB_CUDA(cudaFreeAsync(C->val, ctx->stream));
      C->col = nullptr;
      C->val = nullptr;
    }
    return false;
  }
  finish_fused(ctx, C, bits, cap, opt);
  return true;
}

// Everything from K1 to the allocation of C and the numeric phase.
// The plain (unbatched) path on a possibly windowed view dB of B; C gets
// C->ncols = out_ncols.  Inputs are assumed valid (validation happens first).
// skip (optional): rows already computed elsewhere; their sizes are preset[i]
// and the exact phases leave them out.
// a_rcols (optional): per-row output width of A's rows (stacked batches).
// b_nnz (optional, >= 0): B's stored entries, for the speculative one-launch path.
void spgemm_plain(cb_ctx* ctx, int sr, const cb_csr* A, const DevCSR& dB, int64_t out_ncols,
                  cb_csr* C, const cb_opts& opt, const uint8_t* skip = nullptr,
                  const int64_t* preset = nullptr, const int32_t* a_rcols = nullptr,
                  int64_t b_nnz = -1) {
  const int64_t m = A->nrows, ncols = dB.ncols;
  const bool caller_buf = opt.out_capacity > 0;
  const size_t vsz = value_size(sr);

  // stage-1 workspace: counters, per-row arrays, scan partials
  size_t need = align_up(sizeof(int64_t) * cb::kCounters) + 3 * align_up(8 * (size_t)m + 8) +
                2 * align_up(4 * (size_t)m + 4) + align_up(8 * (size_t)cb::scan_partials(m));
  ensure(ctx, &ctx->ws, &ctx->ws_cap, need);
  Carver cv{static_cast<char*>(ctx->ws)};
  int64_t* counters = cv.take<int64_t>(cb::kCounters);
  int64_t* flops = cv.take<int64_t>(m + 1);
  int64_t* nnz = cv.take<int64_t>(m + 1);
  int32_t* maxb = cv.take<int32_t>(m + 1);
  int32_t* perm_sym = cv.take<int32_t>(m + 1);
  int32_t* perm_num = cv.take<int32_t>(m + 1);
  int64_t* partial = cv.take<int64_t>(cb::scan_partials(m));

  C->nrows = m;
  C->ncols = out_ncols;
  C->nnz = 0;
  if (!caller_buf) {
    C->row_ptr = nullptr;
    C->col = nullptr;
    C->val = nullptr;
    CB_CUDA(dev_alloc(ctx, &C->row_ptr, sizeof(int64_t) * (size_t)(m + 1)));
  }
  if (m == 0) {
    CB_CUDA(cudaMemsetAsync(C->row_ptr, 0, sizeof(int64_t), ctx->stream));
    return;
  }

  DevCSR dA = dev(A);
  dA.rcols = a_rcols;
  const bool fused_ok = !(opt.flags & CB_FLAG_NO_FUSED) && !skip && !preset && !a_rcols && !dB.rpe &&
                        !dB.filter && dB.col_lo == 0;
  // Speculative one-launch path: when the operands' mean row lengths say that
  // every row is probably small, launch the one-launch kernel right away.  It
  // checks every row's bounds itself; only if a row exceeds them is the
  // product recomputed by the path below, which classifies the rows first.
  if (fused_ok && b_nnz >= 0 && try_fused_speculatively(ctx, sr, A, dB, b_nnz, C, opt, caller_buf, vsz))
    return;
  CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
  mark(ctx, opt, 0);
  cb::launch_check_sorted(dB, counters, ctx->stream, ctx->sms);
  cb::launch_classify_sym(dA, dB, flops, maxb, counters, ctx->stream, ctx->sms, skip,
                          ctx->tune.sym_hash_max);
  cb::launch_scatter_sym(m, ncols, flops, perm_sym, nnz, counters, ctx->stream, ctx->sms, skip,
                         preset, ctx->tune.sym_hash_max, a_rcols);
  CB_LAUNCHED();
  mark(ctx, opt, 1);
  ctx->stats.kernels += 3;
  read_counters(ctx, counters, nullptr, 0);
  const int b_sorted = ctx->host[cb::kUnsorted] == 0 ? 1 : 0;

  int64_t sym_cnt[cb::kSymTiers], sym_beg[cb::kSymTiers];
  for (int t = 0; t < cb::kSymTiers; ++t) sym_cnt[t] = ctx->host[cb::kCntSym + t];
  sym_beg[0] = 0;
  sym_beg[1] = 0;
  for (int t = 2; t < cb::kSymTiers; ++t) sym_beg[t] = sym_beg[t - 1] + sym_cnt[t - 1];
  ctx->stats.flops = ctx->host[cb::kTotalFlops];

  // Every row small: one launch forms, sorts and places all rows (k_fused),
  // into C sized by flops (an upper bound of nnz(C)).
  const int lanes = fused_fit(ctx->host[cb::kMaxArow], ctx->host[cb::kMaxFlops], ncols);
  if (lanes && fused_ok) {
    const int64_t cap = caller_buf ? opt.out_capacity : ctx->stats.flops;
    if (!caller_buf && cap > 0) {
      CB_CUDA(dev_alloc(ctx, &C->col, sizeof(int32_t) * (size_t)cap));
      CB_CUDA(dev_alloc(ctx, &C->val, vsz * (size_t)cap));
    }
    mark(ctx, opt, 2);
    mark(ctx, opt, 3);
    const int bits = fused_pass(ctx, sr, lanes, dA, dB, C, cap, opt);
    if (bits & CB_FUSED_ROW_TOO_LARGE) fail(ctx, CB_ERR_CUDA, "fused SpGEMM: row bound violated");
    finish_fused(ctx, C, bits, cap, opt);
    return;
  }
  // Every row of bounded size and width: one persistent launch takes the rows
  // from a work queue and forms each in one pass (k_queue_rows), into C sized
  // by flops.
  if (!(opt.flags & CB_FLAG_NO_FUSED) && !skip && !preset && ncols <= cb::kQueueWidth &&
      ctx->host[cb::kMaxFlops] <= cb::kQueueAcc) {
    const int64_t flops = ctx->stats.flops;
    const int64_t cap = caller_buf ? opt.out_capacity : flops;
    if (!caller_buf && cap > 0) {
      CB_CUDA(dev_alloc(ctx, &C->col, sizeof(int32_t) * (size_t)cap));
      CB_CUDA(dev_alloc(ctx, &C->val, vsz * (size_t)cap));
    }
    mark(ctx, opt, 2);
    mark(ctx, opt, 3);
    const int bits = queue_pass(ctx, sr, dA, dB, m, C, cap, opt);
    if (bits & CB_FUSED_ROW_TOO_LARGE) fail(ctx, CB_ERR_CUDA, "queued SpGEMM: row bound violated");
    finish_fused(ctx, C, bits, cap, opt);
    ctx->stats.flops = flops;
    return;
  }

  const int64_t n_heavy = sym_cnt[cb::kSymHeavy];
  const int64_t spans = (ncols + cb::kSpanCols - 1) / cb::kSpanCols;
  const int wcut = cb::num_window_cut(sr);
  // every (row, span) yields at most count/wcut + 1 windows; counts sum to <= flops
  const int64_t win_cap = n_heavy * spans + ctx->stats.flops / wcut + 1;

  // Heavy-row bitmaps are kept for the numeric phase when they fit a quarter
  // of free device memory (capped at 32 GiB); otherwise the numeric phase
  // rebuilds each window's bitmap from the products.
  const size_t bits_bytes = (size_t)(n_heavy * spans) * cb::kSpanWords * sizeof(unsigned);
  size_t free_b = 0, total_b = 0;
  CB_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const bool keep_bits = n_heavy > 0 && bits_bytes <= free_b / 4 && bits_bytes <= (32ull << 30);
  const size_t racc_bytes = n_heavy > 0 ? cb::rank_scratch_bytes(sr, ctx->sms) : 0;
  size_t need2 = align_up(4 * (size_t)(n_heavy * spans) + 4) +
                 align_up(8 * (size_t)(n_heavy * spans) + 8) +
                 align_up(sizeof(cb::Window) * (size_t)win_cap) + (keep_bits ? align_up(bits_bytes) : 0) +
                 align_up(racc_bytes);
  ensure(ctx, &ctx->ws2, &ctx->ws2_cap, need2);
  Carver cv2{static_cast<char*>(ctx->ws2)};
  int32_t* span_counts = cv2.take<int32_t>(n_heavy * spans + 1);
  int2* span_wins = cv2.take<int2>(n_heavy * spans + 1);
  cb::Window* wins = cv2.take<cb::Window>(win_cap);
  unsigned* hbits = keep_bits ? cv2.take<unsigned>((size_t)(n_heavy * spans) * cb::kSpanWords) : nullptr;
  void* racc = racc_bytes ? cv2.take<char>(racc_bytes) : nullptr;
  const int32_t* heavy_rows = perm_sym + sym_beg[cb::kSymHeavy];

  int launches = 0;
  cb::launch_symbolic(dA, dB, perm_sym, sym_beg, sym_cnt, flops, nnz, span_counts, span_wins, wcut,
                      wins, win_cap, hbits, b_sorted, counters, ctx->stream, ctx->sms, &launches);
  mark(ctx, opt, 2);
  if (ctx->fault_short_row >= 0 && ctx->fault_short_row < m && !skip) {
    cb::launch_fault_shrink(nnz + ctx->fault_short_row, ctx->stream);
    ctx->stats.kernels += 1;
  }
  cb::launch_exclusive_scan(nnz, m, C->row_ptr, partial, ctx->stream);
  // the hash tier's table bounds the row size it can take for this value type
  const int64_t num_hash_max = std::min<int64_t>(ctx->tune.num_hash_max, cb::num_large_max(sr));
  cb::launch_classify_num(sr, m, nnz, perm_num, counters, ctx->stream, ctx->sms, skip,
                          num_hash_max);
  CB_LAUNCHED();
  mark(ctx, opt, 3);
  ctx->stats.kernels += launches + 3 + 2;
  read_counters(ctx, counters, C->row_ptr + m, 1);

  const int64_t total = ctx->host[cb::kCounters];
  int64_t num_cnt[cb::kNumTiers], num_beg[cb::kNumTiers];
  for (int t = 0; t < cb::kNumTiers; ++t) num_cnt[t] = ctx->host[cb::kCntNum + t];
  num_beg[0] = 0;
  num_beg[1] = 0;
  for (int t = 2; t < cb::kNumTiers; ++t) num_beg[t] = num_beg[t - 1] + num_cnt[t - 1];
  const int64_t n_units = ctx->host[cb::kUnits];
  if (ctx->host[cb::kError]) {
    char msg[96];
    std::snprintf(msg, sizeof msg, "symbolic phase consistency check failed (code %lld)",
                  (long long)ctx->host[cb::kError]);
    fail(ctx, CB_ERR_CUDA, msg);
  }
  ctx->stats.nnz = total;
  ctx->stats.heavy_rows = num_cnt[cb::kNumHeavy];
  ctx->stats.heavy_units = n_units;
  C->nnz = total;

  if (caller_buf) {
    if (total > opt.out_capacity) {
      char msg[128];
      std::snprintf(msg, sizeof msg, "output needs %lld entries, capacity %lld",
                    (long long)total, (long long)opt.out_capacity);
      ctx->err = msg;
      throw Fail{CB_ERR_CAPACITY};
    }
  } else if (total > 0) {
    CB_CUDA(dev_alloc(ctx, &C->col, sizeof(int32_t) * (size_t)total));
    CB_CUDA(dev_alloc(ctx, &C->val, vsz * (size_t)total));
  }
  if (total == 0) {
    collect_times(ctx, opt, false);
    return;
  }

  launches = 0;
  mark(ctx, opt, 4);
  cb::launch_numeric(sr, dA, dB, perm_num, num_beg, num_cnt, flops, nnz, heavy_rows, wins,
                     n_units, span_counts, spans, hbits, b_sorted, C->row_ptr, C->col, C->val,
                     counters + cb::kError, ctx->stream, ctx->sms, &launches, num_hash_max, racc,
                     cb::CfBounds{ctx->tune.cf_esc, ctx->tune.cf_pre});
  CB_LAUNCHED();
  mark(ctx, opt, 5);
  ctx->stats.kernels += launches;
  collect_times(ctx, opt, true);

  if (opt.flags & 1) {  // debug: check the kernels' internal consistency word
    read_counters(ctx, counters, nullptr, 0);
    if (ctx->host[cb::kError]) {
      char msg[96];
      std::snprintf(msg, sizeof msg, "internal consistency check failed (code %lld)",
                    (long long)ctx->host[cb::kError]);
      fail(ctx, CB_ERR_CUDA, msg);
    }
  }
}

int64_t total_of(cb_ctx* ctx, const int64_t* in, int64_t n);

// Learned (or upper-bound) sizing (paper Sec. 5: approximate memory
// estimation in place of the symbolic phase).  Each row's capacity comes
// from the MLP's predicted size (upper bound: min(flops, ncols)) times
// (1 + margin); rows whose capacity fits a shared-memory hash table are
// computed in one pass, without a symbolic phase, into a staging area sized
// by the capacities.  A row that overflows its capacity is detected on the
// device and, with the rows too large for the table, goes through the exact
// two-phase path; the one-pass rows are then copied from staging into C.
void spgemm_learned(cb_ctx* ctx, int sr, const cb_csr* A, const DevCSR& dB, int64_t out_ncols,
                    cb_csr* C, const cb_opts& opt, const int32_t* a_rcols = nullptr) {
  const int64_t m = A->nrows, ncols = dB.ncols;
  const int vsz = (int)value_size(sr);
  if (m == 0) {
    spgemm_plain(ctx, sr, A, dB, out_ncols, C, opt);
    return;
  }
  DevCSR dA = dev(A);
  dA.rcols = a_rcols;
  DevBuf work(ctx);
  const size_t nm = (size_t)m + 1;
  const size_t bytes = align_up(8 * nm) * 5 + align_up(4 * nm) * 2 + align_up(16 * nm) + align_up(nm) +
                       align_up(8 * (size_t)cb::kCounters) + align_up(8 * (size_t)cb::scan_partials(m));
  work.alloc(bytes);
  Carver cv{work.as<char>()};
  int64_t* flops = cv.take<int64_t>(nm);
  int64_t* pred = cv.take<int64_t>(nm);
  int64_t* cap = cv.take<int64_t>(nm);
  int64_t* stage_rp = cv.take<int64_t>(nm);
  int64_t* cnt = cv.take<int64_t>(nm);
  int32_t* maxb = cv.take<int32_t>(nm);
  int32_t* perm = cv.take<int32_t>(nm);
  float* feat = cv.take<float>(CB_MLP_NFEAT * nm);
  uint8_t* learned = cv.take<uint8_t>(nm);
  int64_t* counters = cv.take<int64_t>(cb::kCounters);
  int64_t* partial = cv.take<int64_t>(cb::scan_partials(m));

  CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
  cb::launch_classify_sym(dA, dB, flops, maxb, counters, ctx->stream, ctx->sms);
  const bool use_mlp = opt.sizing == CB_SIZING_LEARNED;
  if (use_mlp) {
    cb::launch_row_features(dA, flops, maxb, ncols, feat, ctx->stream, ctx->sms);
    cb::launch_mlp_predict(cb::mlp_bf16(opt.mlp), cb::mlp_master(opt.mlp), cb::mlp_norm(opt.mlp),
                           feat, m, ncols, nullptr, pred, ctx->stream, ctx->sms);
  }
  const int64_t hmax = std::min<int64_t>(ctx->tune.learn_max, cb::learn_hash_max(sr));
  cb::launch_learn_caps(m, use_mlp ? pred : nullptr, flops, ncols, use_mlp ? opt.margin : 0.0f, hmax,
                        cap, learned, ctx->stream, ctx->sms, a_rcols);
  cb::launch_exclusive_scan(cap, m, stage_rp, partial, ctx->stream);
  cb::launch_learned_tiers(m, cap, hmax, perm, counters, ctx->stream, ctx->sms);
  CB_LAUNCHED();
  int pre_launches = use_mlp ? 9 : 7;
  read_counters(ctx, counters, stage_rp + m, 1);
  const int64_t staged = ctx->host[cb::kCounters];
  int64_t seg_cnt[cb::kNumTiers], seg_beg[cb::kNumTiers];
  for (int t = 0; t < cb::kNumTiers; ++t) seg_cnt[t] = ctx->host[cb::kCntNum + t];
  seg_beg[0] = seg_beg[1] = 0;
  for (int t = 2; t < cb::kNumTiers; ++t) seg_beg[t] = seg_beg[t - 1] + seg_cnt[t - 1];

  DevBuf scol(ctx), sval(ctx);
  scol.alloc(sizeof(int32_t) * (size_t)staged);
  sval.alloc((size_t)vsz * (size_t)staged);
  int launches = 0;
  cb::launch_learned_numeric(sr, dA, dB, perm, seg_beg, seg_cnt, flops, cap, stage_rp,
                             scol.as<int32_t>(), sval.p, learned, cnt, counters + cb::kError,
                             ctx->stream, ctx->sms, &launches);
  CB_LAUNCHED();
  // the overflow count is read back with the exact pipeline's first sync
  CB_CUDA(cudaMemcpyAsync(ctx->host + cb::kCounters + 2, counters + cb::kError, sizeof(int64_t),
                          cudaMemcpyDeviceToHost, ctx->stream));
  pre_launches += launches;
  // rows that stayed on the one-pass path carry their size into the exact
  // pipeline; the rest (including overflowed rows) are computed exactly
  spgemm_plain(ctx, sr, A, dB, out_ncols, C, opt, learned, cnt, a_rcols);
  if (C->nnz > 0) {
    cb::launch_compact_rows(vsz, m, learned, stage_rp, cnt, scol.as<int32_t>(), sval.p, C->row_ptr,
                            C->col, C->val, ctx->stream, ctx->sms);
    CB_LAUNCHED();
    ctx->stats.kernels += 1;
  }
  ctx->stats.kernels += pre_launches;
  ctx->stats.overflow_rows = ctx->host[cb::kCounters + 2];
}

// Symbolic counts only: nnz_out[i] = nnz of row i of A.B (view dB).
void count_rows(cb_ctx* ctx, const DevCSR& dA, const DevCSR& dB, int64_t* nnz_out) {
  const int64_t m = dA.nrows, ncols = dB.ncols;
  if (m == 0) return;
  size_t need = align_up(sizeof(int64_t) * cb::kCounters) + align_up(8 * (size_t)m + 8) +
                align_up(4 * (size_t)m + 4);
  ensure(ctx, &ctx->ws, &ctx->ws_cap, need);
  Carver cv{static_cast<char*>(ctx->ws)};
  int64_t* counters = cv.take<int64_t>(cb::kCounters);
  int64_t* flops = cv.take<int64_t>(m + 1);
  int32_t* perm = cv.take<int32_t>(m + 1);
  CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
  cb::launch_check_sorted(dB, counters, ctx->stream, ctx->sms);
  cb::launch_classify_sym(dA, dB, flops, nullptr, counters, ctx->stream, ctx->sms, nullptr,
                          ctx->tune.sym_hash_max);
  cb::launch_scatter_sym(m, ncols, flops, perm, nnz_out, counters, ctx->stream, ctx->sms, nullptr,
                         nullptr, ctx->tune.sym_hash_max, dA.rcols);
  CB_LAUNCHED();
  ctx->stats.kernels += 3;
  read_counters(ctx, counters, nullptr, 0);
  int64_t cnt[cb::kSymTiers], beg[cb::kSymTiers];
  for (int t = 0; t < cb::kSymTiers; ++t) cnt[t] = ctx->host[cb::kCntSym + t];
  beg[0] = beg[1] = 0;
  for (int t = 2; t < cb::kSymTiers; ++t) beg[t] = beg[t - 1] + cnt[t - 1];
  ctx->stats.flops += ctx->host[cb::kTotalFlops];
  const int64_t n_heavy = cnt[cb::kSymHeavy];
  const int64_t spans = (ncols + cb::kSpanCols - 1) / cb::kSpanCols;
  ensure(ctx, &ctx->ws2, &ctx->ws2_cap, align_up(4 * (size_t)(n_heavy * spans) + 4));
  int launches = 0;
  cb::launch_symbolic(dA, dB, perm, beg, cnt, flops, nnz_out, static_cast<int32_t*>(ctx->ws2),
                      nullptr, cb::num_window_cut(CB_PLUS_TIMES_F64), nullptr, 0, nullptr,
                      ctx->host[cb::kUnsorted] == 0 ? 1 : 0, counters, ctx->stream, ctx->sms,
                      &launches);
  CB_LAUNCHED();
  ctx->stats.kernels += launches;
}

// Sum of n int64 values on the device (synchronises); uses ctx->ws.
int64_t total_of(cb_ctx* ctx, const int64_t* in, int64_t n) {
  DevBuf out(ctx);
  out.alloc(sizeof(int64_t) * (size_t)(n + 1));
  ensure(ctx, &ctx->ws2, &ctx->ws2_cap, align_up(8 * (size_t)cb::scan_partials(n)));
  cb::launch_exclusive_scan(in, n, out.as<int64_t>(), static_cast<int64_t*>(ctx->ws2), ctx->stream);
  CB_LAUNCHED();
  CB_CUDA(cudaMemcpyAsync(ctx->host + cb::kCounters + 1, out.as<int64_t>() + n, sizeof(int64_t),
                          cudaMemcpyDeviceToHost, ctx->stream));
  CB_CUDA(cudaStreamSynchronize(ctx->stream));
  return ctx->host[cb::kCounters + 1];
}

// Column-batched SpGEMM (paper Sec. 7.2; batch count from a symbolic step,
// Sec. 7.4): C is formed in contiguous column ranges whose output
// (row_ptr + col + val) fits opt.budget_bytes, each handed to on_batch.
// With exact sizing the batch count comes from the exact symbolic total and
// ranges are equal in width; with learned sizing the predicted total sets
// the first range and the density seen so far the later ones.  A range whose
// output still exceeds the budget is halved.  When
// B's rows are sorted each batch reads only its slab of every B row (slab
// offsets found by search); otherwise batches filter whole rows.
void spgemm_colbatch(cb_ctx* ctx, int sr, const cb_csr* A, const cb_csr* B, cb_csr* C,
                     const cb_opts& opt) {
  const int64_t m = A->nrows, n = B->nrows, k = B->ncols;
  const int64_t per = 4 + (int64_t)value_size(sr);
  const int64_t rp_bytes = 8 * (m + 1);
  if (opt.budget_bytes < rp_bytes + per)
    fail(ctx, CB_ERR_BUDGET, "budget smaller than one row-pointer array plus one entry");
  const int64_t cap = (opt.budget_bytes - rp_bytes) / per;
  if (opt.resume_col < 0 || opt.resume_col > k)
    fail(ctx, CB_ERR_ARG, "resume_col outside [0, B.ncols]");
  if (opt.resume_batch < 0) fail(ctx, CB_ERR_ARG, "resume_batch must be >= 0");
  if (opt.validate) run_validation(ctx, A, B);
  C->nrows = m;
  C->ncols = k;
  C->nnz = 0;
  C->row_ptr = nullptr;
  C->col = nullptr;
  C->val = nullptr;
  ctx->stats.batches = 0;
  if (m == 0 || k == 0 || A->nnz == 0 || B->nnz == 0 || opt.resume_col == k) return;

  const DevCSR dA = dev(A), dBfull = dev(B);
  DevBuf brp(ctx), bcol(ctx), bval(ctx), rownnz(ctx);
  brp.alloc(sizeof(int64_t) * (size_t)(m + 1));
  rownnz.alloc(sizeof(int64_t) * (size_t)(m + 1));

  // The batch count: from the exact symbolic total (paper Sec. 7.4), or,
  // with learned sizing, from the sum of the predicted row sizes times
  // (1 + margin), which skips that whole symbolic pass.
  int b_sorted;
  int64_t total;
  if (opt.sizing == CB_SIZING_LEARNED) {
    ensure(ctx, &ctx->ws, &ctx->ws_cap,
           align_up(sizeof(int64_t) * cb::kCounters) + align_up(8 * (size_t)(m + 1)) +
               align_up(4 * (size_t)(m + 1)) + align_up(16 * (size_t)(m + 1)));
    Carver cv{static_cast<char*>(ctx->ws)};
    int64_t* counters = cv.take<int64_t>(cb::kCounters);
    int64_t* flops = cv.take<int64_t>(m + 1);
    int32_t* maxb = cv.take<int32_t>(m + 1);
    float* feat = cv.take<float>(CB_MLP_NFEAT * (m + 1));
    CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
    cb::launch_check_sorted(dBfull, counters, ctx->stream, ctx->sms);
    cb::launch_classify_sym(dA, dBfull, flops, maxb, counters, ctx->stream, ctx->sms);
    cb::launch_row_features(dA, flops, maxb, k, feat, ctx->stream, ctx->sms);
    cb::launch_mlp_predict(cb::mlp_bf16(opt.mlp), cb::mlp_master(opt.mlp), cb::mlp_norm(opt.mlp),
                           feat, m, k, nullptr, rownnz.as<int64_t>(), ctx->stream, ctx->sms);
    CB_LAUNCHED();
    ctx->stats.kernels += 4;
    read_counters(ctx, counters, nullptr, 0);  // synchronises
    b_sorted = ctx->host[cb::kUnsorted] == 0 ? 1 : 0;
    ctx->stats.flops = ctx->host[cb::kTotalFlops];
    total = total_of(ctx, rownnz.as<int64_t>(), m);  // synchronises
    total = (int64_t)((double)total * (1.0 + (double)opt.margin));
  } else {
    count_rows(ctx, dA, dBfull, rownnz.as<int64_t>());
    b_sorted = ctx->host[cb::kUnsorted] == 0 ? 1 : 0;
    total = total_of(ctx, rownnz.as<int64_t>(), m);
  }
  const int64_t sym_flops = ctx->stats.flops;
  int64_t nb = (total + cap - 1) / cap;
  if (nb < 1) nb = 1;
  if (nb > k) nb = k;

  bcol.alloc(sizeof(int32_t) * (size_t)cap);
  bval.alloc((size_t)(per - 4) * (size_t)cap);

  // slab offsets of every boundary (sorted B only)
  struct Range {
    int64_t lo, hi;
    const int64_t* plo;
    const int64_t* phi;
  };
  std::vector<int64_t> bnd((size_t)nb + 1);
  for (int64_t j = 0; j <= nb; ++j) bnd[(size_t)j] = (int64_t)((__int128)j * k / nb);
  std::vector<std::unique_ptr<DevBuf>> slab_bufs;
  auto slabs_for = [&](const std::vector<int64_t>& b) -> const int64_t* {
    DevBuf* pos = new DevBuf(ctx);
    slab_bufs.emplace_back(pos);
    pos->alloc(sizeof(int64_t) * (size_t)n * b.size() + sizeof(int64_t) * b.size());
    int64_t* dbnd = pos->as<int64_t>() + (size_t)n * b.size();
    CB_CUDA(cudaMemcpyAsync(dbnd, b.data(), sizeof(int64_t) * b.size(), cudaMemcpyHostToDevice,
                            ctx->stream));
    cb::launch_slabs(dBfull, dbnd, (int)b.size(), pos->as<int64_t>(), ctx->stream, ctx->sms);
    CB_LAUNCHED();
    ctx->stats.kernels += 1;
    return pos->as<int64_t>();
  };
  // Exact sizing: nb equal ranges up front.  Learned sizing: ranges are cut
  // as the batches go, the first from the predicted total, every later one
  // from the output density (entries per column) the finished batches
  // showed, aiming at kFill of the budget, so that the predictor's bias
  // costs neither extra batches nor overflowing ones.
  // A resumed call (resume_col > 0) covers columns [resume_col, k) only.  With
  // exact sizing it retraces the full call's halvings: a range that holds
  // resume_col past its start must have overflowed in the full call, so it
  // is halved (the right half queued) until resume_col starts a range; the
  // ranges then follow in the full call's order.  A call resumed at the
  // col_lo of batch b thus forms batches b, b+1, ... as the full call did
  // (the batches are independent: paper Sec. 7.2).
  constexpr double kFill = 0.9;
  const bool adaptive = opt.sizing == CB_SIZING_LEARNED;
  const int64_t start = opt.resume_col;
  std::deque<Range> todo;
  int64_t next_lo = k;
  const int64_t* next_plo = nullptr;
  double width = 0.0;
  if (!adaptive) {
    size_t j = 0;  // the equal range [bnd[j], bnd[j+1]) holding start
    while (bnd[j + 1] <= start) ++j;
    int64_t a = bnd[j], b = bnd[j + 1];
    std::vector<int64_t> right;  // queued right halves' ends, outermost first
    while (a < start) {          // here b - a >= 2, so the halves are nonempty
      const int64_t mid = a + (b - a) / 2;
      if (start < mid) {
        right.push_back(b);
        b = mid;
      } else {
        a = mid;
      }
    }
    std::vector<int64_t> b2{start, b};
    for (auto it = right.rbegin(); it != right.rend(); ++it) b2.push_back(*it);
    for (size_t t = j + 1; t <= (size_t)nb; ++t)
      if (bnd[t] > b2.back()) b2.push_back(bnd[t]);
    const int64_t* pos = b_sorted ? slabs_for(b2) : nullptr;
    for (size_t q = 0; q + 1 < b2.size(); ++q)
      todo.push_back(Range{b2[q], b2[q + 1], pos ? pos + q * (size_t)n : nullptr,
                           pos ? pos + (q + 1) * (size_t)n : nullptr});
  } else {
    next_lo = start;
    next_plo = b_sorted ? slabs_for(std::vector<int64_t>{start}) : nullptr;
    width = (double)k * kFill * (double)cap / (double)std::max<int64_t>(total, 1);
  }
  int64_t done_cols = 0, done_nnz = 0;

  cb_opts inner = opt;
  inner.validate = 0;
  inner.budget_bytes = 0;
  inner.out_capacity = cap;
  int64_t nnz_sum = 0, batch = opt.resume_batch;
  int kernels = ctx->stats.kernels;
  for (;;) {
    if (todo.empty()) {
      if (next_lo >= k) break;
      const int64_t w = std::max<int64_t>(1, (int64_t)std::min(width, (double)k));
      const int64_t hi = std::min<int64_t>(k, next_lo + w);
      const int64_t* phi = b_sorted ? slabs_for(std::vector<int64_t>{hi}) : nullptr;
      todo.push_back(Range{next_lo, hi, next_plo, phi});
      next_lo = hi;
      next_plo = phi;
    }
    const Range r = todo.front();
    todo.pop_front();
    DevCSR view = dBfull;
    view.ncols = r.hi - r.lo;
    view.col_lo = r.lo;
    if (b_sorted) {
      view.rp = r.plo;
      view.rpe = r.phi;
    } else {
      view.filter = 1;
    }
    cb_csr Cb{m, k, 0, brp.as<int64_t>(), bcol.as<int32_t>(), bval.p};
    ctx->stats.kernels = 0;
    try {
      if (opt.sizing == CB_SIZING_EXACT || !(opt.flags & CB_FLAG_LEARNED_ROWS))
        spgemm_plain(ctx, sr, A, view, k, &Cb, inner);
      else spgemm_learned(ctx, sr, A, view, k, &Cb, inner);
    } catch (const Fail& f) {
      if (f.code != CB_ERR_CAPACITY) throw;
      kernels += ctx->stats.kernels;
      if (r.hi - r.lo <= 1)
        fail(ctx, CB_ERR_BUDGET, "one output column does not fit the batch budget");
      const int64_t mid = r.lo + (r.hi - r.lo) / 2;
      const int64_t* pmid = b_sorted ? slabs_for(std::vector<int64_t>{mid}) : nullptr;
      todo.push_front(Range{mid, r.hi, pmid, r.phi});
      todo.push_front(Range{r.lo, mid, r.plo, pmid});
      continue;
    }
    kernels += ctx->stats.kernels;
    nnz_sum += Cb.nnz;
    done_cols += r.hi - r.lo;
    done_nnz += Cb.nnz;
    if (adaptive)
      width = done_nnz > 0 ? kFill * (double)cap * (double)done_cols / (double)done_nnz : (double)k;
    CB_CUDA(cudaStreamSynchronize(ctx->stream));
    const int stop = opt.on_batch((int)batch, r.lo, r.hi, &Cb, opt.user);
    ++batch;
    if (stop) break;
  }
  ctx->stats.flops = sym_flops;
  ctx->stats.nnz = nnz_sum;
  ctx->stats.batches = (int32_t)(batch - opt.resume_batch);
  ctx->stats.kernels = kernels;
  C->nnz = nnz_sum;
}

// Per-row sizes of the product A.B (exact counts, or predictions with
// learned sizing) summed per group of rows: sums[j] = sum of rows
// [bounds[j], bounds[j+1]).  bounds is host memory (n + 1 values).
void row_group_sums(cb_ctx* ctx, const cb_csr* A, const DevCSR& dB, const cb_opts& opt,
                    const std::vector<int64_t>& bounds, std::vector<int64_t>& sums,
                    const int32_t* a_rcols = nullptr) {
  const int64_t m = A->nrows, n = (int64_t)bounds.size() - 1;
  DevBuf rows(ctx), pre(ctx), idx(ctx), got(ctx);
  rows.alloc(sizeof(int64_t) * (size_t)(m + 1));
  pre.alloc(sizeof(int64_t) * (size_t)(m + 1));
  idx.alloc(sizeof(int64_t) * bounds.size());
  got.alloc(sizeof(int64_t) * bounds.size());
  DevCSR dA = dev(A);
  dA.rcols = a_rcols;
  if (opt.sizing == CB_SIZING_LEARNED) {
    ensure(ctx, &ctx->ws, &ctx->ws_cap,
           align_up(sizeof(int64_t) * cb::kCounters) + align_up(8 * (size_t)(m + 1)) +
               align_up(4 * (size_t)(m + 1)) + align_up(16 * (size_t)(m + 1)));
    Carver cv{static_cast<char*>(ctx->ws)};
    int64_t* counters = cv.take<int64_t>(cb::kCounters);
    int64_t* flops = cv.take<int64_t>(m + 1);
    int32_t* maxb = cv.take<int32_t>(m + 1);
    float* feat = cv.take<float>(CB_MLP_NFEAT * (m + 1));
    CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
    cb::launch_classify_sym(dA, dB, flops, maxb, counters, ctx->stream, ctx->sms);
    cb::launch_row_features(dA, flops, maxb, dB.ncols, feat, ctx->stream, ctx->sms);
    cb::launch_mlp_predict(cb::mlp_bf16(opt.mlp), cb::mlp_master(opt.mlp), cb::mlp_norm(opt.mlp),
                           feat, m, dB.ncols, nullptr, rows.as<int64_t>(), ctx->stream, ctx->sms);
  } else {
    count_rows(ctx, dA, dB, rows.as<int64_t>());
  }
  ensure(ctx, &ctx->ws2, &ctx->ws2_cap, align_up(8 * (size_t)cb::scan_partials(m)));
  cb::launch_exclusive_scan(rows.as<int64_t>(), m, pre.as<int64_t>(), static_cast<int64_t*>(ctx->ws2),
                            ctx->stream);
  CB_CUDA(cudaMemcpyAsync(idx.p, bounds.data(), sizeof(int64_t) * bounds.size(),
                          cudaMemcpyHostToDevice, ctx->stream));
  cb::launch_gather(pre.as<int64_t>(), idx.as<int64_t>(), (int64_t)bounds.size(), got.as<int64_t>(),
                    ctx->stream);
  CB_LAUNCHED();
  std::vector<int64_t> h(bounds.size());
  CB_CUDA(cudaMemcpyAsync(h.data(), got.p, sizeof(int64_t) * h.size(), cudaMemcpyDeviceToHost,
                          ctx->stream));
  CB_CUDA(cudaStreamSynchronize(ctx->stream));
  sums.resize((size_t)n);
  double scale = opt.sizing == CB_SIZING_LEARNED ? 1.0 + (double)opt.margin : 1.0;
  for (int64_t j = 0; j < n; ++j) sums[(size_t)j] = (int64_t)((double)(h[(size_t)j + 1] - h[(size_t)j]) * scale);
}

// Per-product sums of flops_i (an upper bound of nnz(C_i)) over the stacked
// rows [bounds[j], bounds[j+1]), and the largest flops_i of any row.
void group_flops(cb_ctx* ctx, const cb_csr* A, const DevCSR& dB, const std::vector<int64_t>& bounds,
                 const int32_t* a_rcols, std::vector<int64_t>& sums, int64_t& max_flops) {
  const int64_t m = A->nrows, n = (int64_t)bounds.size() - 1;
  DevBuf flops(ctx), pre(ctx), idx(ctx), got(ctx), counters(ctx);
  flops.alloc(sizeof(int64_t) * (size_t)(m + 1));
  pre.alloc(sizeof(int64_t) * (size_t)(m + 1));
  idx.alloc(sizeof(int64_t) * bounds.size());
  got.alloc(sizeof(int64_t) * bounds.size());
  counters.alloc(sizeof(int64_t) * cb::kCounters);
  DevCSR dA = dev(A);
  dA.rcols = a_rcols;
  CB_CUDA(cudaMemsetAsync(counters.p, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
  cb::launch_classify_sym(dA, dB, flops.as<int64_t>(), nullptr, counters.as<int64_t>(), ctx->stream,
                          ctx->sms);
  ensure(ctx, &ctx->ws2, &ctx->ws2_cap, align_up(8 * (size_t)cb::scan_partials(m)));
  cb::launch_exclusive_scan(flops.as<int64_t>(), m, pre.as<int64_t>(), static_cast<int64_t*>(ctx->ws2),
                            ctx->stream);
  CB_CUDA(cudaMemcpyAsync(idx.p, bounds.data(), sizeof(int64_t) * bounds.size(),
                          cudaMemcpyHostToDevice, ctx->stream));
  cb::launch_gather(pre.as<int64_t>(), idx.as<int64_t>(), (int64_t)bounds.size(), got.as<int64_t>(),
                    ctx->stream);
  CB_LAUNCHED();
  std::vector<int64_t> h(bounds.size());
  CB_CUDA(cudaMemcpyAsync(h.data(), got.p, sizeof(int64_t) * h.size(), cudaMemcpyDeviceToHost,
                          ctx->stream));
  read_counters(ctx, counters.as<int64_t>(), nullptr, 0);  // synchronises
  max_flops = ctx->host[cb::kMaxFlops];
  sums.resize((size_t)n);
  for (int64_t j = 0; j < n; ++j) sums[(size_t)j] = h[(size_t)j + 1] - h[(size_t)j];
}

// What a CUDA-graph host node hands to the wave callback.
struct GraphWave {
  const cb_opts* opt;
  int wave, first, end;
  cb_csr C;
  const int64_t* nnz;  // pinned host word written by the graph before the node
};

void CUDART_CB graph_wave_host(void* p) {
  GraphWave* g = static_cast<GraphWave*>(p);
  g->C.nnz = *g->nnz;
  g->opt->on_batch(g->wave, g->first, g->end, &g->C, g->opt->user);
}

// Graph mode of a group: each wave runs a launch sequence without host
// synchronisation -- tier sizes, heavy-row and window counts stay on the
// device, C is sized by the wave's flop total, workspaces by upper bounds --
// and all waves are captured into one CUDA graph, launched once.  Returns
// false (nothing done) when a product's flop bound alone exceeds the budget.
bool batched_group_graph(cb_ctx* ctx, int sr, const cb_csr& sA, const DevCSR& dB, const int32_t* rcols,
                         const std::vector<int64_t>& arow, int n, int first, int64_t kmax,
                         const cb_opts& opt, int& wave, int& kernels, int64_t& nnz_total,
                         int64_t& flops_total, bool capture, const int64_t* prow_dev) {
  const int64_t vsz = (int64_t)value_size(sr), per = 4 + vsz;
  std::vector<int64_t> sizes;
  int64_t max_flops = 0;
  group_flops(ctx, &sA, dB, arow, rcols, sizes, max_flops);
  kernels += 3 + 3 + 1;
  const int64_t sym_max = ctx->tune.sym_hash_max;
  const int64_t num_max = std::min<int64_t>(ctx->tune.num_hash_max, cb::num_large_max(sr));
  const int64_t spans = (kmax + cb::kSpanCols - 1) / cb::kSpanCols;
  const int wcut = cb::num_window_cut(sr);
  // waves by the flop bound
  std::vector<int> cut{0};
  int64_t rows = 0, nz = 0;
  const int64_t budget = opt.budget_bytes > 0 ? opt.budget_bytes : INT64_MAX;
  for (int i = 0; i < n; ++i) {
    const int64_t ri = arow[i + 1] - arow[i];
    if (8 * (ri + 1) + sizes[(size_t)i] * per > budget) return false;  // host path sizes it exactly
    if (i > cut.back() && 8 * (rows + ri + 1) + (nz + sizes[(size_t)i]) * per > budget) {
      cut.push_back(i);
      rows = ri;
      nz = sizes[(size_t)i];
    } else {
      rows += ri;
      nz += sizes[(size_t)i];
    }
  }
  cut.push_back(n);
  const int nw = (int)cut.size() - 1;
  int64_t max_rows = 0, max_cap = 1, max_wins = 1;
  for (int w = 0; w < nw; ++w) {
    const int64_t r = arow[cut[w + 1]] - arow[cut[w]];
    max_rows = std::max(max_rows, r);
    int64_t f = 0;
    for (int i = cut[w]; i < cut[w + 1]; ++i) f += sizes[(size_t)i];
    max_cap = std::max(max_cap, f);
    // every (row, span) yields at most count / wcut + 1 windows; counts sum to <= flops
    max_wins = std::max(max_wins, r * spans + f / wcut + 1);
  }
  // everything the graph touches is allocated before the capture
  DevBuf orp(ctx), ocol(ctx), oval(ctx), wsb(ctx), errw(ctx), dscr(ctx);
  orp.alloc(8 * (size_t)(max_rows + 1));
  if (opt.digests) dscr.alloc(16 * (size_t)(max_rows + 1));
  ocol.alloc(4 * (size_t)max_cap);
  oval.alloc((size_t)vsz * (size_t)max_cap);
  const size_t mr = (size_t)max_rows + 1;
  const size_t units = (size_t)max_rows * (size_t)spans + 1;
  const size_t racc_bytes = cb::rank_scratch_bytes(sr, ctx->sms);
  const size_t wsz = align_up(8 * (size_t)cb::kCounters) + 2 * align_up(8 * mr) + 2 * align_up(4 * mr) +
                     align_up(8 * (size_t)cb::scan_partials(max_rows)) + align_up(4 * units) +
                     align_up(8 * units) + align_up(sizeof(cb::Window) * (size_t)max_wins) +
                     align_up(racc_bytes);
  wsb.alloc(wsz);
  errw.alloc(sizeof(int64_t));
  Carver cv{wsb.as<char>()};
  int64_t* counters = cv.take<int64_t>(cb::kCounters);
  int64_t* flops = cv.take<int64_t>(mr);
  int64_t* nnz = cv.take<int64_t>(mr);
  int32_t* perm_sym = cv.take<int32_t>(mr);
  int32_t* perm_num = cv.take<int32_t>(mr);
  int64_t* partial = cv.take<int64_t>(cb::scan_partials(max_rows));
  int32_t* span_counts = cv.take<int32_t>(units);
  int2* span_wins = cv.take<int2>(units);
  cb::Window* wins = cv.take<cb::Window>((size_t)max_wins);
  void* racc = racc_bytes ? cv.take<char>(racc_bytes) : nullptr;
  int64_t* hnnz = nullptr;
  CB_CUDA(cudaMallocHost((void**)&hnnz, sizeof(int64_t) * (size_t)nw));
  struct HostFree {
    int64_t* p;
    ~HostFree() { if (p) cudaFreeHost(p); }
  } hfree{hnnz};
  std::vector<GraphWave> gw((size_t)nw);
  CB_CUDA(cudaMemsetAsync(errw.p, 0, sizeof(int64_t), ctx->stream));
  // Rows of bounded size and width (every output row <= kQueueAcc entries,
  // <= kQueueWidth columns): each wave is one launch of the work-queue kernel.
  const bool queued = !(opt.flags & CB_FLAG_NO_FUSED) && max_flops <= cb::kQueueAcc &&
                      kmax <= cb::kQueueWidth;
  int* qstatus = nullptr;
  if (queued) {
    ensure_fused(ctx, max_rows);
    qstatus = reinterpret_cast<int*>(ctx->fsync + 4);
    CB_CUDA(cudaMemsetAsync(qstatus, 0, sizeof(int), ctx->stream));
  }
  cb::prepare_dev_launchers(sr);  // kernel attributes are set outside the capture
  CB_CUDA(cudaStreamSynchronize(ctx->stream));

  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // the legacy default stream cannot be captured: capture on a private
  // stream then (the context's stream is idle here, synchronised above)
  struct StreamSwap {
    cb_ctx* ctx;
    cudaStream_t saved, own = nullptr;
    ~StreamSwap() {
      ctx->stream = saved;
      if (own) {
        cudaStreamSynchronize(own);
        cudaStreamDestroy(own);
      }
    }
  } swap{ctx, ctx->stream};
  if (capture && (ctx->stream == nullptr || ctx->stream == cudaStreamLegacy ||
                  ctx->stream == cudaStreamPerThread)) {
    CB_CUDA(cudaStreamCreateWithFlags(&swap.own, cudaStreamNonBlocking));
    ctx->stream = swap.own;
  }
  if (capture) CB_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t cap_err = cudaSuccess;
  for (int w = 0; w < nw && cap_err == cudaSuccess; ++w) {
    const int64_t r0 = arow[cut[w]], m = arow[cut[w + 1]] - r0;
    const cb_csr Aw{m, sA.ncols, 0, sA.row_ptr + r0, sA.col, sA.val};
    DevCSR dA = dev(&Aw);
    dA.rcols = rcols + r0;
    if (queued) {
      const cudaError_t qe = cb::launch_queue_rows(sr, dA, dB, m, orp.as<int64_t>(), ocol.as<int32_t>(),
                                                   oval.p, max_cap, ctx->fstat, ctx->fstat_cap,
                                                   ctx->fsync, qstatus, ctx->stream, ctx->sms,
                                                   ctx->fused_spin, ctx->fused_silent);
      if (qe != cudaSuccess) {
        if (!capture) {
          ctx->err = std::string("queued SpGEMM launch: ") + cudaGetErrorString(qe);
          throw Fail{CB_ERR_CUDA};
        }
        if (cap_err == cudaSuccess) cap_err = qe;
      }
      kernels += 1;
    } else {
      cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream);
      cb::launch_check_sorted(dB, counters, ctx->stream, ctx->sms);
      cb::launch_classify_sym(dA, dB, flops, nullptr, counters, ctx->stream, ctx->sms, nullptr, sym_max);
      cb::launch_scatter_sym(m, kmax, flops, perm_sym, nnz, counters, ctx->stream, ctx->sms, nullptr,
                             nullptr, sym_max, dA.rcols);
      cb::launch_symbolic_dev(dA, dB, perm_sym, counters, flops, nnz, span_counts, span_wins, wcut, wins,
                              max_wins, ctx->stream, ctx->sms);
      cb::launch_exclusive_scan(nnz, m, orp.as<int64_t>(), partial, ctx->stream);
      cb::launch_classify_num(sr, m, nnz, perm_num, counters, ctx->stream, ctx->sms, nullptr, num_max);
      cb::launch_numeric_dev(sr, dA, dB, perm_num, counters, flops, nnz, orp.as<int64_t>(),
                             ocol.as<int32_t>(), oval.p, errw.as<int64_t>(), ctx->stream, ctx->sms,
                             perm_sym, wins, span_counts, spans, racc, num_max,
                             cb::CfBounds{ctx->tune.cf_esc, ctx->tune.cf_pre});
      // the symbolic phase's consistency word (window capacity, span cut) joins the error word
      cb::launch_merge_error(counters + cb::kError, errw.as<int64_t>(), ctx->stream);
      kernels += 2 + 2 + 3 + 3 + 2 + 3;
    }
    if (opt.digests) {
      cb::launch_digest((int)value_size(sr), sr == CB_PLUS_TIMES_F64, orp.as<int64_t>(), ocol.as<int32_t>(),
                        oval.p, m, prow_dev + cut[w], cut[w + 1] - cut[w], r0, dscr.as<uint64_t>(),
                        reinterpret_cast<double*>(dscr.as<uint64_t>() + max_rows + 1),
                        opt.digests + 2 * (size_t)(first + cut[w]), ctx->stream, ctx->sms);
      kernels += m > 0 ? 2 : 1;
    }
    cudaMemcpyAsync(hnnz + w, orp.as<int64_t>() + m, sizeof(int64_t), cudaMemcpyDeviceToHost,
                    ctx->stream);
    gw[(size_t)w] = GraphWave{&opt, wave + w, first + cut[w], first + cut[w + 1],
                              cb_csr{m, kmax, 0, orp.as<int64_t>(), ocol.as<int32_t>(), oval.p},
                              hnnz + w};
    if (capture) {
      cudaLaunchHostFunc(ctx->stream, graph_wave_host, &gw[(size_t)w]);
      cap_err = cudaGetLastError();
    } else {
      // the same launch sequence without the capture: the callback runs on this
      // thread after the wave (and may use CUDA)
      CB_LAUNCHED();
      CB_CUDA(cudaStreamSynchronize(ctx->stream));
      gw[(size_t)w].C.nnz = hnnz[w];
      const int stop = opt.on_batch(gw[(size_t)w].wave, gw[(size_t)w].first, gw[(size_t)w].end,
                                    &gw[(size_t)w].C, opt.user);
      if (stop) {
        for (int v = 0; v <= w; ++v) nnz_total += hnnz[v];
        wave += w + 1;
        throw Fail{-1};
      }
    }
  }
  // status bits of the work-queue kernel (all waves)
  const auto check_queue = [&]() {
    if (!queued) return;
    int bits = 0;
    CB_CUDA(cudaMemcpy(&bits, qstatus, sizeof(int), cudaMemcpyDeviceToHost));
    if (bits & CB_FUSED_STALLED) fail(ctx, CB_ERR_TIMEOUT, "queued SpGEMM: a row wait expired");
    if (bits) fail(ctx, CB_ERR_CUDA, "queued SpGEMM: row bound or capacity violated");
  };
  if (!capture) {
    int64_t err_word = 0;
    CB_CUDA(cudaMemcpy(&err_word, errw.p, sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (err_word) fail(ctx, CB_ERR_CUDA, "sync-free wave: internal consistency check failed");
    check_queue();
    for (int w = 0; w < nw; ++w) nnz_total += hnnz[w];
    for (int i = 0; i < n; ++i) flops_total += sizes[(size_t)i];
    wave += nw;
    return true;
  }
  const cudaError_t end_err = cudaStreamEndCapture(ctx->stream, &graph);
  if (cap_err != cudaSuccess || end_err != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    ctx->err = std::string("graph capture: ") +
               cudaGetErrorString(cap_err != cudaSuccess ? cap_err : end_err);
    throw Fail{CB_ERR_CUDA};
  }
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    ctx->err = std::string("graph instantiate: ") + cudaGetErrorString(ie);
    throw Fail{CB_ERR_CUDA};
  }
  const cudaError_t le = cudaGraphLaunch(exec, ctx->stream);
  const cudaError_t se = cudaStreamSynchronize(ctx->stream);
  cudaGraphExecDestroy(exec);
  CB_CUDA(le);
  CB_CUDA(se);
  int64_t err_word = 0;
  CB_CUDA(cudaMemcpy(&err_word, errw.p, sizeof(int64_t), cudaMemcpyDeviceToHost));
  if (err_word) fail(ctx, CB_ERR_CUDA, "graph wave: internal consistency check failed");
  check_queue();
  for (int w = 0; w < nw; ++w) nnz_total += hnnz[w];
  for (int i = 0; i < n; ++i) flops_total += sizes[(size_t)i];
  wave += nw;
  return true;
}

// One run of consecutive products that share a semiring (see cb_spgemm_batched).
void batched_group(cb_ctx* ctx, int sr, const cb_csr* A, const cb_csr* B, int n, int first,
                   const cb_opts& opt, int& wave, int& kernels, int64_t& nnz_total,
                   int64_t& flops_total) {
  const int64_t vsz = (int64_t)value_size(sr), per = 4 + vsz;
  int64_t rowsA = 0, nnzA = 0, rowsB = 0, nnzB = 0, kmax = 0;
  std::vector<int64_t> arow(n + 1), brow(n + 1);
  for (int i = 0; i < n; ++i) {
    arow[i] = rowsA;
    brow[i] = rowsB;
    rowsA += A[i].nrows;
    nnzA += A[i].nnz;
    rowsB += B[i].nrows;
    nnzB += B[i].nnz;
    kmax = B[i].ncols > kmax ? B[i].ncols : kmax;
  }
  arow[n] = rowsA;
  brow[n] = rowsB;
  if (rowsA >= INT32_MAX || rowsB > INT32_MAX)
    fail(ctx, CB_ERR_INDEX, "batch too large to stack (rows beyond int32); split it");
  // stack the group once
  DevBuf sArp(ctx), sAcol(ctx), sAval(ctx), sBrp(ctx), sBcol(ctx), sBval(ctx), parts(ctx), rcols(ctx);
  sArp.alloc(8 * (size_t)(rowsA + 1));
  rcols.alloc(4 * (size_t)(rowsA + 1));
  sAcol.alloc(4 * (size_t)nnzA);
  const int64_t avs = (int64_t)a_value_size(sr), bvs = (int64_t)b_value_size(sr);
  sAval.alloc((size_t)avs * (size_t)nnzA);
  sBrp.alloc(8 * (size_t)(rowsB + 1));
  sBcol.alloc(4 * (size_t)nnzB);
  sBval.alloc((size_t)bvs * (size_t)nnzB);
  const size_t psz = cb::stack_part_size();
  parts.alloc(2 * (size_t)n * psz);
  std::vector<unsigned char> hp(2 * (size_t)n * psz);
  int64_t ao = 0, bo = 0;
  for (int i = 0; i < n; ++i) {
    cb::fill_stack_part(&hp[(size_t)i * psz], A[i].row_ptr, A[i].col, A[i].val, A[i].nrows, arow[i], ao,
                        (int32_t)brow[i], (int32_t)B[i].ncols);
    cb::fill_stack_part(&hp[(size_t)(n + i) * psz], B[i].row_ptr, B[i].col, B[i].val, B[i].nrows,
                        brow[i], bo, 0, (int32_t)B[i].ncols);
    ao += A[i].nnz;
    bo += B[i].nnz;
  }
  CB_CUDA(cudaMemcpyAsync(parts.p, hp.data(), hp.size(), cudaMemcpyHostToDevice, ctx->stream));
  cb::launch_stack(parts.p, n, (int)avs, sArp.as<int64_t>(), sAcol.as<int32_t>(), sAval.p,
                   rcols.as<int32_t>(), ctx->stream, ctx->sms);
  cb::launch_stack(static_cast<char*>(parts.p) + (size_t)n * psz, n, (int)bvs, sBrp.as<int64_t>(),
                   sBcol.as<int32_t>(), sBval.p, nullptr, ctx->stream, ctx->sms);
  CB_LAUNCHED();
  kernels += 2;
  const DevCSR dB{rowsB, kmax, sBrp.as<int64_t>(), sBcol.as<int32_t>(), sBval.p};
  const cb_csr sA{rowsA, rowsB, nnzA, sArp.as<int64_t>(), sAcol.as<int32_t>(), sAval.p};
  // digests: every product's first stacked row, on the device
  DevBuf prow(ctx);
  if (opt.digests) {
    prow.alloc(8 * (size_t)(n + 1));
    CB_CUDA(cudaMemcpyAsync(prow.p, arow.data(), 8 * (size_t)(n + 1), cudaMemcpyHostToDevice,
                            ctx->stream));
  }
  if ((opt.flags & (CB_FLAG_GRAPH | CB_FLAG_SYNC_FREE)) &&
      batched_group_graph(ctx, sr, sA, dB, rcols.as<int32_t>(), arow, n, first, kmax, opt, wave,
                          kernels, nnz_total, flops_total, (opt.flags & CB_FLAG_GRAPH) != 0,
                          prow.as<int64_t>()))
    return;

  // waves: consecutive products whose output fits the budget
  std::vector<int> cut{0};
  if (opt.budget_bytes > 0) {
    std::vector<int64_t> sizes;
    row_group_sums(ctx, &sA, dB, opt, arow, sizes, rcols.as<int32_t>());
    int64_t rows = 0, nz = 0;
    for (int i = 0; i < n; ++i) {
      if (8 * (A[i].nrows + 1) + sizes[(size_t)i] * per > opt.budget_bytes) {
        if (opt.sizing == CB_SIZING_EXACT || 8 * (A[i].nrows + 1) + per > opt.budget_bytes)
          fail(ctx, CB_ERR_BUDGET, "one product's output does not fit the wave budget");
        // a prediction above the budget: the product gets a wave of its own
        // (its exact output is checked against the budget when it runs)
        sizes[(size_t)i] = (opt.budget_bytes - 8 * (A[i].nrows + 1)) / per;
      }
      const int64_t r2 = rows + A[i].nrows, z2 = nz + sizes[(size_t)i];
      if (i > cut.back() && 8 * (r2 + 1) + z2 * per > opt.budget_bytes) {
        cut.push_back(i);
        rows = A[i].nrows;
        nz = sizes[(size_t)i];
      } else {
        rows = r2;
        nz = z2;
      }
    }
  }
  cut.push_back(n);

  cb_opts inner = opt;
  inner.validate = 0;
  inner.budget_bytes = 0;
  DevBuf orp(ctx), ocol(ctx), oval(ctx), dscr(ctx);
  int64_t max_wave_rows = 1;
  for (size_t w = 0; w + 1 < cut.size(); ++w)
    max_wave_rows = std::max(max_wave_rows, arow[cut[w + 1]] - arow[cut[w]]);
  if (opt.digests) dscr.alloc(16 * (size_t)(max_wave_rows + 1));
  int64_t cap = 0;
  if (opt.budget_bytes > 0) {
    int64_t max_rows = 0;
    for (size_t w = 0; w + 1 < cut.size(); ++w)
      max_rows = std::max(max_rows, arow[cut[w + 1]] - arow[cut[w]]);
    cap = (opt.budget_bytes - 8 * (max_rows + 1)) / per;
    orp.alloc(8 * (size_t)(max_rows + 1));
    ocol.alloc(4 * (size_t)std::max<int64_t>(cap, 1));
    oval.alloc((size_t)vsz * (size_t)std::max<int64_t>(cap, 1));
    inner.out_capacity = std::max<int64_t>(cap, 1);
  }
  for (size_t w = 0; w + 1 < cut.size(); ++w) {
    int w0 = cut[w];
    const int w1 = cut[w + 1];
    const cb_csr Aw{arow[w1] - arow[w0], rowsB, 0, sArp.as<int64_t>() + arow[w0], sAcol.as<int32_t>(),
                    sAval.p};
    cb_csr Cw{};
    if (inner.out_capacity > 0) Cw = cb_csr{0, 0, 0, orp.as<int64_t>(), ocol.as<int32_t>(), oval.p};
    ctx->stats.kernels = 0;
    const int32_t* wr = rcols.as<int32_t>() + arow[w0];
    try {
      if (opt.sizing == CB_SIZING_EXACT || !(opt.flags & CB_FLAG_LEARNED_ROWS))
        spgemm_plain(ctx, sr, &Aw, dB, kmax, &Cw, inner, nullptr, nullptr, wr);
      else spgemm_learned(ctx, sr, &Aw, dB, kmax, &Cw, inner, wr);
    } catch (const Fail&) {
      if (inner.out_capacity == 0)  // the wave's own output, allocated by the pipeline
        for (void* q : {(void*)Cw.row_ptr, (void*)Cw.col, Cw.val})
          if (q) cudaFreeAsync(q, ctx->stream);
      throw;
    }
    kernels += ctx->stats.kernels;
    nnz_total += Cw.nnz;
    flops_total += ctx->stats.flops;
    if (opt.digests) {
      const int64_t mw = arow[w1] - arow[w0];
      cb::launch_digest((int)value_size(sr), sr == CB_PLUS_TIMES_F64, Cw.row_ptr, Cw.col, Cw.val, mw,
                        prow.as<int64_t>() + w0, w1 - w0, arow[w0], dscr.as<uint64_t>(),
                        reinterpret_cast<double*>(dscr.as<uint64_t>() + max_wave_rows + 1),
                        opt.digests + 2 * (size_t)(first + w0), ctx->stream, ctx->sms);
      CB_LAUNCHED();
      kernels += mw > 0 ? 2 : 1;
    }
    CB_CUDA(cudaStreamSynchronize(ctx->stream));
    const int stop = opt.on_batch(wave++, first + w0, first + w1, &Cw, opt.user);
    if (inner.out_capacity == 0) {
      for (void* q : {(void*)Cw.row_ptr, (void*)Cw.col, Cw.val})
        if (q) CB_CUDA(cudaFreeAsync(q, ctx->stream));
    }
    if (stop) throw Fail{-1};
  }
}

}  // namespace

namespace cb {
cudaStream_t ctx_stream(cb_ctx* ctx) { return ctx->stream; }
int ctx_sms(cb_ctx* ctx) { return ctx->sms; }
}  // namespace cb

extern "C" {

int cb_row_features(cb_ctx* ctx, const cb_csr* A, const cb_csr* B, float* feat) {
  if (!ctx) return CB_ERR_ARG;
  ctx->err.clear();
  try {
    if (!A || !B || !feat) fail(ctx, CB_ERR_ARG, "null argument");
    check_operand(ctx, A, "A");
    check_operand(ctx, B, "B");
    if (A->ncols != B->nrows) fail(ctx, CB_ERR_SHAPE, "A.ncols != B.nrows");
    const int64_t m = A->nrows;
    if (m == 0) return CB_OK;
    size_t need = align_up(sizeof(int64_t) * cb::kCounters) + align_up(8 * (size_t)m + 8) +
                  align_up(4 * (size_t)m + 4);  // feat is the caller's
    ensure(ctx, &ctx->ws, &ctx->ws_cap, need);
    Carver cv{static_cast<char*>(ctx->ws)};
    int64_t* counters = cv.take<int64_t>(cb::kCounters);
    int64_t* flops = cv.take<int64_t>(m + 1);
    int32_t* maxb = cv.take<int32_t>(m + 1);
    CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
    cb::launch_classify_sym(dev(A), dev(B), flops, maxb, counters, ctx->stream, ctx->sms);
    cb::launch_row_features(dev(A), flops, maxb, B->ncols, feat, ctx->stream, ctx->sms);
    CB_LAUNCHED();
    return CB_OK;
  } catch (const Fail& f) {
    return f.code;
  }
}

int64_t cb_struct_size(int which) {
  switch (which) {
    case 0: return (int64_t)sizeof(cb_csr);
    case 1: return (int64_t)sizeof(cb_opts);
    case 2: return (int64_t)sizeof(cb_tune);
    case 3: return (int64_t)sizeof(cb_stats);
    case 4: return (int64_t)sizeof(cb_spvec);
    case 5: return (int64_t)sizeof(cb_wlabel);
  }
  return -1;
}

void cb_opts_default(cb_opts* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->sizing = CB_SIZING_EXACT;
  opt->validate = 1;
  opt->margin = 0.25f;
}

int cb_ctx_create(cb_ctx** out, void* stream) {
  if (!out) return CB_ERR_ARG;
  *out = nullptr;
  cb_ctx* ctx = new (std::nothrow) cb_ctx();
  if (!ctx) return CB_ERR_OOM;
  ctx->stream = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->host, sizeof(int64_t) * (cb::kCounters + 64)) != cudaSuccess) {
    delete ctx;
    return CB_ERR_CUDA;
  }
  *out = ctx;
  return CB_OK;
}

void cb_ctx_destroy(cb_ctx* ctx) {
  if (!ctx) return;
  if (ctx->ws || ctx->ws2) cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->ws2) cudaFree(ctx->ws2);
  if (ctx->host) cudaFreeHost(ctx->host);
  if (ctx->fstat || ctx->fsync) cudaStreamSynchronize(ctx->stream);
  if (ctx->fstat) cudaFree(ctx->fstat);
  if (ctx->fsync) cudaFree(ctx->fsync);
  if (ctx->spa || ctx->spa_bits) cudaStreamSynchronize(ctx->stream);
  if (ctx->spa) cudaFree(ctx->spa);
  if (ctx->spa_bits) cudaFree(ctx->spa_bits);
  for (cudaEvent_t e : ctx->ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

int cb_ctx_set_stream(cb_ctx* ctx, void* stream) {
  if (!ctx) return CB_ERR_ARG;
  if (ctx->stream != static_cast<cudaStream_t>(stream)) {
    // Workspace was allocated in the old stream's order; finish that work first.
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return CB_ERR_CUDA;
    ctx->stream = static_cast<cudaStream_t>(stream);
  }
  return CB_OK;
}

const char* cb_last_error(const cb_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

const char* cb_status_str(int s) {
  switch (s) {
    case CB_OK: return "ok";
    case CB_ERR_ARG: return "invalid argument";
    case CB_ERR_SHAPE: return "shape mismatch (A.ncols != B.nrows)";
    case CB_ERR_SEMIRING: return "unknown semiring";
    case CB_ERR_INDEX: return "invalid CSR index data";
    case CB_ERR_OOM: return "device out of memory";
    case CB_ERR_BUDGET: return "output budget too small";
    case CB_ERR_TIMEOUT: return "bounded device wait expired";
    case CB_ERR_CUDA: return "CUDA error";
    case CB_ERR_CAPACITY: return "caller-provided output too small";
    case CB_ERR_SCRATCH: return "size beyond the static scratch capacity";
  }
  return "unknown status";
}

int cb_spgemm_ex(cb_ctx* ctx, cb_semiring sr, const cb_csr* A, const cb_csr* B, cb_csr* C,
                 const cb_opts* opt_in) {
  if (!ctx) return CB_ERR_ARG;
  ctx->err.clear();
  ctx->stats = cb_stats{};
  ctx->stats.batches = 1;
  cb_opts opt;
  if (opt_in) opt = *opt_in;
  else cb_opts_default(&opt);
  const bool caller_buf = opt.out_capacity > 0;
  cb_csr saved{};
  if (C) saved = *C;
  try {
    if (!A || !B || !C) fail(ctx, CB_ERR_ARG, "null matrix argument");
    if (!public_semiring(sr)) fail(ctx, CB_ERR_SEMIRING, "unknown semiring");
    check_operand(ctx, A, "A");
    check_operand(ctx, B, "B");
    if (A->ncols != B->nrows) fail(ctx, CB_ERR_SHAPE, "A.ncols != B.nrows");
    if (caller_buf && (!C->row_ptr || !C->col || !C->val))
      fail(ctx, CB_ERR_ARG, "out_capacity > 0 needs C->row_ptr, C->col and C->val");
    if (opt.sizing != CB_SIZING_EXACT && opt.sizing != CB_SIZING_LEARNED &&
        opt.sizing != CB_SIZING_UPPER_BOUND)
      fail(ctx, CB_ERR_ARG, "unknown sizing mode");
    if (opt.sizing == CB_SIZING_LEARNED && !opt.mlp) fail(ctx, CB_ERR_ARG, "learned sizing needs opt->mlp");
    if (!(opt.margin >= 0.0f)) fail(ctx, CB_ERR_ARG, "margin must be >= 0");
    if (opt.budget_bytes > 0) {
      if (!opt.on_batch) fail(ctx, CB_ERR_ARG, "budget_bytes > 0 needs on_batch");
      spgemm_colbatch(ctx, (int)sr, A, B, C, opt);
      check_words(ctx);
      return CB_OK;
    }
    if (opt.validate) run_validation(ctx, A, B);
    if (opt.sizing == CB_SIZING_EXACT)
      spgemm_plain(ctx, (int)sr, A, dev(B), B->ncols, C, opt, nullptr, nullptr, nullptr, B->nnz);
    else spgemm_learned(ctx, (int)sr, A, dev(B), B->ncols, C, opt);
    check_words(ctx);
    return CB_OK;
  } catch (const Fail& f) {
    if (!caller_buf && C) {
      if (C->row_ptr && C->row_ptr != saved.row_ptr) cudaFreeAsync(C->row_ptr, ctx->stream);
      if (C->col && C->col != saved.col) cudaFreeAsync(C->col, ctx->stream);
      if (C->val && C->val != saved.val) cudaFreeAsync(C->val, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      std::memset(C, 0, sizeof *C);
    }
    return f.code;
  }
}

int cb_spgemm_fused(cb_ctx* ctx, cb_semiring sr, const cb_csr* A, const cb_csr* B, cb_csr* C,
                    int64_t capacity, int lanes, int* status) {
  if (!ctx) return CB_ERR_ARG;
  ctx->err.clear();
  ctx->stats = cb_stats{};
  ctx->stats.batches = 1;
  try {
    if (!A || !B || !C || !status) fail(ctx, CB_ERR_ARG, "null argument");
    if (!public_semiring(sr)) fail(ctx, CB_ERR_SEMIRING, "unknown semiring");
    check_operand(ctx, A, "A");
    check_operand(ctx, B, "B");
    if (A->ncols != B->nrows) fail(ctx, CB_ERR_SHAPE, "A.ncols != B.nrows");
    if (lanes != 8 && lanes != 16 && lanes != 32) fail(ctx, CB_ERR_ARG, "lanes must be 8, 16 or 32");
    if (B->ncols > cb::fused_max_cols(lanes))
      fail(ctx, CB_ERR_ARG, "B.ncols beyond the fused path's column bound for these lanes");
    if (capacity < 0 || !C->row_ptr || (capacity > 0 && (!C->col || !C->val)))
      fail(ctx, CB_ERR_ARG, "C needs row_ptr, and col/val for capacity > 0");
    C->nrows = A->nrows;
    C->ncols = B->ncols;
    C->nnz = -1;
    run_fused(ctx, (int)sr, lanes, dev(A), dev(B), C->row_ptr, C->col, C->val, capacity, status);
    check_words(ctx);
    return CB_OK;
  } catch (const Fail& f) {
    return f.code;
  }
}

int64_t cb_fused_max_cols(int lanes) {
  return (lanes == 8 || lanes == 16 || lanes == 32) ? cb::fused_max_cols(lanes) : 0;
}

int cb_fused_lanes(cb_ctx* ctx, const cb_csr* A, const cb_csr* B, int* lanes, int64_t* flops) {
  if (!ctx) return CB_ERR_ARG;
  ctx->err.clear();
  try {
    if (!A || !B || !lanes) fail(ctx, CB_ERR_ARG, "null argument");
    check_operand(ctx, A, "A");
    check_operand(ctx, B, "B");
    if (A->ncols != B->nrows) fail(ctx, CB_ERR_SHAPE, "A.ncols != B.nrows");
    const int64_t m = A->nrows;
    size_t need = align_up(sizeof(int64_t) * cb::kCounters) + align_up(8 * (size_t)m + 8);
    ensure(ctx, &ctx->ws, &ctx->ws_cap, need);
    Carver cv{static_cast<char*>(ctx->ws)};
    int64_t* counters = cv.take<int64_t>(cb::kCounters);
    int64_t* f = cv.take<int64_t>(m + 1);
    CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
    if (m > 0) cb::launch_classify_sym(dev(A), dev(B), f, nullptr, counters, ctx->stream, ctx->sms);
    CB_LAUNCHED();
    read_counters(ctx, counters, nullptr, 0);
    *lanes = fused_fit(ctx->host[cb::kMaxArow], ctx->host[cb::kMaxFlops], B->ncols);
    if (flops) *flops = ctx->host[cb::kTotalFlops];
    return CB_OK;
  } catch (const Fail& f) {
    return f.code;
  }
}

int cb_spgemm(cb_semiring sr, const cb_csr* A, const cb_csr* B, cb_csr* C) {
  cb_ctx* ctx = nullptr;
  int rc = cb_ctx_create(&ctx, nullptr);
  if (rc != CB_OK) return rc;
  rc = cb_spgemm_ex(ctx, sr, A, B, C, nullptr);
  if (rc == CB_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    rc = CB_ERR_CUDA;
    cb_csr_free(C);
  }
  cb_ctx_destroy(ctx);
  return rc;
}

void cb_csr_free(cb_csr* C) {
  if (!C) return;
  if (C->row_ptr || C->col || C->val) cudaDeviceSynchronize();
  if (C->row_ptr) cudaFree(C->row_ptr);
  if (C->col) cudaFree(C->col);
  if (C->val) cudaFree(C->val);
  std::memset(C, 0, sizeof *C);
}

int cb_csr_free_async(cb_ctx* ctx, cb_csr* C) {
  if (!ctx || !C) return CB_ERR_ARG;
  int rc = CB_OK;
  for (void* p : {(void*)C->row_ptr, (void*)C->col, C->val})
    if (p && cudaFreeAsync(p, ctx->stream) != cudaSuccess) rc = CB_ERR_CUDA;
  std::memset(C, 0, sizeof *C);
  return rc;
}

int cb_row_stats(cb_ctx* ctx, const cb_csr* A, const cb_csr* B, int64_t* flops, int32_t* maxb) {
  if (!ctx) return CB_ERR_ARG;
  ctx->err.clear();
  try {
    if (!A || !B) fail(ctx, CB_ERR_ARG, "null matrix argument");
    check_operand(ctx, A, "A");
    check_operand(ctx, B, "B");
    if (A->ncols != B->nrows) fail(ctx, CB_ERR_SHAPE, "A.ncols != B.nrows");
    const int64_t m = A->nrows;
    size_t need = align_up(sizeof(int64_t) * cb::kCounters) + align_up(8 * (size_t)m + 8);
    ensure(ctx, &ctx->ws, &ctx->ws_cap, need);
    Carver cv{static_cast<char*>(ctx->ws)};
    int64_t* counters = cv.take<int64_t>(cb::kCounters);
    int64_t* f = flops ? flops : cv.take<int64_t>(m + 1);
    if (m == 0) return CB_OK;
    CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
    cb::launch_classify_sym(dev(A), dev(B), f, maxb, counters, ctx->stream, ctx->sms);
    CB_LAUNCHED();
    return CB_OK;
  } catch (const Fail& f) {
    return f.code;
  }
}

int cb_row_nnz(cb_ctx* ctx, const cb_csr* A, const cb_csr* B, int64_t* nnz_out) {
  if (!ctx) return CB_ERR_ARG;
  ctx->err.clear();
  try {
    if (!A || !B || !nnz_out) fail(ctx, CB_ERR_ARG, "null argument");
    check_operand(ctx, A, "A");
    check_operand(ctx, B, "B");
    if (A->ncols != B->nrows) fail(ctx, CB_ERR_SHAPE, "A.ncols != B.nrows");
    count_rows(ctx, dev(A), dev(B), nnz_out);
    return CB_OK;
  } catch (const Fail& f) {
    return f.code;
  }
}

int cb_exclusive_scan(cb_ctx* ctx, const int64_t* in, int64_t n, int64_t* out) {
  if (!ctx) return CB_ERR_ARG;
  ctx->err.clear();
  try {
    if (n < 0 || !out || (n > 0 && !in)) fail(ctx, CB_ERR_ARG, "bad scan arguments");
    ensure(ctx, &ctx->ws, &ctx->ws_cap, align_up(8 * (size_t)cb::scan_partials(n)));
    cb::launch_exclusive_scan(in, n, out, static_cast<int64_t*>(ctx->ws), ctx->stream);
    CB_LAUNCHED();
    return CB_OK;
  } catch (const Fail& f) {
    return f.code;
  }
}

// The bucket (propagation-blocking) SpMSpV: no state kept across calls; two
// synchronisations (the product count, to size the buckets, and nnz(y)).
void spmspv_bucket(cb_ctx* ctx, int sr, const cb_csr* A, const cb_spvec* x, cb_spvec* y,
                   const cb_opts& opt, bool caller_buf) {
  const int64_t n = A->ncols, nx = x->nnz;
  const int64_t nb = cb::spmspv_buckets(n);
  const size_t vsz = value_size(sr), avs = cb::spa_value_size(sr);
  const int64_t big = std::max(nx, nb);
  ensure(ctx, &ctx->ws, &ctx->ws_cap,
         align_up(sizeof(int64_t) * cb::kCounters) + 2 * align_up(8 * (size_t)(nx + 1)) +
             4 * align_up(8 * (size_t)(nb + 1)) + align_up(8 * (size_t)cb::scan_partials(big)));
  Carver cv{static_cast<char*>(ctx->ws)};
  int64_t* counters = cv.take<int64_t>(cb::kCounters);
  int64_t* chunks = cv.take<int64_t>(nx + 1);
  int64_t* cpre = cv.take<int64_t>(nx + 1);
  int64_t* cur = cv.take<int64_t>(nb + 1);
  int64_t* bpre = cv.take<int64_t>(nb + 1);
  int64_t* bnnz = cv.take<int64_t>(nb + 1);
  int64_t* ypre = cv.take<int64_t>(nb + 1);
  int64_t* partial = cv.take<int64_t>(cb::scan_partials(big));
  const DevCSR dA = dev(A);
  unsigned long long* ucur = reinterpret_cast<unsigned long long*>(cur);
  // per-CTA bucket counters when the buckets fit shared memory
  const int ncta = cb::spmspv_priv_ctas(nb, ctx->sms);
  DevBuf ccnt(ctx);
  if (ncta) ccnt.alloc(sizeof(int64_t) * (size_t)ncta * (size_t)nb);
  CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
  CB_CUDA(cudaMemsetAsync(cur, 0, sizeof(int64_t) * (size_t)(nb + 1), ctx->stream));
  mark(ctx, opt, 0);
  cb::launch_spmspv_step(sr, 1, dA, x->idx, x->val, nx, chunks, nullptr, nullptr, nullptr, n, nullptr,
                         nullptr, nullptr, nullptr, 0, counters + cb::kError, ctx->stream, ctx->sms);
  cb::launch_exclusive_scan(chunks, nx, cpre, partial, ctx->stream);
  if (ncta) {
    cb::launch_spmspv_bucket_priv(sr, 0, dA, x->idx, x->val, nx, cpre, nb, ccnt.as<int64_t>(), nullptr,
                                  nullptr, nullptr, nullptr, ctx->stream, ctx->sms);
    cb::launch_spmspv_bucket_priv(sr, 2, dA, nullptr, nullptr, 0, nullptr, nb, ccnt.as<int64_t>(), nullptr,
                                  cur, nullptr, nullptr, ctx->stream, ctx->sms);
  } else {
    cb::launch_spmspv_bucket_step(sr, 0, dA, x->idx, x->val, nx, cpre, ucur, nullptr, nullptr, nullptr,
                                  nb, n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0,
                                  ctx->stream, ctx->sms);
  }
  cb::launch_exclusive_scan(cur, nb, bpre, partial, ctx->stream);
  CB_LAUNCHED();
  read_counters(ctx, counters, bpre + nb, 1);
  const int64_t products = ctx->host[cb::kCounters];
  if (ctx->host[cb::kError]) fail(ctx, CB_ERR_INDEX, "an index of x is outside [0, A.nrows)");
  ctx->stats.flops = products;
  ctx->stats.kernels += 4;
  if (products == 0) {
    for (int e = 1; e <= 5; ++e) mark(ctx, opt, e);
    collect_times(ctx, opt, true);
    return;
  }
  DevBuf bcol(ctx), bval(ctx), scol(ctx), sval(ctx);
  bcol.alloc(4 * (size_t)products);
  bval.alloc(avs * (size_t)products);
  scol.alloc(4 * (size_t)products);
  sval.alloc(vsz * (size_t)products);
  if (ncta) {
    cb::launch_spmspv_bucket_priv(sr, 1, dA, x->idx, x->val, nx, cpre, nb, ccnt.as<int64_t>(), bpre,
                                  nullptr, bcol.as<int32_t>(), bval.p, ctx->stream, ctx->sms);
  } else {
    CB_CUDA(cudaMemcpyAsync(cur, bpre, sizeof(int64_t) * (size_t)nb, cudaMemcpyDeviceToDevice,
                            ctx->stream));
    cb::launch_spmspv_bucket_step(sr, 1, dA, x->idx, x->val, nx, cpre, ucur, bcol.as<int32_t>(), bval.p,
                                  nullptr, nb, n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0,
                                  ctx->stream, ctx->sms);
  }
  cb::launch_spmspv_bucket_step(sr, 2, dA, nullptr, nullptr, 0, nullptr, nullptr, bcol.as<int32_t>(),
                                bval.p, bpre, nb, n, scol.as<int32_t>(), sval.p, bnnz, nullptr, nullptr,
                                nullptr, 0, ctx->stream, ctx->sms);
  cb::launch_exclusive_scan(bnnz, nb, ypre, partial, ctx->stream);
  CB_LAUNCHED();
  mark(ctx, opt, 1);
  read_counters(ctx, counters, ypre + nb, 1);
  const int64_t total = ctx->host[cb::kCounters];
  y->nnz = total;
  ctx->stats.nnz = total;
  ctx->stats.kernels += 3;
  if (caller_buf && total > opt.out_capacity) {
    char msg[128];
    std::snprintf(msg, sizeof msg, "y needs %lld entries, capacity %lld", (long long)total,
                  (long long)opt.out_capacity);
    ctx->err = msg;
    throw Fail{CB_ERR_CAPACITY};
  }
  if (!caller_buf && total > 0) {
    CB_CUDA(dev_alloc(ctx, &y->idx, 4 * (size_t)total));
    CB_CUDA(dev_alloc(ctx, &y->val, vsz * (size_t)total));
  }
  cb::launch_spmspv_bucket_step(sr, 3, dA, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, bpre,
                                nb, n, scol.as<int32_t>(), sval.p, bnnz, ypre, y->idx, y->val, total,
                                ctx->stream, ctx->sms);
  CB_LAUNCHED();
  ctx->stats.kernels += 1;
  mark(ctx, opt, 2);
  mark(ctx, opt, 3);
  mark(ctx, opt, 4);
  mark(ctx, opt, 5);
  collect_times(ctx, opt, true);
}

int cb_spmspv(cb_ctx* ctx, cb_semiring sr, const cb_csr* A, const cb_spvec* x, cb_spvec* y,
              const cb_opts* opt_in) {
  if (!ctx) return CB_ERR_ARG;
  ctx->err.clear();
  ctx->stats = cb_stats{};
  ctx->stats.batches = 1;
  cb_opts opt;
  if (opt_in) opt = *opt_in;
  else cb_opts_default(&opt);
  const bool caller_buf = opt.out_capacity > 0;
  cb_spvec saved{};
  if (y) saved = *y;
  try {
    if (!A || !x || !y) fail(ctx, CB_ERR_ARG, "null argument");
    if (!public_semiring(sr)) fail(ctx, CB_ERR_SEMIRING, "unknown semiring");
    check_operand(ctx, A, "A");
    if (x->n != A->nrows) fail(ctx, CB_ERR_SHAPE, "x's length differs from A.nrows");
    if (x->nnz < 0 || (x->nnz > 0 && (!x->idx || !x->val))) fail(ctx, CB_ERR_ARG, "bad x");
    if (caller_buf && (!y->idx || !y->val)) fail(ctx, CB_ERR_ARG, "out_capacity > 0 needs y->idx and y->val");
    const int64_t n = A->ncols, nx = x->nnz, nw = (n + 31) / 32;
    const size_t vsz = value_size(sr);
    y->n = n;
    y->nnz = 0;
    if (!caller_buf) {
      y->idx = nullptr;
      y->val = nullptr;
    }
    if (opt.validate) {
      ensure(ctx, &ctx->ws, &ctx->ws_cap, align_up(sizeof(int64_t) * cb::kCounters));
      int64_t* counters = static_cast<int64_t*>(ctx->ws);
      CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
      cb::launch_validate(dev(A), A->nnz, 0, counters, ctx->stream, ctx->sms);
      CB_LAUNCHED();
      read_counters(ctx, counters, nullptr, 0);
      if (ctx->host[cb::kError]) fail(ctx, CB_ERR_INDEX, "A has invalid CSR index data");
    }
    if (n == 0 || nx == 0) return CB_OK;
    if (opt.flags & CB_FLAG_SPMSPV_BUCKET) {
      spmspv_bucket(ctx, (int)sr, A, x, y, opt, caller_buf);
      return CB_OK;
    }
    // the dense accumulator: (re)allocated for a wider A, re-initialised for another semiring
    const size_t avs = cb::spa_value_size((int)sr);
    if (ctx->spa_n < n) {
      CB_CUDA(cudaStreamSynchronize(ctx->stream));
      if (ctx->spa) cudaFree(ctx->spa);
      if (ctx->spa_bits) cudaFree(ctx->spa_bits);
      ctx->spa = nullptr;
      ctx->spa_bits = nullptr;
      ctx->spa_n = 0;
      ctx->spa_sr = 0;
      CB_CUDA(dev_alloc_sync(ctx, &ctx->spa, 8 * (size_t)n));
      CB_CUDA(dev_alloc_sync(ctx, &ctx->spa_bits, 4 * (size_t)nw));
      CB_CUDA(cudaMemsetAsync(ctx->spa_bits, 0, 4 * (size_t)nw, ctx->stream));
      ctx->spa_n = n;
    }
    const DevCSR dA = dev(A);
    if (ctx->spa_sr != (int)sr) {
      cb::launch_spmspv_step((int)sr, 0, dA, nullptr, nullptr, 0, nullptr, nullptr, ctx->spa, nullptr,
                             ctx->spa_n, nullptr, nullptr, nullptr, nullptr, 0, nullptr, ctx->stream,
                             ctx->sms);
      ctx->spa_sr = (int)sr;
      ctx->stats.kernels += 1;
    }
    (void)avs;
    const int64_t big = std::max(nx, nw);
    ensure(ctx, &ctx->ws, &ctx->ws_cap,
           align_up(sizeof(int64_t) * cb::kCounters) + 2 * align_up(8 * (size_t)(nx + 1)) +
               2 * align_up(8 * (size_t)(nw + 1)) + align_up(8 * (size_t)cb::scan_partials(big)));
    Carver cv{static_cast<char*>(ctx->ws)};
    int64_t* counters = cv.take<int64_t>(cb::kCounters);
    int64_t* chunks = cv.take<int64_t>(nx + 1);
    int64_t* cpre = cv.take<int64_t>(nx + 1);
    int64_t* wcnt = cv.take<int64_t>(nw + 1);
    int64_t* wpre = cv.take<int64_t>(nw + 1);
    int64_t* partial = cv.take<int64_t>(cb::scan_partials(big));
    CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
    mark(ctx, opt, 0);
    cb::launch_spmspv_step((int)sr, 1, dA, x->idx, x->val, nx, chunks, nullptr, nullptr, nullptr, n,
                           nullptr, nullptr, nullptr, nullptr, 0, counters + cb::kError, ctx->stream,
                           ctx->sms);
    cb::launch_exclusive_scan(chunks, nx, cpre, partial, ctx->stream);
    cb::launch_spmspv_step((int)sr, 2, dA, x->idx, x->val, nx, nullptr, cpre, ctx->spa, ctx->spa_bits, n,
                           nullptr, nullptr, nullptr, nullptr, 0, nullptr, ctx->stream, ctx->sms);
    cb::launch_spmspv_step((int)sr, 3, dA, nullptr, nullptr, 0, nullptr, nullptr, nullptr, ctx->spa_bits,
                           n, wcnt, nullptr, nullptr, nullptr, 0, nullptr, ctx->stream, ctx->sms);
    cb::launch_exclusive_scan(wcnt, nw, wpre, partial, ctx->stream);
    CB_LAUNCHED();
    ctx->stats.kernels += 6;
    mark(ctx, opt, 1);
    read_counters(ctx, counters, wpre + nw, 1);
    const int64_t total = ctx->host[cb::kCounters];
    const bool bad_x = ctx->host[cb::kError] != 0;
    int64_t cap = caller_buf ? opt.out_capacity : total;
    if (!caller_buf && total > 0) {
      CB_CUDA(dev_alloc(ctx, &y->idx, 4 * (size_t)total));
      CB_CUDA(dev_alloc(ctx, &y->val, vsz * (size_t)total));
    }
    // compaction always runs: it also resets the accumulator for the next call
    cb::launch_spmspv_step((int)sr, 4, dA, nullptr, nullptr, 0, nullptr, nullptr, ctx->spa,
                           ctx->spa_bits, n, nullptr, wpre, y->idx, y->val, std::min(cap, total),
                           nullptr, ctx->stream, ctx->sms);
    CB_LAUNCHED();
    ctx->stats.kernels += 1;
    mark(ctx, opt, 2);
    mark(ctx, opt, 3);
    mark(ctx, opt, 4);
    mark(ctx, opt, 5);
    y->nnz = total;
    ctx->stats.nnz = total;
    if (bad_x) fail(ctx, CB_ERR_INDEX, "an index of x is outside [0, A.nrows)");
    if (caller_buf && total > opt.out_capacity) {
      char msg[128];
      std::snprintf(msg, sizeof msg, "y needs %lld entries, capacity %lld", (long long)total,
                    (long long)opt.out_capacity);
      ctx->err = msg;
      throw Fail{CB_ERR_CAPACITY};
    }
    collect_times(ctx, opt, true);
    return CB_OK;
  } catch (const Fail& f) {
    if (!caller_buf && y) {
      if (y->idx && y->idx != saved.idx) cudaFreeAsync(y->idx, ctx->stream);
      if (y->val && y->val != saved.val) cudaFreeAsync(y->val, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      const int64_t need = y->nnz;
      std::memset(y, 0, sizeof *y);
      y->nnz = need;
    }
    return f.code;
  }
}

int cb_spvec_free_async(cb_ctx* ctx, cb_spvec* y) {
  if (!ctx || !y) return CB_ERR_ARG;
  int rc = CB_OK;
  for (void* p : {(void*)y->idx, y->val})
    if (p && cudaFreeAsync(p, ctx->stream) != cudaSuccess) rc = CB_ERR_CUDA;
  std::memset(y, 0, sizeof *y);
  return rc;
}

int cb_merge(cb_ctx* ctx, cb_semiring sr, int k, const cb_csr* parts, cb_csr* C, const cb_opts* opt_in) {
  if (!ctx) return CB_ERR_ARG;
  ctx->err.clear();
  ctx->stats = cb_stats{};
  ctx->stats.batches = 1;
  cb_opts opt;
  if (opt_in) opt = *opt_in;
  else cb_opts_default(&opt);
  const bool caller_buf = opt.out_capacity > 0;
  cb_csr saved{};
  if (C) saved = *C;
  try {
    if (!parts || !C || k < 1) fail(ctx, CB_ERR_ARG, "cb_merge needs k >= 1 parts and an output");
    if (!public_semiring(sr)) fail(ctx, CB_ERR_SEMIRING, "unknown semiring");
    if (opt.budget_bytes > 0 || opt.sizing != CB_SIZING_EXACT)
      fail(ctx, CB_ERR_ARG, "cb_merge takes exact sizing and no budget");
    if (caller_buf && (!C->row_ptr || !C->col || !C->val))
      fail(ctx, CB_ERR_ARG, "out_capacity > 0 needs C->row_ptr, C->col and C->val");
    const int64_t m = parts[0].nrows, n = parts[0].ncols;
    int64_t total = 0;
    for (int l = 0; l < k; ++l) {
      check_operand(ctx, &parts[l], "part");
      if (parts[l].nrows != m || parts[l].ncols != n) fail(ctx, CB_ERR_SHAPE, "parts differ in shape");
      total += parts[l].nnz;
    }
    if (opt.validate) {
      ensure(ctx, &ctx->ws, &ctx->ws_cap, align_up(sizeof(int64_t) * cb::kCounters));
      int64_t* counters = static_cast<int64_t*>(ctx->ws);
      CB_CUDA(cudaMemsetAsync(counters, 0, sizeof(int64_t) * cb::kCounters, ctx->stream));
      for (int l = 0; l < k; ++l) cb::launch_validate(dev(&parts[l]), parts[l].nnz, 0, counters, ctx->stream, ctx->sms);
      CB_LAUNCHED();
      read_counters(ctx, counters, nullptr, 0);
      if (ctx->host[cb::kError]) fail(ctx, CB_ERR_INDEX, "a part has invalid CSR index data");
    }
    if ((int64_t)k * m >= INT32_MAX) fail(ctx, CB_ERR_INDEX, "k * nrows beyond int32 indices");
    const size_t vsz = value_size(sr);
    // the selector product's semiring: the semiring itself, whose B and C
    // types agree, or for CB_MAXW_LABEL its merge form (B = C = cb_wlabel)
    const int msr = sr == CB_MAXW_LABEL ? kMergeMaxwLabel : (int)sr;
    const size_t asz = a_value_size(msr);
    // B = [P_0; ...; P_{k-1}] stacked by rows; A = the selector (k entries per row)
    DevBuf sBrp(ctx), sBcol(ctx), sBval(ctx), hparts(ctx), aRp(ctx), aCol(ctx), aVal(ctx);
    sBrp.alloc(8 * (size_t)(k * m + 1));
    sBcol.alloc(4 * (size_t)total);
    sBval.alloc(vsz * (size_t)total);
    const size_t psz = cb::stack_part_size();
    hparts.alloc((size_t)k * psz);
    std::vector<unsigned char> hp((size_t)k * psz);
    int64_t off = 0;
    for (int l = 0; l < k; ++l) {
      cb::fill_stack_part(&hp[(size_t)l * psz], parts[l].row_ptr, parts[l].col, parts[l].val, m, l * m, off,
                          0, (int32_t)n);
      off += parts[l].nnz;
    }
    CB_CUDA(cudaMemcpyAsync(hparts.p, hp.data(), hp.size(), cudaMemcpyHostToDevice, ctx->stream));
    if (m > 0) cb::launch_stack(hparts.p, k, (int)vsz, sBrp.as<int64_t>(), sBcol.as<int32_t>(), sBval.p,
                                nullptr, ctx->stream, ctx->sms);
    aRp.alloc(8 * (size_t)(m + 1));
    aCol.alloc(4 * (size_t)(k * m));
    aVal.alloc(asz * (size_t)(k * m));
    uint64_t one = 1;  // multiplicative identity: 1, 1.0, 0 (min,+), true
    if (sr == CB_PLUS_TIMES_F64) {
      const double d = 1.0;
      std::memcpy(&one, &d, sizeof d);
    } else if (sr == CB_MIN_PLUS_U32) {
      one = 0;
    }
    cb::launch_merge_selector(m, k, (int)asz, one, aRp.as<int64_t>(), aCol.as<int32_t>(), aVal.p,
                              ctx->stream, ctx->sms);
    if (m == 0) CB_CUDA(cudaMemsetAsync(aRp.p, 0, sizeof(int64_t), ctx->stream));
    CB_LAUNCHED();
    const cb_csr sel{m, k * m, k * m, aRp.as<int64_t>(), aCol.as<int32_t>(), aVal.p};
    const DevCSR dB{k * m, n, sBrp.as<int64_t>(), sBcol.as<int32_t>(), sBval.p};
    opt.validate = 0;
    spgemm_plain(ctx, msr, &sel, dB, n, C, opt);
    ctx->stats.kernels += 2;
    check_words(ctx);
    return CB_OK;
  } catch (const Fail& f) {
    if (!caller_buf && C) {
      if (C->row_ptr && C->row_ptr != saved.row_ptr) cudaFreeAsync(C->row_ptr, ctx->stream);
      if (C->col && C->col != saved.col) cudaFreeAsync(C->col, ctx->stream);
      if (C->val && C->val != saved.val) cudaFreeAsync(C->val, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      std::memset(C, 0, sizeof *C);
    }
    return f.code;
  }
}

int cb_spgemm_batched(cb_ctx* ctx, int count, const cb_semiring* sr, const cb_csr* A,
                      const cb_csr* B, const cb_opts* opt_in) {
  if (!ctx) return CB_ERR_ARG;
  ctx->err.clear();
  ctx->stats = cb_stats{};
  cb_opts opt;
  if (opt_in) opt = *opt_in;
  else cb_opts_default(&opt);
  int wave = 0, kernels = 0;
  int64_t nnz = 0, flops = 0;
  try {
    if (count < 0 || (count > 0 && (!sr || !A || !B))) fail(ctx, CB_ERR_ARG, "bad batch arguments");
    if (!opt.on_batch) fail(ctx, CB_ERR_ARG, "batched SpGEMM needs on_batch");
    if (opt.sizing == CB_SIZING_LEARNED && !opt.mlp) fail(ctx, CB_ERR_ARG, "learned sizing needs opt->mlp");
    if (opt.sizing != CB_SIZING_EXACT && opt.sizing != CB_SIZING_LEARNED)
      fail(ctx, CB_ERR_ARG, "batched SpGEMM supports exact and learned sizing");
    for (int i = 0; i < count; ++i) {
      if (!public_semiring(sr[i])) fail(ctx, CB_ERR_SEMIRING, "unknown semiring");
      check_operand(ctx, &A[i], "A[i]");
      check_operand(ctx, &B[i], "B[i]");
      if (A[i].ncols != B[i].nrows) fail(ctx, CB_ERR_SHAPE, "A[i].ncols != B[i].nrows");
    }
    if (opt.validate)
      for (int i = 0; i < count; ++i) run_validation(ctx, &A[i], &B[i]);
    for (int g0 = 0; g0 < count;) {
      int g1 = g0 + 1;
      while (g1 < count && sr[g1] == sr[g0]) ++g1;
      batched_group(ctx, (int)sr[g0], A + g0, B + g0, g1 - g0, g0, opt, wave, kernels, nnz, flops);
      g0 = g1;
    }
    check_words(ctx);
  } catch (const Fail& f) {
    if (f.code != -1) return f.code;  // -1: the consumer stopped early
  }
  ctx->stats.batches = wave;
  ctx->stats.kernels = kernels;
  ctx->stats.nnz = nnz;
  ctx->stats.flops = flops;
  return CB_OK;
}

int cb_ctx_set_tune(cb_ctx* ctx, cb_tune* t) {
  if (!ctx || !t) return CB_ERR_ARG;
  auto clamp = [](int v, int lo, int hi) { return v < lo ? lo : v > hi ? hi : v; };
  cb::Tune u;
  u.sym_hash_max = clamp(t->sym_hash_max, cb::kSymSmallMax, cb::kSymLargeMax);
  u.num_hash_max = clamp(t->num_hash_max, u.sym_hash_max, 4096);
  u.learn_max = clamp(t->learn_max, 0, 8192);
  // compression-ratio bounds: 0 <= cf_esc <= 2 (a row's products must fit
  // its table), cf_prereduce >= 1 (NaN or above 1e30: off)
  const float esc = t->cf_esc, pre = t->cf_prereduce;
  u.cf_esc = !(esc > 0.0f) ? 0.0f : esc > 2.0f ? 2.0f : esc;
  u.cf_pre = !(pre >= 1.0f) ? (pre != pre ? 1e30f : 1.0f) : pre > 1e30f ? 1e30f : pre;
  ctx->tune = u;
  t->sym_hash_max = u.sym_hash_max;
  t->num_hash_max = u.num_hash_max;
  t->learn_max = u.learn_max;
  t->cf_esc = u.cf_esc;
  t->cf_prereduce = u.cf_pre;
  return CB_OK;
}

int cb_ctx_get_tune(const cb_ctx* ctx, cb_tune* t) {
  if (!ctx || !t) return CB_ERR_ARG;
  t->sym_hash_max = ctx->tune.sym_hash_max;
  t->num_hash_max = ctx->tune.num_hash_max;
  t->learn_max = ctx->tune.learn_max;
  t->cf_esc = ctx->tune.cf_esc;
  t->cf_prereduce = ctx->tune.cf_pre;
  return CB_OK;
}

int cb_autotune(cb_ctx* ctx, cb_semiring sr, const cb_csr* A, const cb_csr* B, const cb_opts* opt_in,
                cb_tune* best, float* best_ms) {
  if (!ctx || !best) return CB_ERR_ARG;
  ctx->err.clear();
  cb_opts opt;
  if (opt_in) opt = *opt_in;
  else cb_opts_default(&opt);
  opt.budget_bytes = 0;
  opt.validate = 0;
  opt.flags = CB_FLAG_NO_FUSED;  // the bounds only steer the two-phase path
  const cb::Tune saved = ctx->tune;
  cb_csr C{};
  try {
    if (!A || !B) fail(ctx, CB_ERR_ARG, "null matrix argument");
    if (!public_semiring(sr)) fail(ctx, CB_ERR_SEMIRING, "unknown semiring");
    check_operand(ctx, A, "A");
    check_operand(ctx, B, "B");
    if (A->ncols != B->nrows) fail(ctx, CB_ERR_SHAPE, "A.ncols != B.nrows");
    if (opt.sizing == CB_SIZING_LEARNED && !opt.mlp) fail(ctx, CB_ERR_ARG, "learned sizing needs opt->mlp");
    run_validation(ctx, A, B);
    // output buffers sized once by an exact run
    spgemm_plain(ctx, (int)sr, A, dev(B), B->ncols, &C, opt);
    CB_CUDA(cudaStreamSynchronize(ctx->stream));
    opt.out_capacity = C.nnz > 0 ? C.nnz : 1;
    if (C.nnz == 0) {
      CB_CUDA(dev_alloc(ctx, &C.col, 4));
      CB_CUDA(dev_alloc(ctx, &C.val, 8));
    }
    const int big = cb::num_large_max((int)sr);
    const int syms[] = {512, 1024, 2048, 4096};
    const int nums[] = {512, 1024, 2048, 4096};
    const int learns[] = {64, 512, 2048};
    cudaEvent_t e0, e1;
    CB_CUDA(cudaEventCreate(&e0));
    CB_CUDA(cudaEventCreate(&e1));
    float best_t = 1e30f;
    cb::Tune best_u = saved;
    auto trial = [&](const cb::Tune& u) {
      ctx->tune = u;
      cb_csr Cc{0, 0, 0, C.row_ptr, C.col, C.val};
      if (opt.sizing == CB_SIZING_EXACT) spgemm_plain(ctx, (int)sr, A, dev(B), B->ncols, &Cc, opt);
      else spgemm_learned(ctx, (int)sr, A, dev(B), B->ncols, &Cc, opt);  // warm-up
      CB_CUDA(cudaEventRecord(e0, ctx->stream));
      if (opt.sizing == CB_SIZING_EXACT) spgemm_plain(ctx, (int)sr, A, dev(B), B->ncols, &Cc, opt);
      else spgemm_learned(ctx, (int)sr, A, dev(B), B->ncols, &Cc, opt);
      CB_CUDA(cudaEventRecord(e1, ctx->stream));
      CB_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      CB_CUDA(cudaEventElapsedTime(&t, e0, e1));
      if (t < best_t) {
        best_t = t;
        best_u = u;
      }
    };
    for (int sh : syms)
      for (int nh : nums) {
        if (nh < sh || nh > big) continue;
        cb::Tune u = saved;
        u.sym_hash_max = sh;
        u.num_hash_max = nh;
        if (opt.sizing == CB_SIZING_EXACT) {
          trial(u);
        } else {
          for (int lm : learns) {
            u.learn_max = lm;
            trial(u);
          }
        }
      }
    // then the compression-ratio bounds of the hash tiers, under the best tier bounds
    const float escs[] = {0.0f, 1.25f, 2.0f};
    const float pres[] = {2.0f, 4.0f, 16.0f, 1e30f};
    const cb::Tune tiers = best_u;
    for (float ce : escs)
      for (float cp : pres) {
        cb::Tune u = tiers;
        u.cf_esc = ce;
        u.cf_pre = cp;
        if (ce == tiers.cf_esc && cp == tiers.cf_pre) continue;  // timed above
        trial(u);
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tune = best_u;
    best->sym_hash_max = best_u.sym_hash_max;
    best->num_hash_max = best_u.num_hash_max;
    best->learn_max = best_u.learn_max;
    best->cf_esc = best_u.cf_esc;
    best->cf_prereduce = best_u.cf_pre;
    if (best_ms) *best_ms = best_t;
    cb_csr_free_async(ctx, &C);
    return CB_OK;
  } catch (const Fail& f) {
    ctx->tune = saved;
    cb_csr_free_async(ctx, &C);
    return f.code;
  }
}

int cb_autotune_cached(cb_ctx* ctx, cb_semiring sr, const cb_csr* A, const cb_csr* B,
                       const cb_opts* opt, const char* cache_path, cb_tune* best, float* best_ms,
                       int* hit) {
  if (!ctx || !best || !cache_path || !hit) return CB_ERR_ARG;
  *hit = 0;
  ctx->err.clear();
  if (!A || !B) {
    ctx->err = "null matrix argument";
    return CB_ERR_ARG;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess) {
    ctx->err = "cudaGetDeviceProperties failed";
    return CB_ERR_CUDA;
  }
  char key[512];
  const int32_t sizing = opt ? opt->sizing : CB_SIZING_EXACT;
  if (cb_tune_key(prop.name, sr, sizing, A->nrows, A->nnz, B->nnz, key, sizeof key) != CB_OK) {
    ctx->err = "tune cache key too long";
    return CB_ERR_ARG;
  }
  cb_tune t{};
  float ms = 0.f;
  int found = 0;
  if (cb_tune_cache_get(cache_path, key, &t, &ms, &found) != CB_OK) {
    ctx->err = std::string("tune cache unreadable or not a cb tune cache: ") + cache_path;
    return CB_ERR_ARG;
  }
  if (found) {
    cb_ctx_set_tune(ctx, &t);  // clamps into range
    *best = t;
    if (best_ms) *best_ms = ms;
    *hit = 1;
    return CB_OK;
  }
  float tms = 0.f;
  const int rc = cb_autotune(ctx, sr, A, B, opt, best, &tms);
  if (rc != CB_OK) return rc;
  if (best_ms) *best_ms = tms;
  if (cb_tune_cache_put(cache_path, key, best, tms) != CB_OK) {
    ctx->err = std::string("tune cache not writable: ") + cache_path;
    return CB_ERR_ARG;
  }
  return CB_OK;
}

int cb_ctx_set_fault(cb_ctx* ctx, int kind, int64_t arg, int64_t arg2) {
  if (!ctx) return CB_ERR_ARG;
  switch (kind) {
    case CB_FAULT_ALLOC:
      if (arg < 0) return CB_ERR_ARG;
      ctx->fault_alloc = arg;
      ctx->allocs_seen = 0;
      return CB_OK;
    case CB_FAULT_SHORT_ROW:
      ctx->fault_short_row = arg < 0 ? -1 : arg;
      return CB_OK;
    case CB_FAULT_SILENT_TILE:
      if (arg < 0) {
        ctx->fused_silent = -1;
        ctx->fused_spin = cb::kFusedSpinDefault;
        return CB_OK;
      }
      if (arg2 < 1 || arg2 > (int64_t)cb::kFusedSpinDefault) return CB_ERR_ARG;
      ctx->fused_silent = arg;
      ctx->fused_spin = (unsigned)arg2;
      return CB_OK;
  }
  return CB_ERR_ARG;
}

int cb_last_stats(const cb_ctx* ctx, cb_stats* out) {
  if (!ctx || !out) return CB_ERR_ARG;
  *out = ctx->stats;
  return CB_OK;
}

}  // extern "C"
