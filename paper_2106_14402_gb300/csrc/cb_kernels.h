// Host-side launch wrappers for the SpGEMM kernels (no templates cross this
// header, so the C ABI layer compiles without the device code).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

struct cb_mlp;

namespace cb {

// Tier bounds chosen at run time (autotuned): rows with u = min(flops, ncols)
// <= sym_hash_max are counted in hash tables (else bitmaps); rows with
// nnz <= num_hash_max are computed in hash tables (else rank windows;
// num_hash_max >= sym_hash_max); with learned sizing, rows whose capacity is
// <= learn_max skip the symbolic phase.
struct Tune {
  int sym_hash_max = 512;
  int num_hash_max = 512;
  int learn_max = 512;
  // hash-tier rows by compression ratio cf = flops / nnz (k_num_hash):
  // expand-sort-compress at cf <= cf_esc, warp pre-reduction at cf >= cf_pre
  float cf_esc = 1.25f;
  float cf_pre = 4.0f;
};

// The compression-ratio bounds a numeric launch uses (from Tune).
struct CfBounds {
  float esc = 0.0f;
  float pre = 1e30f;
};

struct Window;

// A CSR operand as the kernels see it.  For B it may be a column window:
// only columns in [col_lo, col_lo + ncols) belong to the view.  Row k spans
// [rp[k], rpe[k]) (rpe == nullptr: rp[k + 1]).  With filter == 0 every entry
// of a row lies inside the window (slab offsets); with filter != 0 rows are
// whole and entries outside the window are skipped.
struct DevCSR {
  int64_t nrows, ncols;
  const int64_t* rp;
  const int32_t* col;
  const void* val;
  const int64_t* rpe = nullptr;
  int64_t col_lo = 0;
  int filter = 0;
  // A only: per-row output width (columns of row i lie in [0, rcols[i]));
  // nullptr = the width of B's view
  const int32_t* rcols = nullptr;
};

// Counters block in device memory (int64 each).
enum Counter {
  kCntSym = 0,          // [5] rows per symbolic tier
  kCurSym = 5,          // [5] scatter cursors
  kCntNum = 10,         // [5] rows per numeric tier
  kCurNum = 15,         // [5]
  kTotalFlops = 20,
  kUnits = 21,          // rank windows appended by the symbolic phase
  kError = 22,          // validation / overflow error word
  kErrDetail = 23,
  kUnsorted = 24,       // > 0 when some row of B is not non-decreasing
  kMaxFlops = 25,       // largest flops_i (k_classify_sym)
  kMaxArow = 26,        // longest row of A (k_classify_sym)
  kCounters = 32
};

// Validation of one CSR operand: row_ptr[0] == 0, non-decreasing,
// row_ptr[n] == nnz, 0 <= col < ncols.  Sets counters[kError] to a nonzero
// code on failure (1 = row_ptr, 2 = column), kErrDetail to an offending index.
void launch_validate(const DevCSR& M, int64_t nnz, int code_base, int64_t* counters,
                     cudaStream_t s, int sms);

// K1: flops_i, maxB_i and the symbolic tier histogram; total flops.
void launch_classify_sym(const DevCSR& A, const DevCSR& B, int64_t* flops, int32_t* maxb,
                         int64_t* counters, cudaStream_t s, int sms,
                         const uint8_t* skip = nullptr, int64_t sym_hash_max = 512);
// K2: rows into per-tier segments of perm; heavy rows also get nnz[i] = 0.
void launch_scatter_sym(int64_t m, int64_t ncols, const int64_t* flops, int32_t* perm,
                        int64_t* nnz, int64_t* counters, cudaStream_t s, int sms,
                        const uint8_t* skip = nullptr, const int64_t* preset = nullptr,
                        int64_t sym_hash_max = 512, const int32_t* rcols = nullptr);

// K4: out[0] = 0, out[i+1] = out[i] + in[i]; partial needs scan_partials(n) int64.
// Entries per scan tile (one partial sum per tile); the allocation-free
// variant sizes its static scratch from it.
constexpr int64_t kScanTileItems = 4096;
// Largest tile count one scan launch takes (the grid's x limit).
constexpr int64_t kScanMaxTiles = 2147483647;
int64_t scan_partials(int64_t n);
// Returns the error of its own launches (cudaErrorInvalidValue when n needs
// more than kScanMaxTiles tiles), not an error left pending by earlier calls.
cudaError_t launch_exclusive_scan(const int64_t* in, int64_t n, int64_t* out, int64_t* partial,
                           cudaStream_t s);

// out[j] = prefix[idx[j]] for j < n.
void launch_gather(const int64_t* prefix, const int64_t* idx, int64_t n, int64_t* out,
                   cudaStream_t s);

// Column-batch slab offsets: pos[j * B.nrows + k] = first entry of B row k
// with column >= bnd[j] (device int64 bnd[nb1]); B's rows must be sorted.
void launch_slabs(const DevCSR& B, const int64_t* bnd, int nb1, int64_t* pos, cudaStream_t s,
                  int sms);

// Numeric binning by exact row size.
void launch_classify_num(int sr, int64_t m, const int64_t* nnz, int32_t* perm,
                         int64_t* counters, cudaStream_t s, int sms,
                         const uint8_t* skip = nullptr, int64_t num_hash_max = 512);

// Learned sizing (rows whose capacity fits a hash table skip the symbolic
// phase): capacities + routing, their tiers, the one-pass numeric into
// staging, and the copy from staging into C.
void launch_learn_caps(int64_t m, const int64_t* pred, const int64_t* flops, int64_t ncols,
                       float margin, int64_t hash_max, int64_t* cap, uint8_t* learned,
                       cudaStream_t s, int sms, const int32_t* rcols = nullptr);
void launch_learned_tiers(int64_t m, const int64_t* cap, int64_t hash_max, int32_t* perm,
                          int64_t* counters, cudaStream_t s, int sms);
int learn_hash_max(int sr);
void launch_learned_numeric(int sr, const DevCSR& A, const DevCSR& B, const int32_t* perm,
                            const int64_t* seg_begin, const int64_t* seg_count,
                            const int64_t* flops, const int64_t* cap, const int64_t* stage_rp,
                            int32_t* scol, void* sval, uint8_t* learned, int64_t* cnt,
                            int64_t* overflows, cudaStream_t s, int sms, int* launches);
void launch_compact_rows(int vsz, int64_t m, const uint8_t* learned, const int64_t* stage_rp,
                         const int64_t* cnt, const int32_t* scol, const void* sval,
                         const int64_t* Crp, int32_t* Ccol, void* Cval, cudaStream_t s, int sms);

// K3: symbolic phase, all tiers.  perm holds the tier segments in order;
// seg_begin[t] / seg_count[t] are host copies of the tier layout.  Heavy
// rows (tier 4) write span_counts[h * spans + span] and, when wins is
// non-null, append their rank windows (cut every `wcut` entries) to wins
// (capacity win_cap; counters[kUnits] counts them).
// (span_wins[h * spans + span] = {first window, window count}; hbits, when
// non-null, receives each heavy row's bitmap: kSpanWords words per (row, span).)
void launch_symbolic(const DevCSR& A, const DevCSR& B, const int32_t* perm,
                     const int64_t* seg_begin, const int64_t* seg_count, const int64_t* flops,
                     int64_t* nnz, int32_t* span_counts, int2* span_wins, int wcut,
                     Window* wins, int64_t win_cap, unsigned* hbits, int b_sorted,
                     int64_t* counters, cudaStream_t s, int sms, int* launches);
// Sets counters[kUnsorted] > 0 if some row of B decreases in column.
void launch_check_sorted(const DevCSR& B, int64_t* counters, cudaStream_t s, int sms);

// K5-K7: numeric phase over the numeric tier segments + rank windows,
// writing sorted rows of C at Crp.
int num_window_cut(int sr);
int num_large_max(int sr);
void launch_numeric(int sr, const DevCSR& A, const DevCSR& B, const int32_t* perm,
                    const int64_t* seg_begin, const int64_t* seg_count, const int64_t* flops,
                    const int64_t* nnz, const int32_t* heavy_rows, const Window* wins,
                    int64_t n_wins, const int32_t* span_counts, int64_t spans,
                    const unsigned* hbits, int b_sorted, const int64_t* Crp, int32_t* Ccol,
                    void* Cval, int64_t* err, cudaStream_t s, int sms, int* launches,
                    int64_t num_hash_max = 512, void* racc = nullptr, CfBounds cf = {});

// Batched products (cb_batched.cu): stack parts into one CSR.
size_t stack_part_size();
void fill_stack_part(void* dst, const int64_t* rp, const int32_t* col, const void* val, int64_t nrows,
                     int64_t row_off, int64_t nnz_off, int32_t col_add, int32_t width);
// rcols_out (optional): every stacked row gets its part's width
// Selector matrix of the k-way merge (m rows, k entries each at columns
// l*m + i, values = one_bits of the value size vsz).
void launch_merge_selector(int64_t m, int k, int vsz, uint64_t one_bits, int64_t* rp, int32_t* col,
                           void* val, cudaStream_t s, int sms);
void launch_stack(const void* parts_dev, int nparts, int vsz, int64_t* rp_out, int32_t* col_out,
                  void* val_out, int32_t* rcols_out, cudaStream_t s, int sms);
// Digests of the nprod products of a wave (cb_opts.digests; definition in
// cb_batched.cu): the wave's stacked C (m rows) starts at stacked row
// row_base; product p of the wave holds stacked rows [prow[p], prow[p+1]).
// rdig / rsum: scratch of m entries each; out: 2 words per product.
void launch_digest(int vsz, bool f64, const int64_t* rp, const int32_t* col, const void* val, int64_t m,
                   const int64_t* prow, int nprod, int64_t row_base, uint64_t* rdig, double* rsum,
                   uint64_t* out, cudaStream_t s, int sms);

// Learned sizer (k_mlp.cu).
const void* mlp_bf16(const cb_mlp* m);
const float* mlp_master(const cb_mlp* m);
const float* mlp_norm(const cb_mlp* m);
void launch_row_features(const DevCSR& A, const int64_t* flops, const int32_t* maxb, int64_t ncols,
                         float* feat, cudaStream_t s, int sms);
void launch_mlp_predict(const void* wb, const float* master, const float* norm, const float* feat,
                        int64_t m, int64_t ncols, float* z, int64_t* pred, cudaStream_t s, int sms);

// One-launch SpGEMM for products whose rows are all small (k_fused.cu):
// every row of A holds at most `lanes` entries and every output row at most
// 8 * lanes products (lanes = 8, 16 or 32), columns below fused_max_cols.
// tstat holds at least fused_tiles(lanes, A.nrows) words and sync 16 words,
// all zero when first used; they must not be shared by launches in flight.
// sync: [0] launch epoch, [1] finished CTAs, [2..3] nnz(C) of the last
// launch (int64), [6..7] its product count, [8..9] the product accumulator;
// words 4 and 5 are free for the caller (the context keeps a status there).
// SpMSpV steps (k_spmspv.cu): 0 SPA init over n, 1 chunk counts of the x
// entries (bad indices set *err), 2 push into the SPA (cpre = scanned chunk
// counts, cpre[nx] = total), 3 popcounts of the touched bitmap, 4 compaction
// into y (wpre = scanned popcounts; nothing past cap) resetting SPA and bitmap.
// dst = max(dst, src) on the device (error words kept across launch sequences).
void launch_merge_error(const int64_t* src, int64_t* dst, cudaStream_t s);
size_t spa_value_size(int sr);
// Bucket (propagation-blocking) SpMSpV steps (k_spmspv.cu): 0 products per
// bucket into cur (zeroed), 1 products appended at cur (preset to bpre),
// 2 per-bucket reduction into the staging area + bnnz, 3 copy to y at ypre.
int64_t spmspv_buckets(int64_t n);
// Per-CTA counted form of steps 0 and 1 (CTAs = spmspv_priv_ctas(nb, sms), 0
// when the buckets do not fit shared memory): pass 0 counts into ccnt[b][cta],
// pass 2 scans ccnt over CTAs (bucket totals into tot), pass 1 scatters.
int spmspv_priv_ctas(int64_t nb, int sms);
void launch_spmspv_bucket_priv(int sr, int pass, const DevCSR& A, const int32_t* x_idx,
                               const void* x_val, int64_t nx, const int64_t* cpre, int64_t nb,
                               int64_t* ccnt, const int64_t* bpre, int64_t* tot, int32_t* bcol,
                               void* bval, cudaStream_t s, int sms);
void launch_spmspv_bucket_step(int sr, int step, const DevCSR& A, const int32_t* x_idx,
                               const void* x_val, int64_t nx, const int64_t* cpre,
                               unsigned long long* cur, int32_t* bcol, void* bval, const int64_t* bpre,
                               int64_t nb, int64_t n, int32_t* scol, void* sval, int64_t* bnnz,
                               const int64_t* ypre, int32_t* y_idx, void* y_val, int64_t cap,
                               cudaStream_t s, int sms);
void launch_spmspv_step(int sr, int step, const DevCSR& A, const int32_t* x_idx, const void* x_val,
                        int64_t nx, int64_t* chunks, const int64_t* cpre, void* spa,
                        unsigned* touched, int64_t n, int64_t* wcnt, const int64_t* wpre,
                        int32_t* y_idx, void* y_val, int64_t cap, int64_t* err, cudaStream_t s,
                        int sms);
// Symbolic and numeric passes whose tier sizes, heavy-row count, window
// count and B's sortedness are read on the device (counters from
// launch_check_sorted / launch_classify_sym / launch_classify_num): no host
// synchronisation, so the sequence can be captured into a CUDA graph.  The
// caller sizes span_counts / span_wins (rows x spans) and wins (win_cap, an
// upper bound) in advance; heavy-row bitmaps are rebuilt, not stored.
void prepare_symbolic_dev();
void prepare_dev_launchers(int sr);  // sets the shared-memory attributes of both (not capturable)
void launch_symbolic_dev(const DevCSR& A, const DevCSR& B, const int32_t* perm, int64_t* counters,
                         const int64_t* flops, int64_t* nnz, int32_t* span_counts, int2* span_wins,
                         int wcut, Window* wins, int64_t win_cap, cudaStream_t s, int sms);
void launch_numeric_dev(int sr, const DevCSR& A, const DevCSR& B, const int32_t* perm,
                        const int64_t* counters, const int64_t* flops, const int64_t* nnz,
                        const int64_t* Crp, int32_t* Ccol, void* Cval, int64_t* err, cudaStream_t s,
                        int sms, const int32_t* perm_sym, const Window* wins,
                        const int32_t* span_counts, int64_t spans, void* racc, int64_t num_hash_max,
                        CfBounds cf = {});
// Bytes of the global accumulator slices of the rank-window numeric kernel
// (semirings whose windows accumulate in L2; 0 otherwise).
size_t rank_scratch_bytes(int sr, int sms);
int64_t fused_tiles(int lanes, int64_t nrows);
int64_t fused_max_cols(int lanes);
// Each look-back wait polls an earlier tile at most spin_limit times
// (kFusedSpinDefault, about a second), then records CB_FUSED_STALLED and
// publishes anyway.  silent_tile >= 0 (fault injection) is a tile that
// never publishes its total.
constexpr unsigned kFusedSpinDefault = 1u << 20;
// One-pass rows from a device work queue (k_queue.cu): every row of A.B with
// at most kQueueAcc entries and an output width (B's columns, or A.rcols[i])
// of at most kQueueWidth; one CTA per row at a time, rows dequeued in order,
// offsets by look-back.  Shares the one-launch kernel's tile-status array
// (one word per row, tstat_cap >= m) and sync words (its queue counter at
// words 10..11; nnz(C) at 2..3 as there); status gets CB_FUSED_* bits.
constexpr int kQueueAcc = 4096;
constexpr int64_t kQueueWidth = 65536;
cudaError_t launch_queue_rows(int sr, const DevCSR& A, const DevCSR& B, int64_t m, int64_t* Crp,
                              int32_t* Ccol, void* Cval, int64_t cap, unsigned long long* tstat,
                              int64_t tstat_cap, unsigned* sync, int* status, cudaStream_t s, int sms,
                              unsigned spin_limit = kFusedSpinDefault, int64_t silent_row = -1);
cudaError_t launch_fused(int sr, int lanes, const DevCSR& A, const DevCSR& B, int64_t* Crp,
                         int32_t* Ccol, void* Cval, int64_t cap, unsigned long long* tstat,
                         int64_t tstat_cap, unsigned* sync, int* status, cudaStream_t s, int sms,
                         unsigned spin_limit = kFusedSpinDefault, int64_t silent_tile = -1);

// Fault injection: *nnz_row -= 1 when positive (one launch of one thread).
void launch_fault_shrink(int64_t* nnz_row, cudaStream_t s);

// Debug build (-DCB_CHECK): read and clear the bounds-check word of each
// kernel file on stream s (synchronises); returns the first failed check's
// code (0: none, -1: the read failed) and its index in *index.  Always 0 in
// the normal build.
int64_t check_take_numeric(cudaStream_t s, int64_t* index);
int64_t check_take_symbolic(cudaStream_t s, int64_t* index);
int64_t check_take_queue(cudaStream_t s, int64_t* index);
int64_t check_take_rows(cudaStream_t s, int64_t* index);
int64_t check_take_fused(cudaStream_t s, int64_t* index);

}  // namespace cb
