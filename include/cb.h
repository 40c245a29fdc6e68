/*
 * cb.h -- C ABI of the GB300 semiring SpGEMM library (libcb.so).
 *
 * Operation (paper Sec. 3.1, the SpGEMM notation; Sec. 4.1, multithreaded SpGEMM):
 *   C = A (+).(x) B  with A in S^{m x n}, B in S^{n x k}, C in S^{m x k},
 *   computed row by row with Gustavson's formulation: row i of C merges the
 *   rows of B selected by the stored entries of row i of A.  The pattern of C
 *   is structural: (i,j) is stored iff some stored A(i,p) meets some stored
 *   B(p,j); every such pair contributes one (x)-product, and products are
 *   (+)-combined (entries equal to zero or to the (+)-identity are kept).
 *   Sec. 4.1 splits the work into (1) a flops estimate and load balance,
 *   (2) a symbolic phase that sizes C, (3) a numeric phase with a hash
 *   accumulator; Sec. 7.2 forms C in column batches when it does not fit.
 *
 * Data layout (all matrices): CSR by rows.
 *   row_ptr  int64[nrows + 1], row_ptr[0] = 0, non-decreasing, row_ptr[nrows] = nnz
 *   col      int32[nnz], 0 <= col < ncols (ncols <= INT32_MAX)
 *   val      nnz values of the operand's type under the semiring (bool
 *            stored as uint8 0/1, any nonzero input byte counts as true).
 *            Semirings 1-5 use one type for A, B and C; the heterogeneous
 *            CB_MAXW_LABEL takes three (paper Sec. 1: two input types and
 *            one output type).
 * Inputs may have unsorted and duplicate columns within a row (duplicates
 * contribute separately).  Output rows always have strictly increasing
 * columns.  All cb_csr pointers are DEVICE pointers unless a function says
 * otherwise.
 *
 * Errors: every function returns an int status (CB_OK = 0).  Nothing throws
 * across the ABI, nothing aborts, no kernel traps.  On error the output
 * cb_csr is left zeroed and owns nothing; cb_last_error(ctx) gives a message.
 *
 * Streams: a cb_ctx is bound to one CUDA stream; all work is ordered on it.
 * Functions that must learn a size on the host (the total nnz of C, to
 * allocate it) synchronise that stream once; the functions marked "async"
 * never synchronise.
 */
#ifndef CB_H_
#define CB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Semirings and their value types. */
typedef enum {
  CB_PLUS_TIMES_I64 = 1, /* (+,x) over int64, wrapping two's complement          */
  CB_PLUS_TIMES_F64 = 2, /* (+,x) over IEEE fp64 (any summation order, FMA ok)   */
  CB_MIN_PLUS_U32 = 3,   /* (min,+) over uint32, + saturates at UINT32_MAX (inf) */
  CB_OR_AND_BOOL = 4,    /* (or,and) over bool stored as uint8                   */
  CB_SEL2ND_MIN_I32 = 5, /* (select2nd,min) over int32: (x)(a,b) = b, (+) = min  */
  CB_MAXW_LABEL = 6      /* heterogeneous: A float32, B int32, C cb_wlabel (below) */
} cb_semiring;

/* Output value of CB_MAXW_LABEL (8 bytes: w at offset 0, label at 4).
 * (x)(a, b) = {a, b} for an A weight a and a B label b; (+) keeps the pair
 * with the larger w in IEEE 754 totalOrder (-NaN < -inf < ... < -0 < +0 <
 * ... < +inf < +NaN), and of equal w the smaller label.  C(i,j) is thus the
 * label B(k,j) reached through the heaviest edge A(i,k), with that weight.
 * The order is exact (no arithmetic on w), so results are bit-exact. */
typedef struct {
  float w;
  int32_t label;
} cb_wlabel;

/* Status codes. */
enum {
  CB_OK = 0,
  CB_ERR_ARG = 1,       /* null pointer, negative size, bad option             */
  CB_ERR_SHAPE = 2,     /* A.ncols != B.nrows                                  */
  CB_ERR_SEMIRING = 3,  /* unknown semiring                                    */
  CB_ERR_INDEX = 4,     /* ncols > INT32_MAX, bad row_ptr, column out of range */
  CB_ERR_OOM = 5,       /* device allocation failed                            */
  CB_ERR_BUDGET = 6,    /* one output row (or batch unit) exceeds the budget   */
  CB_ERR_TIMEOUT = 7,   /* a bounded device-side wait expired                  */
  CB_ERR_CUDA = 8,      /* a CUDA runtime call failed                          */
  CB_ERR_CAPACITY = 9,  /* caller-provided output too small; C->nnz = needed   */
  CB_ERR_SCRATCH = 10   /* size beyond a fixed static scratch capacity         */
};

typedef struct {
  int64_t nrows, ncols, nnz;
  int64_t *row_ptr; /* device, int64[nrows + 1] */
  int32_t *col;     /* device, int32[nnz]        */
  void *val;        /* device, nnz values        */
} cb_csr;

typedef struct cb_ctx cb_ctx;

/* How C's per-row sizes are obtained before the numeric phase. */
typedef enum {
  CB_SIZING_EXACT = 0,       /* symbolic phase (paper Sec. 4.1, phase (2))      */
  CB_SIZING_LEARNED = 1,     /* MLP prediction, exact fallback on overflow      */
  CB_SIZING_UPPER_BOUND = 2  /* min(flops_i, ncols) per row, exact fallback     */
} cb_sizing;

/* Consumer of one column batch C[:, col_lo:col_hi) (paper Sec. 7.2: batched
 * SpGEMM forms the output in batches that the application consumes).  Cb is
 * valid only during the call (device pointers, columns are global indices).
 * Return nonzero to stop early (cb_spgemm_ex then returns CB_OK). */
typedef int (*cb_batch_fn)(int batch, int64_t col_lo, int64_t col_hi,
                           const cb_csr *Cb, void *user);

/* Learned sizer weights (see cb_mlp_* below). */
typedef struct cb_mlp cb_mlp;

typedef struct {
  int32_t sizing;       /* cb_sizing; default CB_SIZING_EXACT                        */
  int32_t validate;     /* nonzero (default): check A and B on the device first      */
  int64_t out_capacity; /* >0: C->row_ptr/col/val are caller buffers of this capacity */
  int64_t budget_bytes; /* >0: column-batched; each batch's C (row_ptr+col+val) fits  */
  cb_batch_fn on_batch; /* required when budget_bytes > 0                             */
  void *user;           /* passed to on_batch                                         */
  const cb_mlp *mlp;    /* required when sizing == CB_SIZING_LEARNED                   */
  float margin;         /* learned sizing: table capacity = pred * (1 + margin)       */
  int32_t flags;        /* CB_FLAG_* bits, default 0                                  */
  uint64_t *digests;    /* cb_spgemm_batched only, optional (default NULL): device
                           uint64[2 * count] receiving a digest of every C_i, written
                           before its wave's on_batch in every mode (see there)        */
  int64_t resume_col;   /* column-batched calls (budget_bytes > 0): form only the
                           columns [resume_col, B.ncols) (default 0; 0..B.ncols, else
                           CB_ERR_ARG).  To resume a stopped or failed call, pass the
                           col_lo of the first batch not consumed and resume_batch =
                           its index: with exact sizing the same arguments then give
                           the same batches from there on; with learned sizing the
                           remaining columns are cut afresh (paper Sec. 7.2: the
                           batches are independent)                                 */
  int32_t resume_batch; /* index on_batch receives for the first batch formed
                           (default 0, >= 0)                                         */
} cb_opts;

/* cb_opts.flags bits. */
enum {
  CB_FLAG_CHECK = 1,  /* synchronise at the end and fail (CB_ERR_CUDA) if a kernel's
                         internal consistency word is set (debug)                   */
  CB_FLAG_TIMING = 2, /* record CUDA events between the phases on ctx's stream and
                         report their durations in cb_stats (synchronises at the end) */
  CB_FLAG_LEARNED_ROWS = 4, /* batched modes with learned sizing: besides the batch
                         count, also size each batch's rows from predictions
                         (default: predictions set the batch count only and each
                         batch runs the exact two-phase path) */
  CB_FLAG_GRAPH = 16,  /* cb_spgemm_batched, exact sizing: cut waves by the flop bound
                         (row pointers + flops entries per product within the budget),
                         run each wave as a launch sequence without host synchronisation
                         (tier sizes, heavy-row and window counts kept on the device; C
                         sized by the wave's flop total) and capture all waves of a group
                         into one CUDA graph, launched once; on_batch then runs as a graph
                         host node, must not call CUDA, and its return value is ignored.
                         A group with a product whose flop bound alone exceeds the budget
                         runs as without the flag. */
  CB_FLAG_SYNC_FREE = 32, /* cb_spgemm_batched: the launch sequence of CB_FLAG_GRAPH
                         without the capture; on_batch runs on the calling thread after
                         each wave (and may use CUDA) */
  CB_FLAG_SPMSPV_BUCKET = 64, /* cb_spmspv: the bucket (propagation-blocking) form
                         instead of the dense accumulator (see cb_spmspv) */
  CB_FLAG_NO_FUSED = 8 /* exact sizing: always run the two-phase path.  By default
                         (1) when the mean row lengths of A and B fit the bounds of
                         cb_spgemm_fused (below), that one launch is tried first,
                         with no flop count (a library-allocated C then holds up to
                         8 x lanes entries per row); if a row exceeds the bounds the
                         call continues with the flop count; (2) a product whose rows
                         all meet those bounds is formed by that one launch after the
                         flop count, C sized by flops (an upper bound of nnz(C));
                         (3) otherwise, when every output row has at most 4096
                         products and at most 65536 columns (B's, or the stacked
                         product's own), one persistent launch forms the rows in
                         one pass each, taking them from a device work queue (also
                         per wave of cb_spgemm_batched in every mode) */
};

/* Fill *opt with defaults (exact sizing, validation on, library-allocated C). */
void cb_opts_default(cb_opts *opt);

/* sizeof of the ABI's structs as this library was compiled (for bindings
 * that lay them out by hand): which = 0 cb_csr, 1 cb_opts, 2 cb_tune,
 * 3 cb_stats, 4 cb_spvec, 5 cb_wlabel; -1 for any other value. */
int64_t cb_struct_size(int which);

/* Create a context bound to `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream) on the current device.  The context owns a reusable device
 * workspace.  Returns CB_OK or CB_ERR_CUDA / CB_ERR_OOM. */
int cb_ctx_create(cb_ctx **ctx, void *cuda_stream);
void cb_ctx_destroy(cb_ctx *ctx);
/* Rebind the context to another stream. */
int cb_ctx_set_stream(cb_ctx *ctx, void *cuda_stream);
const char *cb_last_error(const cb_ctx *ctx);
const char *cb_status_str(int status);

/* C = A (+).(x) B, synchronous convenience form: creates a temporary context
 * on the default stream, allocates C (free with cb_csr_free), validates the
 * inputs, and returns when C is complete. */
int cb_spgemm(cb_semiring sr, const cb_csr *A, const cb_csr *B, cb_csr *C);

/* C = A (+).(x) B on ctx's stream with options (NULL = defaults).
 *   - If opt->out_capacity > 0, C->row_ptr (nrows+1), C->col and C->val
 *     (out_capacity entries) are caller-provided device buffers; if nnz(C)
 *     exceeds out_capacity the call returns CB_ERR_CAPACITY with C->nnz set
 *     to the required size and nothing written to C->col/val.
 *   - Otherwise the library allocates C's arrays with stream-ordered
 *     allocation on ctx's stream; release them with cb_csr_free.
 *   - If opt->budget_bytes > 0, C is formed in column batches (Sec. 7.2):
 *     each batch is handed to opt->on_batch and released afterwards; *C
 *     receives only the shape and the total nnz.
 * The stream is synchronised once (to learn nnz(C)); on return the output is
 * complete only in stream order (synchronise before reading it from the host
 * through another stream). */
int cb_spgemm_ex(cb_ctx *ctx, cb_semiring sr, const cb_csr *A, const cb_csr *B,
                 cb_csr *C, const cb_opts *opt);

/* Batched SpGEMM: count independent products C_i = A_i (+).(x)_{sr[i]} B_i
 * (the paper's GPU path picks a library per call by flops and compression,
 * Sec. 5; here all products of a batch share one launch sequence).
 * Consecutive products with the same semiring form a group; a group is laid
 * out as one block-diagonal product (A_i stacked by rows with their columns
 * shifted to the stacked rows of B_i; B_i stacked by rows with their own
 * columns) and cut into waves of consecutive products whose output (row
 * pointers + columns + values) fits opt->budget_bytes (0 = one wave per
 * group).  Wave sizes come from exact symbolic counts or, with learned
 * sizing, from predicted sizes times (1 + margin); a wave whose exact output
 * still exceeds the budget returns CB_ERR_CAPACITY.  Each wave is handed to
 *   opt->on_batch(wave, first, end, &Cw, opt->user)
 * where Cw stacks C_first .. C_{end-1} by rows (Cw.row_ptr covers all their
 * rows, in order; columns are each product's own), valid only during the
 * call; a nonzero return stops the batch (CB_OK).  opt->on_batch is
 * required; inputs are device CSR as for cb_spgemm_ex; sizing may be exact
 * or learned.  The stacked rows of each group must fit int32 indices
 * (CB_ERR_INDEX otherwise).
 * Digests (opt->digests != NULL): outputs of batched calls are transient (in
 * graph mode on_batch cannot even read them), so the call can leave a
 * check of each product behind.  With sm(x) the splitmix64 output function
 * (x += 0x9E3779B97F4A7C15; x = (x ^ x>>30) * 0xBF58476D1CE4E5B9;
 * x = (x ^ x>>27) * 0x94D049BB133111EB; x ^ x>>31) and all arithmetic mod
 * 2^64, product i's words are
 *   digests[2i]   = sum over its rows r of sm(sm(2r) + len_r)
 *                 + sum over its entries (row r, position j in the row,
 *                   column c, value v) of sm(sm(sm(sm(2r+1) + j) + c) + bits(v)),
 *                   bits(v) = v's bytes zero-extended to 64 bits, and 0 for
 *                   CB_PLUS_TIMES_F64, whose first word covers the pattern only;
 *   digests[2i+1] = for CB_PLUS_TIMES_F64, the bits of the double
 *                   V = sum over entries of v * w(r, c), w(r, c) = 1 + 2^-53 *
 *                   (sm(sm(2r+1) ^ c) >> 11), summed with compensated
 *                   (Neumaier) summation in a fixed order, so that
 *                   |V - exact| <= 16 u sum |v w| (u = 2^-53); else 0.
 *   r counts the product's own rows from 0.  The digests cost one extra read
 *   of C and one 16-byte scratch word per row of the largest wave. */
int cb_spgemm_batched(cb_ctx *ctx, int count, const cb_semiring *sr, const cb_csr *A,
                      const cb_csr *B, const cb_opts *opt);

/* Release arrays that the library allocated for C; zeroes *C.  Waits for all
 * work on the device to finish first, so it is safe right after an
 * asynchronous cb_spgemm_ex. */
void cb_csr_free(cb_csr *C);
/* Stream-ordered release on ctx's stream: the arrays are freed after the work
 * already queued on that stream (e.g. the kernels that write C) completes.
 * The caller must not use C's arrays on other streams afterwards. */
int cb_csr_free_async(cb_ctx *ctx, cb_csr *C);

/* ---- individual steps of the path (device outputs, async) ---------------
 * cb_row_stats: paper Sec. 4.1, phase (1), and Table 1 (flops).  For each row
 *   i of A: flops[i] = sum over stored A(i,p) of nnz(B(p,:)) (int64[m]),
 *   maxb[i] = max of those B row lengths (int32[m], 0 for empty rows).
 *   Either output may be NULL.
 * cb_row_nnz: paper Sec. 4.1, phase (2) (the symbolic phase that finds the
 *   pattern of C).  nnz_out[i] = number of distinct columns in row i of A.B
 *   (int64[m]).
 * cb_exclusive_scan: row pointers from row sizes: out[0] = 0,
 *   out[i+1] = out[i] + in[i] for i < n (int64 in[n], out[n+1]).
 */
int cb_row_stats(cb_ctx *ctx, const cb_csr *A, const cb_csr *B, int64_t *flops,
                 int32_t *maxb);
int cb_row_nnz(cb_ctx *ctx, const cb_csr *A, const cb_csr *B, int64_t *nnz_out);
int cb_exclusive_scan(cb_ctx *ctx, const int64_t *in, int64_t n, int64_t *out);

/* ---- learned row-size predictor -------------------------------------------
 * Paper Sec. 5 (optimizations): the GPU path estimates the output's memory
 * needs with approximate algorithms instead of an exact symbolic pass; Sec.
 * 7.4 sizes batched SpGEMM from such a step.  Here the estimate is a small
 * MLP over three row features f_i = (nnz(A_i), flops_i, max_p nnz(B_p)),
 * the last two taken relative to the row's output width w_i (B's column
 * count), which lets one network serve products of any size:
 *   l = (log2(1 + f_0), log2(1 + f_1) - log2 w_i, log2(1 + f_2) - log2 w_i);
 *   x = bf16((l - mu) / sigma); h1 = bf16(relu(W1 x + b1));
 *   h2 = bf16(relu(W2 h1 + b2)); z = w3 . h2 + b3;
 *   pred_i = clamp(ceil(sigmoid(z) * flops_i), maxB_i, min(flops_i, w_i)).
 * A feature row is CB_MLP_NFEAT floats: nnz(A_i), flops_i, maxB_i, w_i.
 * Weights are used as bf16 copies of fp32 master weights, products are
 * accumulated in fp32.  Parameters are one fp32 vector of CB_MLP_NPARAM
 * values laid out W1[64][3], b1[64], W2[64][64], b2[64], w3[64], b3[1];
 * `norm` is mu[3] followed by sigma[3].  A cb_mlp lives on the device that
 * was current when it was created. */
#define CB_MLP_HIDDEN 64
#define CB_MLP_NPARAM 4481
#define CB_MLP_NFEAT 4
/* Create from host parameters and normalisation (copied); CB_ERR_OOM/CUDA. */
int cb_mlp_create(cb_mlp **out, const float *params, const float *norm);
void cb_mlp_destroy(cb_mlp *m);
/* Copy the fp32 master parameters, the normalisation and the Adam step
 * count back to host memory (checkpointing); any output may be NULL. */
int cb_mlp_get(const cb_mlp *m, float *params, float *norm, int64_t *step);
/* Raw features of every row of A.B: feat[4*i + 0..3] = (nnz(A_i), flops_i,
 * maxB_i, B->ncols) as floats (device float[4*m]). */
int cb_row_features(cb_ctx *ctx, const cb_csr *A, const cb_csr *B, float *feat);
/* K8: logits z[i] and sizes pred[i] for nrows feature rows (device; either
 * output may be NULL); ncols > 0 caps the sizes further (0: only each row's
 * own width). */
int cb_mlp_predict(cb_ctx *ctx, const cb_mlp *m, const float *feat, int64_t nrows, int64_t ncols,
                   float *z, int64_t *pred);
/* K9: mean pinball-loss gradient (quantile tau) over rows with flops > 0
 * against exact sizes nnz[i] (device int64); grad: device float[NPARAM],
 * loss: device float[1] (may be NULL).  Leaves the model unchanged. */
int cb_mlp_grad(cb_ctx *ctx, const cb_mlp *m, const float *feat, const int64_t *nnz,
                int64_t nrows, float tau, float *grad, float *loss);
/* Train in place with Adam (beta 0.9/0.999, eps 1e-8) for `epochs` passes
 * over the rows in mini-batches of `batch` rows; epoch_loss (host float
 * [epochs], may be NULL) receives each epoch's mean loss. */
int cb_mlp_train(cb_ctx *ctx, cb_mlp *m, const float *feat, const int64_t *nnz, int64_t nrows,
                 int epochs, int64_t batch, float lr, float tau, float *epoch_loss);

/* ---- allocation-free scan ------------------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers
 * that cannot allocate device memory when they need the row-pointer scan: a
 * process whose device memory is entirely owned by another allocator (for
 * example a framework's caching pool that reserved the GPU), or a
 * latency-critical loop that must not pay for cudaMalloc's implicit device
 * synchronisation.
 *
 * cb_exclusive_scan_noalloc: same result as cb_exclusive_scan (out[0] = 0,
 *   out[i+1] = out[i] + in[i]; device int64 in[n], out[n+1]), enqueued on
 *   `cuda_stream` (a cudaStream_t, NULL = legacy default stream) of the
 *   current device.  It takes no context and calls no cudaMalloc, cudaFree or
 *   other allocating routine: its scratch (one int64 partial sum per 4096
 *   entries) is a fixed device array of 65,537 int64 (512 KiB + 8 bytes)
 *   inside the library, which every GPU that loads the library holds until
 *   the process exits.
 *   - n may be at most 268,435,456; larger n returns CB_ERR_SCRATCH and
 *     launches nothing.  Bad pointers or n < 0 return CB_ERR_ARG.
 *   - The array's device address belongs to a CUDA context.  The first call
 *     in each context (the device's primary context, a context created after
 *     cudaDeviceReset, or a driver-API context the caller made current) looks
 *     the address up with that context current and caches it under the
 *     context's unique id; make that first call before any stream capture.
 *     A call on a thread with no current context makes the current device's
 *     primary context current.
 *   - Only errors of this call's own launches are reported: an error left
 *     pending by an earlier CUDA call on the thread is neither reported nor
 *     cleared.
 *   - Every call on a device shares the one array, and the array keeps the
 *     last call's contents (nothing needs clearing: each call writes every
 *     entry it reads).  Calls whose work overlaps on the GPU (unordered
 *     streams, or several host threads) race on it and give wrong results:
 *     order them on one stream or with events.
 *   Returns CB_OK or CB_ERR_CUDA (launch failure). */
int cb_exclusive_scan_noalloc(const int64_t *in, int64_t n, int64_t *out, void *cuda_stream);

/* ---- tier bounds and autotuning -------------------------------------------
 * The paper's GPU path picks a library per call by compression factor and
 * flops (Sec. 5); here one set of kernels covers all rows and the bounds
 * between its row tiers are chosen per workload:
 *   sym_hash_max  rows with min(flops_i, ncols) <= this are counted in a
 *                 shared-memory hash table, the rest with dense bitmaps
 *                 (512..4096, default 512);
 *   num_hash_max  rows with nnz(C_i) <= this are computed in a hash table +
 *                 in-row sort, the rest in rank windows (sym_hash_max..4096,
 *                 default 512);
 *   learn_max     with learned or upper-bound sizing, rows whose capacity is
 *                 <= this skip the symbolic phase (0..8192, default 512);
 *   cf_esc, cf_prereduce  the accumulator of a hash-tier row by its
 *                 compression ratio cf = flops_i / nnz(C_i) (paper Sec. 4.1:
 *                 hash for high compression, merging for low, chosen per
 *                 line): cf <= cf_esc expands the products into the table in
 *                 arrival order, sorts them and combines each column's run
 *                 (0..2, default 1.25; 0 = never); cf >= cf_prereduce combines
 *                 the products of each warp step that share a column before
 *                 the hash probe (>= 1, default 4; 1e30 = never); otherwise
 *                 one hash probe per product.
 * cb_ctx_set_tune clamps the values into range (and writes back what it set);
 * cb_autotune tries the compression-ratio bounds after the tier bounds.
 * cb_autotune times cb_spgemm_ex-equivalent runs of A.B on the two-phase
 * path (the bounds steer only that path; the one-launch and work-queue
 * kernels are left out) under a grid of
 * bounds (learn_max too when opt->sizing is learned), keeps the fastest in
 * the context and returns it with its time in ms; it allocates and frees its
 * own output and synchronises the stream. */
typedef struct {
  int32_t sym_hash_max, num_hash_max, learn_max;
  float cf_esc, cf_prereduce;
} cb_tune;
int cb_ctx_set_tune(cb_ctx *ctx, cb_tune *tune);
int cb_ctx_get_tune(const cb_ctx *ctx, cb_tune *tune);
int cb_autotune(cb_ctx *ctx, cb_semiring sr, const cb_csr *A, const cb_csr *B, const cb_opts *opt,
                cb_tune *best, float *best_ms);

/* ---- autotune cache (host only) -------------------------------------------
 * Tuned bounds persist in a JSON file keyed by device name, semiring, sizing
 * mode and size class of the operands, so a later run skips the timing grid.
 * The file is {"format": "cb-tune-cache-1", "entries": {key: {"sym_hash_max",
 * "num_hash_max", "learn_max", "cf_esc", "cf_prereduce", "ms"}}}; updates
 * rewrite it through a temporary file and a rename.
 *
 * cb_tune_key writes "<device>|sr<id>|sizing<mode>|m2^a|a2^b|b2^c" into
 * buf (buf_len bytes including the terminator), where a, b, c are the
 * nearest powers of two of nrows, nnz(A) and nnz(B) (0 for sizes <= 1).
 * CB_ERR_ARG on a null or too small buffer or a negative size.
 *
 * cb_tune_cache_get: *found = 1 and *tune (and *ms when not NULL) filled
 * when key is present; *found = 0 when the key or the file is absent.
 * CB_ERR_ARG when the file cannot be read or is not such a cache (it is
 * then left untouched by cb_tune_cache_put as well).
 *
 * cb_tune_cache_put inserts or replaces key's entry (CB_ERR_ARG when the
 * file cannot be read back as a cache or written).  Readers never see a
 * partial file; of two processes updating the file at once the later rename
 * wins, so the other's new entry may be lost (it is tuned again on its next
 * miss).
 *
 * cb_autotune_cached: with the key of this context's device and the
 * operands, a cached entry is set on the context (clamped as by
 * cb_ctx_set_tune) and returned with its recorded time and *hit = 1, with no
 * GPU work; otherwise it runs cb_autotune, stores the result and returns it
 * with *hit = 0.  A cache error returns CB_ERR_ARG with the reason in
 * cb_last_error. */
int cb_tune_key(const char *device_name, cb_semiring sr, int32_t sizing, int64_t nrows, int64_t nnz_a,
                int64_t nnz_b, char *buf, int64_t buf_len);
int cb_tune_cache_get(const char *path, const char *key, cb_tune *tune, float *ms, int *found);
int cb_tune_cache_put(const char *path, const char *key, const cb_tune *tune, float ms);
int cb_autotune_cached(cb_ctx *ctx, cb_semiring sr, const cb_csr *A, const cb_csr *B,
                       const cb_opts *opt, const char *cache_path, cb_tune *best, float *best_ms,
                       int *hit);

/* ---- semiring SpMSpV ----------------------------------------------------------
 * y^T = x^T A over a semiring: y_c = (+) over stored x entries (i, x_i) and
 * stored A(i, c) of x_i (x) A(i, c) (Sec. 4.3, SpMSpV; the row form suits
 * CSR: for y = A x pass A's transpose in CSR, i.e. A in CSC).  x is a sparse
 * vector of length A->nrows (indices in any order, duplicates contribute
 * separately); y gets length A->ncols, indices strictly increasing, the
 * pattern structural.  (x) takes x's value on the left: with (select2nd,
 * min), y_c = min of A(i, c) over the x entries i; under CB_MAXW_LABEL x
 * holds float32 weights, A int32 labels and y cb_wlabel values.
 * The product is pushed into a dense accumulator kept in the context (one
 * value per column of A plus a bitmap); it is initialised once per width
 * and semiring and reset sparsely after each call.  The stream is
 * synchronised once (to learn nnz(y)); y->idx / y->val are allocated by the
 * library (free with cb_spvec_free_async) unless opt->out_capacity > 0, in
 * which case they are the caller's (CB_ERR_CAPACITY with y->nnz = needed if
 * too small).  opt->validate checks A (row pointers and columns); x's
 * indices are always checked on the device (CB_ERR_INDEX).
 * With opt->flags & CB_FLAG_SPMSPV_BUCKET the column-partitioned form of
 * Sec. 4.3 runs instead (buckets that block y, also called propagation
 * blocking): every product is appended to the bucket of its column (1024
 * columns per bucket), each bucket is (+)-combined by one CTA in a shared-
 * memory accumulator and written in column order; it keeps no state in the
 * context and needs O(products) scratch, with two synchronisations (the
 * product count and nnz(y)). */
typedef struct {
  int64_t n;    /* length                                    */
  int64_t nnz;  /* stored entries                            */
  int32_t *idx; /* device, nnz indices                       */
  void *val;    /* device, nnz values of the semiring's type */
} cb_spvec;
int cb_spmspv(cb_ctx *ctx, cb_semiring sr, const cb_csr *A, const cb_spvec *x, cb_spvec *y,
              const cb_opts *opt);
/* Stream-ordered release of a library-allocated y; zeroes *y. */
int cb_spvec_free_async(cb_ctx *ctx, cb_spvec *y);

/* ---- semiring merge of k partial results ---------------------------------
 * C = P_0 (+) P_1 (+) ... (+) P_{k-1}, entry by entry over the union of the
 * patterns: the combination of the partial products of a SUMMA stage or of
 * the layers of the communication-avoiding SpGEMM (Sec. 3.2).  All parts are
 * device CSR of one shape holding values of the semiring's C type (rows may
 * be unsorted and hold duplicates, which combine the same way); C has
 * sorted, unique columns.  It runs as the SpGEMM (selector) (+).(x)
 * [P_0; ...; P_{k-1}], whose selector row i holds the multiplicative
 * identity at column l*m + i of every part l, so every tier of the SpGEMM
 * (and its one-launch kernel for small rows) serves it; for CB_MAXW_LABEL
 * the selector product runs in that semiring's merge form ((x) passes the
 * part's cb_wlabel through, (+) is CB_MAXW_LABEL's).
 * opt: validate, out_capacity (caller buffers as for cb_spgemm_ex), flags;
 * exact sizing only, no budget.  Returns CB_ERR_SHAPE if the parts differ
 * in shape, CB_ERR_INDEX if k * nrows reaches INT32_MAX. */
int cb_merge(cb_ctx *ctx, cb_semiring sr, int k, const cb_csr *parts, cb_csr *C, const cb_opts *opt);

/* ---- one-launch SpGEMM for small rows -----------------------------------
 * The row-wise SpGEMM of Sec. 4.1 with its symbolic and numeric phases fused
 * into one kernel launch, for products whose rows are all small:
 *   - every row of A holds at most `lanes` entries (lanes = 8, 16 or 32),
 *   - every row of C has at most 8 * lanes products (flops_i),
 *   - B->ncols <= cb_fused_max_cols(lanes) (2^26 - 1 for 8 lanes).
 * Each row is formed by `lanes` threads (products in registers, sorted by a
 * register bitonic network, equal columns merged), and each CTA finds its
 * output offset from the earlier CTAs' row totals, so C comes out compact
 * and sorted without a host synchronisation.
 *   C->row_ptr (A->nrows + 1 int64), C->col (int32) and C->val (the
 *   semiring's type) are caller-provided device buffers, col/val holding
 *   `capacity` entries; C->nrows/ncols are set, C->nnz to -1 (nnz(C) is
 *   C->row_ptr[nrows] on the device).
 *   `status` is a device int that the kernel ORs CB_FUSED_* bits into (the
 *   caller zeroes it); any bit set means C is not valid.
 * Inputs are not validated (see cb_spgemm_ex).  Nothing is synchronised; the
 * first call on a context, or one with more rows than any earlier call,
 * allocates the context's tile-status array (so call once before capturing
 * the launch into a CUDA graph); later calls allocate nothing.  Calls on one
 * context must be ordered on its stream.  Returns CB_ERR_ARG for bad
 * arguments or lanes, else CB_OK / CB_ERR_CUDA. */
enum {
  CB_FUSED_CAPACITY = 1,      /* nnz(C) > capacity: nothing past capacity written */
  CB_FUSED_ROW_TOO_LARGE = 2, /* a row beyond the lanes' bounds (left empty)      */
  CB_FUSED_STALLED = 4        /* a CTA gave up waiting for an earlier CTA's total  */
};
int cb_spgemm_fused(cb_ctx *ctx, cb_semiring sr, const cb_csr *A, const cb_csr *B, cb_csr *C,
                    int64_t capacity, int lanes, int *status);
/* Largest column count cb_spgemm_fused takes with `lanes` lanes per row. */
int64_t cb_fused_max_cols(int lanes);
/* Smallest lanes (8, 16, 32) whose bounds every row of A.B meets, or 0 if
 * none; *flops (optional) receives the total product count, an upper bound
 * of nnz(C).  Synchronises ctx's stream. */
int cb_fused_lanes(cb_ctx *ctx, const cb_csr *A, const cb_csr *B, int *lanes, int64_t *flops);

/* Statistics of the most recent cb_spgemm_ex on this context (host memory). */
typedef struct {
  int64_t flops;        /* number of (x)-products                              */
  int64_t nnz;          /* nnz(C)                                              */
  int64_t heavy_rows;   /* rows computed in rank windows                       */
  int64_t heavy_units;  /* rank windows launched for heavy rows                */
  int64_t overflow_rows;/* rows recomputed exactly after a sizing overflow     */
  int32_t batches;      /* column batches (1 when not batched)                 */
  int32_t kernels;      /* kernel launches issued by the call                  */
  /* phase durations in ms (CB_FLAG_TIMING only, else 0): K1+K2 flops and
   * binning; K3 symbolic; K4 scan + numeric binning; K5-K7 numeric. */
  float ms_stats, ms_symbolic, ms_scan, ms_numeric;
} cb_stats;
int cb_last_stats(const cb_ctx *ctx, cb_stats *out);

/* ---- fault injection -----------------------------------------------------
 * Test hooks for the failure paths (allocation failure, a bounded device wait
 * that expires).  They make the failure on the host side or give a wait a
 * producer that never publishes; nothing here faults, traps or hangs a GPU.
 *   CB_FAULT_ALLOC: arg = k >= 1 makes the k-th device allocation that the
 *     context makes from now on (its workspaces, C, staging buffers) fail as
 *     if the device were out of memory, once; the call returns CB_ERR_OOM
 *     with C zeroed and owning nothing, and the context stays usable.
 *     arg = 0 turns it off.  arg2 is ignored.
 *   CB_FAULT_SILENT_TILE: in the one-launch kernel (cb_spgemm_fused and the
 *     automatic branch of cb_spgemm_ex) tile `arg` (>= 0; 32 rows per tile
 *     at 8 lanes, 16 at 16, 8 at 32), and in the work-queue kernel row
 *     `arg`, never publishes its total, and every look-back wait gives up
 *     after arg2 polls (1 <= arg2 <= 2^20).
 *     Waiting tiles record CB_FUSED_STALLED and publish anyway, so the launch
 *     ends; cb_spgemm_ex returns CB_ERR_TIMEOUT with C zeroed.  arg < 0
 *     restores the defaults (no silent tile, 2^20 polls).
 *   CB_FAULT_SHORT_ROW: on the two-phase path, row `arg`'s exact size is made
 *     one short after the symbolic phase (the inconsistent count a faulty
 *     symbolic kernel would leave); arg < 0 turns it off.  Every write of the
 *     numeric phase stays inside C's arrays: the normal library drops the
 *     row's surplus entry (CB_FLAG_CHECK reports it as a consistency failure
 *     when a hash tier forms the row), the CB_CHECK debug library reports
 *     the failed bound (see the debug build below).
 * Returns CB_ERR_ARG for an unknown kind or an argument out of range. */
enum { CB_FAULT_ALLOC = 1, CB_FAULT_SILENT_TILE = 2, CB_FAULT_SHORT_ROW = 3 };
int cb_ctx_set_fault(cb_ctx *ctx, int kind, int64_t arg, int64_t arg2);

/* ---- debug build -----------------------------------------------------------
 * libcb_check.so is this library compiled with -DCB_CHECK: the same entry
 * points, plus a run-time bounds check on every CSR write and every shared or
 * global hash-table access of the SpGEMM kernels (flop count, symbolic,
 * numeric, one-launch and work-queue kernels, the learned-sizing copy).  A
 * failed check skips the access and records its code and index on the device
 * (no trap); cb_spgemm_ex, cb_spgemm_batched, cb_spgemm_fused and cb_merge
 * then synchronise and return CB_ERR_CUDA with "bounds check <code> failed at
 * index <i> (<file> kernels)" in cb_last_error (C zeroed when library-
 * allocated).  It is slower and meant for tests and debugging. */

#ifdef __cplusplus
}
#endif
#endif /* CB_H_ */
