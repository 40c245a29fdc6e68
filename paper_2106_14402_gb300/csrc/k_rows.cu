// Row-level kernels of the SpGEMM path: input validation, the per-row flops
// estimate and load-balance binning (paper Sec. 4.1, phase (1)), the int64
// exclusive scan that turns row sizes into row pointers, and the list of
// heavy-row column-slice work units.
#include "cb_common.cuh"
#include "cb_kernels.h"

namespace cb {

namespace {

__device__ __forceinline__ void set_error(int64_t* counters, int64_t code, int64_t detail) {
  if (atomicCAS((unsigned long long*)&counters[kError], 0ull, (unsigned long long)code) == 0ull)
    counters[kErrDetail] = detail;
}

__global__ void k_validate(DevCSR M, int64_t nnz, int code_base, int64_t* counters) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (tid == 0 && (M.rp[0] != 0 || M.rp[M.nrows] != nnz)) set_error(counters, code_base + 1, 0);
  for (int64_t i = tid; i < M.nrows; i += stride)
    if (M.rp[i + 1] < M.rp[i]) set_error(counters, code_base + 1, i);
  for (int64_t q = tid; q < nnz; q += stride) {
    int32_t c = M.col[q];
    if (c < 0 || (int64_t)c >= M.ncols) set_error(counters, code_base + 2, q);
  }
}

// K1: one warp per row of A.  flops_i = sum of B row lengths over the row's
// stored entries (the flops count of Table 1), maxb_i = the longest of them.
__global__ void __launch_bounds__(256) k_classify_sym(DevCSR A, DevCSR B, int64_t* flops,
                                                      int32_t* maxb, int64_t* counters,
                                                      const uint8_t* skip, int64_t sym_hash_max) {
  __shared__ unsigned long long hist[kSymTiers];
  __shared__ unsigned long long total;
  __shared__ long long max_f, max_a;
  if (threadIdx.x < kSymTiers) hist[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    total = 0;
    max_f = 0;
    max_a = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < A.nrows;
       i += nwarps) {
    const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
    long long f = 0;
    int mx = 0;
    for (int64_t p = a0 + lane; p < a1; p += 32) {
      const int k = A.col[p];
      const int64_t len = row_end(B, k) - B.rp[k];
      f += len;
      mx = max(mx, (int)min(len, (int64_t)INT_MAX));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      f += __shfl_down_sync(0xffffffffu, f, o);
      mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
      flops[i] = f;
      if (maxb) maxb[i] = mx;
      atomicAdd(&hist[skip && skip[i] ? 0 : sym_tier(min((int64_t)f, row_width(A, B, i)), sym_hash_max)],
                1ull);
      atomicAdd(&total, (unsigned long long)f);
      atomicMax(&max_f, f);
      atomicMax(&max_a, (long long)(a1 - a0));
    }
  }
  __syncthreads();
  if (threadIdx.x < kSymTiers && hist[threadIdx.x])
    atomicAdd((unsigned long long*)&counters[kCntSym + threadIdx.x], hist[threadIdx.x]);
  if (threadIdx.x == 0) {
    if (total) atomicAdd((unsigned long long*)&counters[kTotalFlops], total);
    if (max_f) atomicMax((long long*)&counters[kMaxFlops], max_f);
    if (max_a) atomicMax((long long*)&counters[kMaxArow], max_a);
  }
}

struct TierBySize {
  const int64_t* v;
  int64_t cap, t1, t2, t3;
  const uint8_t* skip;         // rows with skip[i] != 0 are left out (tier 0)
  const int32_t* rcap = nullptr;  // per-row cap (replaces cap when set)
  __device__ __forceinline__ int operator()(int64_t i) const {
    if (skip && skip[i]) return 0;
    const int64_t u = min(v[i], rcap ? (int64_t)rcap[i] : cap);
    return u == 0 ? 0 : u <= t1 ? 1 : u <= t2 ? 2 : u <= t3 ? 3 : 4;
  }
};

__global__ void __launch_bounds__(256) k_tier_count(int64_t m, TierBySize tier, int64_t* cnt) {
  __shared__ unsigned long long hist[5];
  if (threadIdx.x < 5) hist[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&hist[tier(i)], 1ull);
  __syncthreads();
  if (threadIdx.x < 5 && hist[threadIdx.x])
    atomicAdd((unsigned long long*)&cnt[threadIdx.x], hist[threadIdx.x]);
}

// K2: place row i into the segment of its tier inside perm (tiers 1..4 in
// order; tier 0 rows are empty or skipped and get no slot).  zero_nnz
// (optional): rows of tier 0 and 4 get nnz = 0 (tier 4 rows are summed slice
// by slice later), except skipped rows, which get preset[i].
__global__ void __launch_bounds__(256) k_tier_scatter(int64_t m, TierBySize tier, int32_t* perm,
                                                      const int64_t* cnt, int64_t* cur,
                                                      int64_t* zero_nnz, const int64_t* preset) {
  __shared__ int local[5];
  __shared__ long long base[5];
  if (threadIdx.x < 5) local[threadIdx.x] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int t = -1, slot = 0;
  if (i < m) {
    t = tier(i);
    if (zero_nnz) {
      if (tier.skip && tier.skip[i]) zero_nnz[i] = preset ? preset[i] : 0;
      else if (t == 0 || t == 4) zero_nnz[i] = 0;
    }
    if (t > 0) slot = atomicAdd(&local[t], 1);
  }
  __syncthreads();
  if (threadIdx.x > 0 && threadIdx.x < 5 && local[threadIdx.x]) {
    long long seg = 0;
    for (int u = 1; u < (int)threadIdx.x; ++u) seg += cnt[u];
    base[threadIdx.x] =
        seg + (long long)atomicAdd((unsigned long long*)&cur[threadIdx.x], (unsigned long long)local[threadIdx.x]);
  }
  __syncthreads();
  if (t > 0) perm[base[t] + slot] = (int32_t)i;
}

// K4: three-pass exclusive scan (tile reduce, scan of tile sums, apply).
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
static_assert(kScanTile == kScanTileItems, "scan tile size is shared with the allocation-free scan");

__device__ __forceinline__ long long block_exclusive_scan(long long x, long long* warp_tot,
                                                         long long& block_total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    long long v = lane < nw ? warp_tot[lane] : 0;
    long long vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < nw) warp_tot[lane] = vi - v;
    if (lane == nw - 1) warp_tot[32] = vi;
  }
  __syncthreads();
  block_total = warp_tot[32];
  const long long r = warp_tot[w] + incl - x;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int64_t* in, int64_t n,
                                                              int64_t* partial) {
  __shared__ long long wt[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  long long s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j)
    if (base + j < n) s += in[base + j];
  long long tot;
  block_exclusive_scan(s, wt, tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partials(int64_t* partial, int64_t nb,
                                                                int64_t* out_total) {
  __shared__ long long wt[33];
  long long carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int64_t b = b0 + threadIdx.x;
    const long long v = b < nb ? partial[b] : 0;
    long long tot;
    const long long ex = block_exclusive_scan(v, wt, tot);
    if (b < nb) partial[b] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *out_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int64_t* in, int64_t n,
                                                             const int64_t* partial, int64_t* out) {
  __shared__ long long wt[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  long long v[kScanItems];
  long long s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < n ? in[base + j] : 0;
    s += v[j];
  }
  long long tot;
  long long run = block_exclusive_scan(s, wt, tot) + partial[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
}

// Column-batch slab offsets (paper Sec. 7.2, batched SpGEMM): for every row
// k of B and every batch boundary bnd[j] (j < nb1), pos[j * n + k] is the
// first entry of row k whose column is >= bnd[j].  Rows must be
// non-decreasing.  One warp per row, one cooperative search per boundary.
__global__ void __launch_bounds__(256) k_slabs(DevCSR B, const int64_t* bnd, int nb1, int64_t* pos) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const Group g(5, lane);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < B.nrows;
       r += nwarps) {
    const int64_t q0 = B.rp[r], q1 = B.rp[r + 1];
    for (int j = 0; j < nb1; ++j) {
      const int64_t v = group_lower_bound(B.col, q0, q1, bnd[j], g);
      if (lane == 0) pos[(int64_t)j * B.nrows + r] = v;
    }
  }
}

// out[j] = prefix[idx[j]] for j < n (gather of a few prefix values).
__global__ void k_gather(const int64_t* prefix, const int64_t* idx, int64_t n, int64_t* out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    out[j] = prefix[idx[j]];
}

inline int grid_for(int64_t work, int per_block, int cap) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

}  // namespace

void launch_validate(const DevCSR& M, int64_t nnz, int code_base, int64_t* counters,
                     cudaStream_t s, int sms) {
  k_validate<<<grid_for(nnz + M.nrows, 256, sms * 8), 256, 0, s>>>(M, nnz, code_base, counters);
}

void launch_classify_sym(const DevCSR& A, const DevCSR& B, int64_t* flops, int32_t* maxb,
                         int64_t* counters, cudaStream_t s, int sms, const uint8_t* skip,
                         int64_t sym_hash_max) {
  k_classify_sym<<<grid_for(A.nrows, 8, sms * 8), 256, 0, s>>>(A, B, flops, maxb, counters, skip,
                                                                sym_hash_max);
}

void launch_scatter_sym(int64_t m, int64_t ncols, const int64_t* flops, int32_t* perm,
                        int64_t* nnz, int64_t* counters, cudaStream_t s, int,
                        const uint8_t* skip, const int64_t* preset, int64_t sym_hash_max,
                        const int32_t* rcols) {
  TierBySize t{flops, ncols, kSymWarpMax, kSymSmallMax, sym_hash_max, skip, rcols};
  k_tier_scatter<<<grid_for(m, 256, 1 << 30), 256, 0, s>>>(m, t, perm, counters + kCntSym,
                                                            counters + kCurSym, nnz, preset);
}

namespace {
__global__ void k_merge_error(const int64_t* src, int64_t* dst) {
  if (threadIdx.x == 0 && *src) atomicMax(reinterpret_cast<long long*>(dst), (long long)*src);
}
}  // namespace

void launch_merge_error(const int64_t* src, int64_t* dst, cudaStream_t s) {
  k_merge_error<<<1, 32, 0, s>>>(src, dst);
}

int64_t scan_partials(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

// The kernels are launched with cudaLaunchKernel, whose return value is the
// error of that launch alone (a <<<>>> launch is only seen through
// cudaGetLastError, which also reports errors left by earlier calls).
cudaError_t launch_exclusive_scan(const int64_t* in, int64_t n, int64_t* out, int64_t* partial,
                                  cudaStream_t s) {
  if (n < 0) return cudaErrorInvalidValue;
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb > kScanMaxTiles) return cudaErrorInvalidValue;
  int64_t* total = out + n;
  void* reduce_args[] = {(void*)&in, (void*)&n, (void*)&partial};
  void* partials_args[] = {(void*)&partial, (void*)&nb, (void*)&total};
  void* apply_args[] = {(void*)&in, (void*)&n, (void*)&partial, (void*)&out};
  cudaError_t e = cudaLaunchKernel((const void*)k_scan_reduce, dim3((unsigned)nb), dim3(kScanThreads),
                                   reduce_args, 0, s);
  if (e == cudaSuccess)
    e = cudaLaunchKernel((const void*)k_scan_partials, dim3(1), dim3(kScanThreads), partials_args, 0, s);
  if (e == cudaSuccess)
    e = cudaLaunchKernel((const void*)k_scan_apply, dim3((unsigned)nb), dim3(kScanThreads), apply_args,
                         0, s);
  return e;
}

void launch_gather(const int64_t* prefix, const int64_t* idx, int64_t n, int64_t* out,
                   cudaStream_t s) {
  if (n > 0) k_gather<<<grid_for(n, 256, 1024), 256, 0, s>>>(prefix, idx, n, out);
}

void launch_slabs(const DevCSR& B, const int64_t* bnd, int nb1, int64_t* pos, cudaStream_t s,
                  int sms) {
  if (B.nrows == 0 || nb1 == 0) return;
  k_slabs<<<grid_for(B.nrows, 8, sms * 8), 256, 0, s>>>(B, bnd, nb1, pos);
}

void launch_classify_num(int, int64_t m, const int64_t* nnz, int32_t* perm, int64_t* counters,
                         cudaStream_t s, int sms, const uint8_t* skip, int64_t num_hash_max) {
  TierBySize t{nnz, INT64_MAX, kNumWarpMax, kNumSmallMax, num_hash_max, skip};
  k_tier_count<<<grid_for(m, 256, sms * 8), 256, 0, s>>>(m, t, counters + kCntNum);
  k_tier_scatter<<<grid_for(m, 256, 1 << 30), 256, 0, s>>>(m, t, perm, counters + kCntNum,
                                                            counters + kCurNum, nullptr, nullptr);
}

// Learned sizing: capacity of each row from its predicted size, and whether
// the row takes the one-pass hash path (cap <= hash_max) or the exact path.
// cap = min(bound, max(pred, ceil(pred * (1 + margin)))), bound = min(flops, ncols);
// learned rows also get their tier histogram in cnt[0..4] (by cap).
__global__ void __launch_bounds__(256) k_learn_caps(int64_t m, const int64_t* pred,
                                                    const int64_t* flops, int64_t ncols,
                                                    float margin, int64_t hash_max, int64_t* cap,
                                                    uint8_t* learned, const int32_t* rcols) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = flops[i];
    const int64_t w = rcols ? (int64_t)rcols[i] : ncols;
    const int64_t bound = f < w ? f : w;
    int64_t p = pred ? pred[i] : bound;
    int64_t c = (int64_t)ceil((double)p * (1.0 + (double)margin));
    if (c < p) c = p;
    if (c > bound) c = bound;
    const bool l = f > 0 && c <= hash_max;
    learned[i] = l ? 1 : 0;
    cap[i] = l ? c : 0;
  }
}

// Fault injection: one row's exact size one short, as a faulty symbolic
// phase would leave it.
__global__ void k_fault_shrink(int64_t* n) {
  if (*n > 0) *n -= 1;
}

// Copy the rows computed in one pass from their staging slots into C.
// One warp per row.
template <class T>
__global__ void __launch_bounds__(256) k_compact_rows(int64_t m, const uint8_t* learned,
                                                      const int64_t* stage_rp, const int64_t* cnt,
                                                      const int32_t* scol, const T* sval,
                                                      const int64_t* Crp, int32_t* Ccol, T* Cval) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += nwarps) {
    if (!learned[i]) continue;
    const int64_t src = stage_rp[i], dst = Crp[i], n = cnt[i];
    if (!chk(dst + n <= Crp[i + 1], 45, dst + n)) continue;
    for (int64_t t = lane; t < n; t += 32) {
      Ccol[dst + t] = scol[src + t];
      Cval[dst + t] = sval[src + t];
    }
  }
}

void launch_fault_shrink(int64_t* nnz_row, cudaStream_t s) {
  k_fault_shrink<<<1, 1, 0, s>>>(nnz_row);
}

void launch_learn_caps(int64_t m, const int64_t* pred, const int64_t* flops, int64_t ncols,
                       float margin, int64_t hash_max, int64_t* cap, uint8_t* learned,
                       cudaStream_t s, int sms, const int32_t* rcols) {
  if (m == 0) return;
  k_learn_caps<<<grid_for(m, 256, sms * 8), 256, 0, s>>>(m, pred, flops, ncols, margin, hash_max,
                                                          cap, learned, rcols);
}

void launch_learned_tiers(int64_t m, const int64_t* cap, int64_t hash_max, int32_t* perm,
                          int64_t* counters, cudaStream_t s, int sms) {
  TierBySize t{cap, INT64_MAX, kNumWarpMax, kNumSmallMax, hash_max, nullptr};
  k_tier_count<<<grid_for(m, 256, sms * 8), 256, 0, s>>>(m, t, counters + kCntNum);
  k_tier_scatter<<<grid_for(m, 256, 1 << 30), 256, 0, s>>>(m, t, perm, counters + kCntNum,
                                                            counters + kCurNum, nullptr, nullptr);
}

void launch_compact_rows(int vsz, int64_t m, const uint8_t* learned, const int64_t* stage_rp,
                         const int64_t* cnt, const int32_t* scol, const void* sval,
                         const int64_t* Crp, int32_t* Ccol, void* Cval, cudaStream_t s, int sms) {
  if (m == 0) return;
  const int g = grid_for(m, 8, sms * 16);
  switch (vsz) {
    case 8:
      k_compact_rows<uint64_t><<<g, 256, 0, s>>>(m, learned, stage_rp, cnt, scol,
                                                 static_cast<const uint64_t*>(sval), Crp, Ccol,
                                                 static_cast<uint64_t*>(Cval));
      break;
    case 4:
      k_compact_rows<uint32_t><<<g, 256, 0, s>>>(m, learned, stage_rp, cnt, scol,
                                                 static_cast<const uint32_t*>(sval), Crp, Ccol,
                                                 static_cast<uint32_t*>(Cval));
      break;
    default:
      k_compact_rows<uint8_t><<<g, 256, 0, s>>>(m, learned, stage_rp, cnt, scol,
                                                static_cast<const uint8_t*>(sval), Crp, Ccol,
                                                static_cast<uint8_t*>(Cval));
  }
}

CB_CHECK_READER(rows)

}  // namespace cb
