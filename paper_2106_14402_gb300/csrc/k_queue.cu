// One-pass SpGEMM for rows of bounded size and width, run by a persistent
// kernel that takes rows from a device work queue.  It serves the batched
// workloads of many independent products (paper Sec. 5 runs one library
// call per product; here the stacked rows of all products of a wave are one
// queue), where every output row holds at most kQueueAcc entries and lies in
// a column range of at most kQueueWidth columns.
//
// The three phases of Sec. 4.1 collapse per row, in one CTA:
//   1. flops bound and load balance: a warp per stored A entry walks that
//      entry's B row with coalesced loads;
//   2. symbolic: the products' columns set bits of a dense bitmap of the
//      row's column range; popcounts, prefix-summed, give nnz(C_i) and every
//      column's rank;
//   3. numeric: the products are combined with the semiring's atomic at the
//      rank of their column in a shared-memory accumulator, so the row reads
//      out in column order (columns from the bitmap, values by rank) with no
//      sort.
// Rows are dequeued in order with one atomic per row, and a row's output
// offset comes from a decoupled look-back over the rows before it, whose
// CTAs are all running (they dequeued earlier) and never wait on later rows:
// no cooperative launch is needed.  Row status words carry the launch epoch
// of the one-launch kernel (shared tile-status array and sync words), so no
// reset is needed between launches.  Waits are bounded: a row that gives up
// records CB_FUSED_STALLED and publishes anyway.  (spin_limit and silent_row
// serve fault injection: a row that never publishes.)
#include <algorithm>

#include "cb.h"
#include "cb_common.cuh"
#include "cb_kernels.h"

namespace cb {
namespace {

constexpr int kQThreads = 256;
constexpr int kQWarps = kQThreads / 32;
constexpr int kQWords = kQueueWidth / 32;   // bitmap words of the widest row
constexpr unsigned kQFull = 0xFFFFFFFFu;

// status words: [63:40] epoch, [39:38] kind, [37:0] value (as in k_fused.cu)
constexpr int kQEpochShift = 40;
constexpr unsigned kQEpochMask = (1u << 24) - 1;
constexpr unsigned long long kQAgg = 1ull << 38;
constexpr unsigned long long kQInc = 2ull << 38;
constexpr unsigned long long kQKind = 3ull << 38;
constexpr unsigned long long kQVal = (1ull << 38) - 1;

__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

template <int SR>
__global__ void __launch_bounds__(kQThreads) k_queue_rows(DevCSR A, DevCSR B, int64_t m,
                                                          int64_t* __restrict__ Crp,
                                                          int32_t* __restrict__ Ccol,
                                                          typename Sem<SR>::TC* __restrict__ Cval,
                                                          int64_t cap, unsigned long long* tstat,
                                                          int64_t tstat_cap, unsigned* sync,
                                                          int* status, unsigned spin_limit,
                                                          int64_t silent_row) {
  typedef Sem<SR> S;
  typedef typename S::A Acc;
  typedef typename S::TA TA;
  typedef typename S::TB TB;
  __shared__ unsigned bits[kQWords];
  __shared__ unsigned short pre[kQWords];   // entries in the row's earlier words (< kQueueAcc)
  __shared__ Acc acc[kQueueAcc];
  __shared__ int s_wsum[kQWarps];
  __shared__ int s_min[kQWarps];
  __shared__ long long s_red[kQWarps];
  __shared__ long long s_row, s_base;
  __shared__ int s_nnz, s_touched;
  __shared__ unsigned s_epoch, s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TA* __restrict__ Aval = reinterpret_cast<const TA*>(A.val);
  const TB* __restrict__ Bval = reinterpret_cast<const TB*>(B.val);
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(sync + 10);
  if (tid == 0) s_epoch = *reinterpret_cast<volatile unsigned*>(sync) & kQEpochMask;
  for (int t = tid; t < kQueueAcc; t += kQThreads) acc[t] = S::ident();
  __syncthreads();
  const unsigned long long ep = (unsigned long long)s_epoch << kQEpochShift;

  for (;;) {
    if (tid == 0) s_row = (long long)atomicAdd(queue, 1ull);
    __syncthreads();
    const int64_t r = s_row;
    if (r >= m) break;
    const int64_t width = row_width(A, B, r);
    const int nw = (int)((width + 31) >> 5);
    const int64_t a0 = A.rp[r], a1 = A.rp[r + 1];
    for (int w = tid; w < nw; w += kQThreads) bits[w] = 0u;
    __syncthreads();

    // symbolic: the row's columns (a warp per stored A entry)
    for (int64_t p = a0 + warp; p < a1; p += kQWarps) {
      const int k = __ldg(A.col + p);
      const int64_t q1 = row_end(B, k);
      for (int64_t q = __ldg(B.rp + k) + lane; q < q1; q += 32) {
        const unsigned c = (unsigned)__ldg(B.col + q) - (unsigned)B.col_lo;
        if (guard(c < (unsigned)width, 42, c)) atomicOr(&bits[c >> 5], 1u << (c & 31));
      }
    }
    __syncthreads();

    // ranks: exclusive prefix of the word popcounts (each thread a run of words)
    const int per = (nw + kQThreads - 1) / kQThreads;
    const int w0 = tid * per;
    int mine = 0;
    for (int w = w0; w < w0 + per && w < nw; ++w) mine += __popc(bits[w]);
    int incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(kQFull, incl, d);
      if (lane >= d) incl += y;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    int before = 0, nnz = 0;
#pragma unroll
    for (int v = 0; v < kQWarps; ++v) {
      const int x = s_wsum[v];
      before += v < warp ? x : 0;
      nnz += x;
    }
    int touched = nnz;  // accumulator slots the numeric pass may write
    if (nnz > kQueueAcc) {  // the row does not fit this kernel (uniform)
      if (tid == 0) atomicOr(status, CB_FUSED_ROW_TOO_LARGE);
      nnz = 0;
      touched = kQueueAcc;
    }
    {
      int run = before + incl - mine;
      for (int w = w0; w < w0 + per && w < nw; ++w) {
        pre[w] = (unsigned short)(run < kQueueAcc ? run : kQueueAcc);
        run += __popc(bits[w]);
      }
    }
    // publish the row's size, then find its offset from the rows before it
    if (tid == 0 && r != silent_row)  // (fault injection: a row that never publishes)
      atomicExch(&tstat[r], ep | (r == 0 ? kQInc : kQAgg) | (unsigned long long)nnz);
    __syncthreads();  // the ranks are complete
    long long excl = 0;
    for (int64_t top = r - 1; top >= 0; top -= kQThreads) {
      const int64_t j = top - tid;
      unsigned long long wv = 0;
      bool inc_here = false;
      long long val = 0;
      if (j >= 0) {
        unsigned spins = 0;
        for (;;) {
          wv = ld_volatile64(&tstat[j]);
          if ((wv & ~((1ull << kQEpochShift) - 1)) == ep && (wv & kQKind)) break;
          if (++spins >= spin_limit) {
            atomicOr(status, CB_FUSED_STALLED);
            wv = ep | kQInc;
            break;
          }
          __nanosleep(32);
        }
        inc_here = (wv & kQKind) == kQInc;
        val = (long long)(wv & kQVal);
      }
      // the nearest inclusive prefix in this window (smallest thread index)
      int first = __reduce_min_sync(kQFull, inc_here ? tid : kQThreads);
      if (lane == 0) s_min[warp] = first;
      __syncthreads();
      int stop = kQThreads;
#pragma unroll
      for (int v = 0; v < kQWarps; ++v) stop = min(stop, s_min[v]);
      long long part = (j >= 0 && tid <= stop) ? val : 0;
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) part += __shfl_xor_sync(kQFull, part, d);
      if (lane == 0) s_red[warp] = part;
      __syncthreads();
#pragma unroll
      for (int v = 0; v < kQWarps; ++v) excl += s_red[v];
      __syncthreads();
      if (stop < kQThreads) break;
    }
    if (tid == 0) {
      if (r > 0 && r != silent_row) atomicExch(&tstat[r], ep | kQInc | (unsigned long long)(excl + nnz));
      s_base = excl;
      s_nnz = nnz;
      s_touched = touched;
      Crp[r] = excl;
      if (r == m - 1) {
        Crp[m] = excl + nnz;
        __threadfence();  // before this CTA counts itself finished
      }
    }

    // numeric: products at their column's rank
    for (int64_t p = a0 + warp; p < a1; p += kQWarps) {
      const int k = __ldg(A.col + p);
      const TA a = S::kUsesA ? ldg_val(Aval + p) : TA();
      const int64_t q1 = row_end(B, k);
      for (int64_t q = __ldg(B.rp + k) + lane; q < q1; q += 32) {
        const unsigned c = (unsigned)__ldg(B.col + q) - (unsigned)B.col_lo;
        if (c < (unsigned)width) {
          const unsigned wb = bits[c >> 5];
          const int slot = (int)pre[c >> 5] + __popc(wb & ((1u << (c & 31)) - 1u));
          if (guard(slot < kQueueAcc, 43, slot)) S::atomic(&acc[slot], S::mul(a, ldg_val(Bval + q)));
        }
      }
    }
    __syncthreads();

    // write the row: values by rank (coalesced), columns from the bitmap;
    // the accumulator returns to the identity for the next row
    const long long base = s_base;
    const int n = s_nnz;
    if (base + n > cap) {
      if (tid == 0 && n > 0) atomicOr(status, CB_FUSED_CAPACITY);
      for (int t = tid; t < s_touched; t += kQThreads) acc[t] = S::ident();
    } else {
      for (int t = tid; t < s_touched; t += kQThreads) {
        if (t < n) st_out(Cval + base + t, S::out(acc[t]));
        acc[t] = S::ident();
      }
      for_bitmap_columns<kDenseWordBits, kQThreads>(bits, pre, nw, n, [&](int j, int c) {
        const long long o = base + j;
        if (chk(o < base + n, 44, o)) st_out(Ccol + o, (int32_t)(B.col_lo + c));
      });
    }
    __syncthreads();
  }

  // the last CTA to finish records nnz(C), advances the epoch and resets
  // the queue (status words are cleared when the 24-bit epoch wraps)
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(&sync[1], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    if (tid == 0) {
      __threadfence();
      unsigned long long* s64 = reinterpret_cast<unsigned long long*>(sync);
      s64[1] = m > 0 ? (unsigned long long)*reinterpret_cast<volatile int64_t*>(Crp + m) : 0ull;
    }
    const unsigned ne = (s_epoch + 1) & kQEpochMask;
    if (ne == 0)
      for (int64_t j = tid; j < tstat_cap; j += kQThreads) tstat[j] = 0;
    __syncthreads();
    if (tid == 0) {
      *queue = 0;
      sync[1] = 0;
      __threadfence();
      atomicExch(&sync[0], ne);
    }
  }
}

template <int SR>
cudaError_t launch_queue_sr(const DevCSR& A, const DevCSR& B, int64_t m, int64_t* Crp, int32_t* Ccol,
                            void* Cval, int64_t cap, unsigned long long* tstat, int64_t tstat_cap,
                            unsigned* sync, int* status, cudaStream_t s, int sms, unsigned spin_limit,
                            int64_t silent_row) {
  if (m > tstat_cap) return cudaErrorInvalidValue;
  static int per_sm = 0;  // resident CTAs per SM (same for every device of one kind)
  if (per_sm == 0) {
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_queue_rows<SR>, kQThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
  }
  const int64_t grid = std::min<int64_t>(m, (int64_t)per_sm * sms);
  k_queue_rows<SR><<<(unsigned)grid, kQThreads, 0, s>>>(A, B, m, Crp, Ccol,
                                                       static_cast<typename Sem<SR>::TC*>(Cval), cap,
                                                       tstat, tstat_cap, sync, status,
                                                       spin_limit < 1 ? 1u : spin_limit, silent_row);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_queue_rows(int sr, const DevCSR& A, const DevCSR& B, int64_t m, int64_t* Crp,
                              int32_t* Ccol, void* Cval, int64_t cap, unsigned long long* tstat,
                              int64_t tstat_cap, unsigned* sync, int* status, cudaStream_t s, int sms,
                              unsigned spin_limit, int64_t silent_row) {
  if (m <= 0) return cudaSuccess;
  switch (sr) {
#define CB_CASE(SRV) \
  case SRV: return launch_queue_sr<SRV>(A, B, m, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms, spin_limit, silent_row);
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
  }
  return cudaErrorInvalidValue;
}

CB_CHECK_READER(queue)

}  // namespace cb
