// One-launch SpGEMM for products whose rows are all small: every row of A
// holds at most G entries and every output row at most 8G products
// (G = 8, 16 or 32 lanes per row).  The symbolic and numeric phases of the
// paper's row-wise SpGEMM (Sec. 4.1) collapse into one pass over the rows:
//
//   1. a group of G lanes takes one row; lane g loads A entry g and the
//      bounds of B row A.col[g]; a scan over the group numbers the row's
//      products t = 0..F-1;
//   2. lane g forms products t = r*G + g (r = 0..7) -- the owning A entry is
//      found by a binary search over the group's scan with shuffles -- and
//      keeps the key (column << log2(8G)) | t in a register, the product in
//      shared memory;
//   3. the 8G keys are sorted in registers (bitonic network: in-lane stages
//      on registers, cross-lane stages on shuffles); equal columns are then
//      adjacent and are merged into one output entry (in t order, so FP64
//      sums are deterministic), staged in shared memory in column order;
//   4. each CTA publishes its tile's row total and finds its output offset
//      with a CTA-wide look-back over the earlier tiles' totals (each thread
//      polls one earlier tile; the nearest tile that published its inclusive
//      prefix ends the walk), then writes row pointers and entries with
//      coalesced stores.
//
// The grid is a cooperative launch (every CTA resident), so each CTA walks
// tiles blockIdx.x, blockIdx.x + gridDim.x, ... and the tile it waits for is
// always being worked on.  Tile status words carry a launch epoch that the
// last CTA to finish advances, so no reset is needed between launches (CUDA
// graph replays included).  Polls are bounded: a tile that gives up records
// an error and publishes anyway, so no CTA waits forever.
#include <algorithm>

#include "cb.h"
#include "cb_common.cuh"
#include "cb_kernels.h"

namespace cb {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kFE = 8;                // products per lane
constexpr int kFWarps = 8;            // warps per CTA
constexpr int kFThreads = kFWarps * 32;
constexpr unsigned kFPad = 0xFFFFFFFFu;
constexpr unsigned kFSpin = 1u << 20;  // polls of one earlier tile before giving up (~1 s)

// tile status word: [63:40] launch epoch (24 bits), [39:38] kind, [37:0] value
constexpr int kEpochShift = 40;
constexpr unsigned kEpochMask = (1u << 24) - 1;
constexpr unsigned long long kKindAgg = 1ull << 38;   // value = this tile's total
constexpr unsigned long long kKindInc = 2ull << 38;   // value = total of tiles 0..this
constexpr unsigned long long kKindMask = 3ull << 38;
constexpr unsigned long long kValMask = (1ull << 38) - 1;

constexpr int clog2(int x) { return x <= 1 ? 0 : 1 + clog2(x / 2); }

template <class T>
__device__ __forceinline__ T shfl_idx(T v, int src, int width) {
  if constexpr (sizeof(T) == 1) {
    return (T)__shfl_sync(kFull, (int)v, src, width);
  } else {
    return __shfl_sync(kFull, v, src, width);
  }
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

template <int SR, int G>
__global__ void __launch_bounds__(kFThreads) k_fused(DevCSR A, DevCSR B, int64_t* __restrict__ Crp,
                                                     int32_t* __restrict__ Ccol,
                                                     typename Sem<SR>::T* __restrict__ Cval,
                                                     int64_t cap, unsigned long long* tstat,
                                                     int64_t tstat_cap, unsigned* sync, int* status) {
  typedef Sem<SR> S;
  typedef typename S::A Acc;
  typedef typename S::T T;
  constexpr int F = G * kFE;            // products per row at most
  constexpr int LOGF = clog2(F);
  constexpr int RPW = 32 / G;           // rows per warp
  constexpr int TR = kFWarps * RPW;     // rows per tile
  __shared__ __align__(16) Acc sval[kFWarps][32 * kFE];
  __shared__ __align__(16) unsigned skey[kFWarps][32 * kFE];
  __shared__ int snz[TR];
  __shared__ long long soff[TR];
  __shared__ long long s_red[kFWarps];
  __shared__ int s_min[kFWarps];
  __shared__ long long s_base;
  __shared__ unsigned s_epoch, s_last;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / G, g = lane % G;
  const T* __restrict__ Aval = reinterpret_cast<const T*>(A.val);
  const T* __restrict__ Bval = reinterpret_cast<const T*>(B.val);
  Acc* sv = &sval[warp][grp * F];
  unsigned* sk = &skey[warp][grp * F];
  if (threadIdx.x == 0) s_epoch = *reinterpret_cast<volatile unsigned*>(sync) & kEpochMask;
  __syncthreads();
  const unsigned long long ep = (unsigned long long)s_epoch << kEpochShift;
  const int64_t ntiles = (A.nrows + TR - 1) / TR;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // ---- 1. the row's A entries and the product numbering
    const int64_t i = tile * TR + warp * RPW + grp;
    int64_t a0 = 0, a1 = 0;
    if (i < A.nrows) {
      a0 = A.rp[i];
      a1 = A.rp[i + 1];
    }
    const int64_t nA = a1 - a0;
    int64_t b0 = 0;
    T av = T();
    int len = 0;
    bool bad = nA > G;
    if (!bad && g < nA) {
      const int64_t p = a0 + g;
      const int k = A.col[p];
      if (S::kUsesA) av = Aval[p];
      b0 = B.rp[k];
      const int64_t bl = B.rp[k + 1] - b0;
      len = bl > F ? F + 1 : (int)bl;
    }
    int incl = len;
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, d, G);
      if (g >= d) incl += y;
    }
    int Fr = __shfl_sync(kFull, incl, G - 1, G);
    const int o = incl - len;  // first product of lane g's entry (Fr past the row's entries)
    bad = bad || Fr > F;
    if (bad) Fr = 0;

    // ---- 2. products: lane g takes t = r*G + g
    unsigned key[kFE];
#pragma unroll
    for (int r = 0; r < kFE; ++r) {
      const int t = r * G + g;
      int m = 0;  // largest lane with o_m <= t: the entry that owns product t
#pragma unroll
      for (int s = G / 2; s >= 1; s >>= 1) {
        const int om = __shfl_sync(kFull, o, m + s, G);
        if (om <= t) m += s;
      }
      const int om = __shfl_sync(kFull, o, m, G);
      const int64_t bq = __shfl_sync(kFull, b0, m, G);
      const T a = S::kUsesA ? shfl_idx(av, m, G) : T();
      key[r] = kFPad;
      if (t < Fr) {
        const int64_t q = bq + (t - om);
        key[r] = ((unsigned)B.col[q] << LOGF) | (unsigned)t;
        sv[t] = S::mul(a, Bval[q]);
      }
    }

    // ---- 3. sort the row's keys: element e = g*8 + r of a bitonic network
#pragma unroll
    for (int k = 2; k <= F; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j >= 1; j >>= 1) {
        if (j >= kFE) {
          const int lm = j / kFE;
          const bool asc = ((g * kFE) & k) == 0;
          const bool keep_min = ((g & lm) == 0) == asc;
#pragma unroll
          for (int r = 0; r < kFE; ++r) {
            const unsigned y = __shfl_xor_sync(kFull, key[r], lm);
            key[r] = keep_min ? min(key[r], y) : max(key[r], y);
          }
        } else {
#pragma unroll
          for (int r = 0; r < kFE; ++r) {
            if ((r & j) == 0) {
              const int r2 = r | j;
              const bool asc = k >= kFE ? ((g * kFE) & k) == 0 : (r & k) == 0;
              const unsigned lo = min(key[r], key[r2]), hi = max(key[r], key[r2]);
              key[r] = asc ? lo : hi;
              key[r2] = asc ? hi : lo;
            }
          }
        }
      }
    }

    // merge equal columns: a head is the first key of its column
    reinterpret_cast<uint4*>(sk)[g * 2] = make_uint4(key[0], key[1], key[2], key[3]);
    reinterpret_cast<uint4*>(sk)[g * 2 + 1] = make_uint4(key[4], key[5], key[6], key[7]);
    const unsigned prev_last = __shfl_up_sync(kFull, key[kFE - 1], 1, G);
    const unsigned next_first = __shfl_down_sync(kFull, key[0], 1, G);
    __syncwarp();
    unsigned heads = 0;
#pragma unroll
    for (int r = 0; r < kFE; ++r) {
      const unsigned c = key[r] >> LOGF;
      const unsigned pc = r == 0 ? (g == 0 ? kFPad : prev_last >> LOGF) : key[r - 1] >> LOGF;
      if (key[r] != kFPad && (c != pc || (r == 0 && g == 0))) heads |= 1u << r;
    }
    const int hc = __popc(heads);
    int hpos = hc;
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
      const int y = __shfl_up_sync(kFull, hpos, d, G);
      if (g >= d) hpos += y;
    }
    const int nz = __shfl_sync(kFull, hpos, G - 1, G);
    hpos -= hc;
    Acc hv[kFE];
#pragma unroll
    for (int r = 0; r < kFE; ++r) {
      hv[r] = S::ident();
      if (heads & (1u << r)) {
        const unsigned c = key[r] >> LOGF;
        Acc v = sv[key[r] & (F - 1)];
        const unsigned nc = (r + 1 < kFE ? key[r + 1 < kFE ? r + 1 : r] : next_first) >> LOGF;
        if (nc == c && (r + 1 < kFE || g + 1 < G)) {  // a run of equal columns: walk it
          for (int e2 = g * kFE + r + 1; e2 < F; ++e2) {
            const unsigned k2 = sk[e2];
            if ((k2 >> LOGF) != c) break;
            v = S::add(v, sv[k2 & (F - 1)]);
          }
        }
        hv[r] = v;
      }
    }
    __syncwarp();
    {
      int p = hpos;
#pragma unroll
      for (int r = 0; r < kFE; ++r) {
        if (heads & (1u << r)) {
          sk[p] = key[r] >> LOGF;
          sv[p] = hv[r];
          ++p;
        }
      }
    }
    if (g == 0) snz[warp * RPW + grp] = bad ? 0 : nz;
    if (bad && g == 0 && i < A.nrows) atomicOr(status, CB_FUSED_ROW_TOO_LARGE);
    __syncthreads();

    // ---- 4. tile offsets, publish, look back
    if (warp == 0) {
      const int v = lane < TR ? snz[lane] : 0;
      int inc = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += y;
      }
      if (lane < TR) soff[lane] = inc - v;
      const int agg = __shfl_sync(kFull, inc, 31);
      if (lane == 0) {
        s_red[0] = agg;
        atomicExch(&tstat[tile], ep | (tile == 0 ? kKindInc : kKindAgg) | (unsigned long long)agg);
      }
    }
    __syncthreads();
    const long long agg = s_red[0];
    long long excl = 0;
    for (int64_t top = tile - 1; top >= 0; top -= kFThreads) {
      const int64_t j = top - threadIdx.x;
      unsigned long long w = 0;
      bool inc_here = false;
      long long val = 0;
      if (j >= 0) {
        unsigned spins = 0;
        for (;;) {
          w = ld_volatile(&tstat[j]);
          if ((w & ~((1ull << kEpochShift) - 1)) == ep && (w & kKindMask)) break;
          if (++spins >= kFSpin) {
            atomicOr(status, CB_FUSED_STALLED);
            w = ep | kKindInc;
            break;
          }
        }
        inc_here = (w & kKindMask) == kKindInc;
        val = (long long)(w & kValMask);
      }
      // the nearest inclusive prefix in this window (smallest thread index)
      int first = inc_here ? (int)threadIdx.x : kFThreads;
      first = __reduce_min_sync(kFull, first);
      if (lane == 0) s_min[warp] = first;
      __syncthreads();
      int stop = kFThreads;
#pragma unroll
      for (int w8 = 0; w8 < kFWarps; ++w8) stop = min(stop, s_min[w8]);
      long long part = (j >= 0 && (int)threadIdx.x <= stop) ? val : 0;
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) part += __shfl_xor_sync(kFull, part, d);
      if (lane == 0) s_red[warp] = part;
      __syncthreads();
#pragma unroll
      for (int w8 = 0; w8 < kFWarps; ++w8) excl += s_red[w8];
      __syncthreads();
      if (stop < kFThreads) break;
    }
    if (threadIdx.x == 0) {
      if (tile > 0) atomicExch(&tstat[tile], ep | kKindInc | (unsigned long long)(excl + agg));
      s_base = excl;
    }
    __syncthreads();
    const long long base = s_base;

    // ---- 5. write the tile: row pointers, then each warp its rows
    if (threadIdx.x < TR) {
      const int64_t ir = tile * TR + threadIdx.x;
      if (ir < A.nrows) Crp[ir] = base + soff[threadIdx.x];
      if (ir == A.nrows - 1) Crp[A.nrows] = base + agg;
    }
    if (base + agg > cap) {
      if (threadIdx.x == 0) atomicOr(status, CB_FUSED_CAPACITY);
    } else {
#pragma unroll
      for (int rr = 0; rr < RPW; ++rr) {
        const int row = warp * RPW + rr;
        const int n = snz[row];
        const long long off = base + soff[row];
        const unsigned* rk = &skey[warp][rr * F];
        const Acc* rv = &sval[warp][rr * F];
        for (int t = lane; t < n; t += 32) {
          Ccol[off + t] = (int32_t)rk[t];
          Cval[off + t] = S::out(rv[t]);
        }
      }
    }
    __syncthreads();
  }

  // the last CTA to finish advances the epoch (clearing the status words
  // when the 24-bit epoch wraps, so that no stale word can match)
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&sync[1], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    const unsigned ne = (s_epoch + 1) & kEpochMask;
    if (ne == 0)
      for (int64_t j = threadIdx.x; j < tstat_cap; j += kFThreads) tstat[j] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
      sync[1] = 0;
      __threadfence();
      atomicExch(&sync[0], ne);
    }
  }
}

template <int SR, int G>
cudaError_t launch_fused_t(const DevCSR& A, const DevCSR& B, int64_t* Crp, int32_t* Ccol, void* Cval,
                           int64_t cap, unsigned long long* tstat, int64_t tstat_cap, unsigned* sync,
                           int* status, cudaStream_t s, int sms) {
  constexpr int TR = kFWarps * (32 / G);
  static int per_sm = 0;  // resident CTAs per SM (same for every device of one kind)
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<SR, G>, kFThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
  }
  const int64_t tiles = (A.nrows + TR - 1) / TR;
  if (tiles > tstat_cap) return cudaErrorInvalidValue;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)per_sm * sms);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kFThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fused<SR, G>, A, B, Crp, Ccol,
                            static_cast<typename Sem<SR>::T*>(Cval), cap, tstat, tstat_cap, sync,
                            status);
}

template <int SR>
cudaError_t launch_fused_sr(int lanes, const DevCSR& A, const DevCSR& B, int64_t* Crp, int32_t* Ccol,
                            void* Cval, int64_t cap, unsigned long long* tstat, int64_t tstat_cap,
                            unsigned* sync, int* status, cudaStream_t s, int sms) {
  switch (lanes) {
    case 8: return launch_fused_t<SR, 8>(A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms);
    case 16: return launch_fused_t<SR, 16>(A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms);
    case 32: return launch_fused_t<SR, 32>(A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int64_t fused_tiles(int lanes, int64_t nrows) {
  const int tr = kFWarps * (32 / lanes);
  return (nrows + tr - 1) / tr;
}

int64_t fused_max_cols(int lanes) { return (1ll << (32 - clog2(lanes * kFE))) - 1; }

cudaError_t launch_fused(int sr, int lanes, const DevCSR& A, const DevCSR& B, int64_t* Crp,
                         int32_t* Ccol, void* Cval, int64_t cap, unsigned long long* tstat,
                         int64_t tstat_cap, unsigned* sync, int* status, cudaStream_t s, int sms) {
  switch (sr) {
    case 1: return launch_fused_sr<1>(lanes, A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms);
    case 2: return launch_fused_sr<2>(lanes, A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms);
    case 3: return launch_fused_sr<3>(lanes, A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms);
    case 4: return launch_fused_sr<4>(lanes, A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms);
    case 5: return launch_fused_sr<5>(lanes, A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms);
  }
  return cudaErrorInvalidValue;
}

}  // namespace cb
