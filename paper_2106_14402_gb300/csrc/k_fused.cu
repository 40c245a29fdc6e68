// One-launch SpGEMM for products whose rows are all small: every row of A
// holds at most G entries and every output row at most 8G products
// (G = 8, 16 or 32 lanes per row).  The symbolic and numeric phases of the
// paper's row-wise SpGEMM (Sec. 4.1) collapse into one pass over the rows:
//
//   1. a group of G lanes takes one row; lane g loads A entry g and the
//      bounds of B row A.col[g]; a scan over the group numbers the row's
//      products t = 0..F-1;
//   2. the group's lanes read the B rows with coalesced loads and form up to
//      8 products each (product t's A entry is t / 8 when every such B row
//      has at most 8 entries, else a binary search over the group's scan
//      finds it); keys (column << log2(8G)) | t and products are staged in
//      shared memory and each lane takes 8 consecutive keys;
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
// an error and publishes anyway, so no CTA waits forever.  (spin_limit and
// silent_tile serve fault injection: a tile that never publishes.)
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

// Ascending sort of the G*8 keys of a lane group, element e = g*8 + r, by a
// bitonic network in the form where every comparator puts the minimum at the
// lower index: each merge of two sorted halves of size k/2 starts with a
// "flip" stage (e against e ^ (k-1)) and continues with half-cleaners
// (e against e ^ j, j = k/4 .. 1).  Partners within a lane are registers
// (compile-time indices), partners across lanes come by shuffle.  KSTART =
// 2*8 skips the merges inside a lane when every lane's 8 keys are already
// ascending.
template <int G, int KSTART>
__device__ __forceinline__ void bitonic_sort(unsigned (&key)[kFE], int g) {
  constexpr int F = G * kFE;
#pragma unroll
  for (int k = KSTART; k <= F; k <<= 1) {
    if (k <= kFE) {
#pragma unroll
      for (int r = 0; r < kFE; ++r)
        if ((r & (k >> 1)) == 0) {
          const int r2 = r ^ (k - 1);
          const unsigned lo = min(key[r], key[r2]), hi = max(key[r], key[r2]);
          key[r] = lo;
          key[r2] = hi;
        }
    } else {
      const int lm = k / kFE - 1;
      const bool lower = (g & (k / (2 * kFE))) == 0;
      unsigned y[kFE];
#pragma unroll
      for (int r = 0; r < kFE; ++r) y[r] = __shfl_xor_sync(kFull, key[kFE - 1 - r], lm);
#pragma unroll
      for (int r = 0; r < kFE; ++r) key[r] = lower ? min(key[r], y[r]) : max(key[r], y[r]);
    }
#pragma unroll
    for (int j = k >> 2; j >= 1; j >>= 1) {
      if (j < kFE) {
#pragma unroll
        for (int r = 0; r < kFE; ++r)
          if ((r & j) == 0) {
            const int r2 = r | j;
            const unsigned lo = min(key[r], key[r2]), hi = max(key[r], key[r2]);
            key[r] = lo;
            key[r2] = hi;
          }
      } else {
        const int lm = j / kFE;
        const bool lower = (g & lm) == 0;
#pragma unroll
        for (int r = 0; r < kFE; ++r) {
          const unsigned y = __shfl_xor_sync(kFull, key[r], lm);
          key[r] = lower ? min(key[r], y) : max(key[r], y);
        }
      }
    }
  }
}

template <int SR, int G>
__global__ void __launch_bounds__(kFThreads, 4) k_fused(DevCSR A, DevCSR B, int64_t* __restrict__ Crp,
                                                     int32_t* __restrict__ Ccol,
                                                     typename Sem<SR>::TC* __restrict__ Cval,
                                                     int64_t cap, unsigned long long* tstat,
                                                     int64_t tstat_cap, unsigned* sync, int* status,
                                                     unsigned spin_limit, int64_t silent_tile) {
  typedef Sem<SR> S;
  typedef typename S::A Acc;
  typedef typename S::TA TA;
  typedef typename S::TB TB;
  constexpr int F = G * kFE;            // products per row at most
  constexpr int LOGF = clog2(F);
  constexpr int RPW = 32 / G;           // rows per warp
  constexpr int TR = kFWarps * RPW;     // rows per tile
  __shared__ __align__(16) Acc sval[kFWarps][32 * kFE];
  __shared__ __align__(16) unsigned skey[kFWarps][32 * kFE];
  __shared__ int snz[TR];
  __shared__ int sfl[TR];  // products of each row of the tile
  __shared__ long long soff[TR];
  __shared__ long long s_red[kFWarps];
  __shared__ int s_min[kFWarps];
  __shared__ long long s_base;
  __shared__ unsigned s_epoch, s_last;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / G, g = lane % G;
  const TA* __restrict__ Aval = reinterpret_cast<const TA*>(A.val);
  const TB* __restrict__ Bval = reinterpret_cast<const TB*>(B.val);
  Acc* sv = &sval[warp][grp * F];
  unsigned* sk = &skey[warp][grp * F];
  // Bank swizzles of a row's shared arrays: entry t lives at t ^ h, h < 8,
  // chosen so that the 32 lanes of a warp storing entry 8b + r of their own
  // block b (or reading 32 consecutive entries of one row) spread over all
  // banks: 8-byte values over 16 bank pairs twice, 4-byte keys over 32 banks.
  const auto pv = [grp](int t) { return t ^ (((t >> 4) | grp * (G / 2)) & 7); };
  const auto pk = [grp](int t) { return t ^ (((t >> 5) | grp * (G / 4)) & 7); };
  // the launch epoch is read now and shared at the first tile's publication,
  // off the critical path of the first loads
  unsigned epoch0 = 0;
  if (threadIdx.x == 0) epoch0 = *reinterpret_cast<volatile unsigned*>(sync) & kEpochMask;
  unsigned long long ep = 0;
  const int64_t ntiles = (A.nrows + TR - 1) / TR;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // ---- 1. the row's A entries and the product numbering
    const int64_t i = tile * TR + warp * RPW + grp;
    int64_t a0 = 0, a1 = 0;
    if (i < A.nrows) {
      a0 = __ldg(A.rp + i);
      a1 = __ldg(A.rp + i + 1);
    }
    const int64_t nA = a1 - a0;
    int64_t b0 = 0;
    TA av = TA();
    int len = 0;
    bool bad = nA > G;
    if (!bad && g < nA) {
      const int64_t p = a0 + g;
      const int k = __ldg(A.col + p);
      if (S::kUsesA) av = ldg_val(Aval + p);
      b0 = __ldg(B.rp + k);
      const int64_t bl = __ldg(B.rp + k + 1) - b0;
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

    // ---- 2. products, numbered t < 8G and formed by lanes that read B rows
    // with coalesced loads (lane g, register r takes slot r*G + g).  Fast form
    // (every entry's B row holds <= 8 entries): t = entry*8 + element, so the
    // slot needs no search.  General form: t is the product's rank in the row
    // and a binary search over the group's scan finds its A entry.  Keys
    // (column << log2(8G) | t) and products go to shared memory; lane g then
    // takes keys g*8 .. g*8+7 (entry g's B row in the fast form, already
    // ascending when B's rows are sorted).
    const bool fast = __all_sync(kFull, bad || len <= kFE);
#pragma unroll
    for (int r = 0; r < kFE; ++r) {
      const int t = r * G + g;
      int m, first;
      bool valid;
      if (fast) {
        m = t >> 3;
        first = t & ~7;
        const int lm = __shfl_sync(kFull, len, m, G);  // every lane shuffles
        valid = !bad && (t & 7) < lm;
      } else {
        m = 0;  // largest lane with o_m <= t: the entry that owns product t
#pragma unroll
        for (int s2 = G / 2; s2 >= 1; s2 >>= 1) {
          const int om = __shfl_sync(kFull, o, m + s2, G);
          if (om <= t) m += s2;
        }
        first = __shfl_sync(kFull, o, m, G);
        valid = t < Fr;
      }
      const int64_t bq = __shfl_sync(kFull, b0, m, G);
      const TA a = S::kUsesA ? shfl_idx(av, m, G) : TA();
      unsigned kt = kFPad;
      if (valid) {
        const int64_t q = bq + (t - first);
        kt = ((unsigned)__ldg(B.col + q) << LOGF) | (unsigned)t;
        sv[pv(t)] = S::mul(a, ldg_val(Bval + q));
      }
      sk[pk(t)] = kt;
    }
    __syncwarp();
    unsigned key[kFE];
#pragma unroll
    for (int r = 0; r < kFE; ++r) key[r] = sk[pk(g * kFE + r)];

    // ---- 3. sort the row's keys (lanes whose 8 keys are already ascending --
    // sorted B rows in the fast form -- skip the in-lane merges)
    bool run_sorted = true;
#pragma unroll
    for (int r = 0; r + 1 < kFE; ++r) run_sorted = run_sorted && key[r] <= key[r + 1];
    if (__all_sync(kFull, run_sorted)) bitonic_sort<G, 2 * kFE>(key, g);
    else bitonic_sort<G, 2>(key, g);

    // merge equal columns: a head is the first key of its column
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kFE; ++r) sk[pk(g * kFE + r)] = key[r];
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
        Acc v = sv[pv(key[r] & (F - 1))];
        const unsigned nc = (r + 1 < kFE ? key[r + 1 < kFE ? r + 1 : r] : next_first) >> LOGF;
        if (nc == c && (r + 1 < kFE || g + 1 < G)) {  // a run of equal columns: walk it
          for (int e2 = g * kFE + r + 1; e2 < F; ++e2) {
            const unsigned k2 = sk[pk(e2)];
            if ((k2 >> LOGF) != c) break;
            v = S::add(v, sv[pv(k2 & (F - 1))]);
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
          sk[pk(p)] = key[r] >> LOGF;
          sv[pv(p)] = hv[r];
          ++p;
        }
      }
    }
    if (g == 0) {
      snz[warp * RPW + grp] = bad ? 0 : nz;
      sfl[warp * RPW + grp] = Fr;
    }
    if (bad && g == 0 && i < A.nrows) atomicOr(status, CB_FUSED_ROW_TOO_LARGE);
    if (threadIdx.x == 0 && tile == blockIdx.x) s_epoch = epoch0;
    __syncthreads();
    ep = (unsigned long long)s_epoch << kEpochShift;

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
      // the tile's product count joins the launch's total (sync[8..9])
      const int tf = __reduce_add_sync(kFull, lane < TR ? sfl[lane] : 0);
      if (lane == 0 && tf) atomicAdd(reinterpret_cast<unsigned long long*>(sync + 8), (unsigned long long)tf);
      if (lane == 0) {
        s_red[0] = agg;
        if (tile != silent_tile)  // fault injection: a producer that never publishes
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
          if (++spins >= spin_limit) {
            atomicOr(status, CB_FUSED_STALLED);
            w = ep | kKindInc;
            break;
          }
          __nanosleep(40);  // leave issue slots to the CTAs still computing
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
      if (tile > 0 && tile != silent_tile)
        atomicExch(&tstat[tile], ep | kKindInc | (unsigned long long)(excl + agg));
      s_base = excl;
    }
    __syncthreads();
    const long long base = s_base;

    // ---- 5. write the tile: row pointers, then each warp its rows
    if (threadIdx.x < TR) {
      const int64_t ir = tile * TR + threadIdx.x;
      if (ir < A.nrows) Crp[ir] = base + soff[threadIdx.x];
      if (ir == A.nrows - 1) {
        Crp[A.nrows] = base + agg;
        __threadfence();  // before this CTA counts itself finished
      }
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
        if (!chk(off + n <= cap && n <= F, 46, off + n)) continue;
        for (int t = lane; t < n; t += 32) {
          Ccol[off + t] = (int32_t)rk[t ^ (((t >> 5) | rr * (G / 4)) & 7)];
          Cval[off + t] = S::out(rv[t ^ (((t >> 4) | rr * (G / 2)) & 7)]);
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
    // totals of the launch for the host: nnz(C) (sync[2..3]) and the
    // product count (sync[6..7]); the product accumulator restarts at 0
    if (threadIdx.x == 0) {
      __threadfence();
      unsigned long long* s64 = reinterpret_cast<unsigned long long*>(sync);
      s64[1] = (unsigned long long)*reinterpret_cast<volatile int64_t*>(Crp + A.nrows);
      s64[3] = atomicExch(s64 + 4, 0ull);
    }
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
                           int* status, cudaStream_t s, int sms, unsigned spin_limit,
                           int64_t silent_tile) {
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
                            static_cast<typename Sem<SR>::TC*>(Cval), cap, tstat, tstat_cap, sync,
                            status, spin_limit < 1 ? 1u : spin_limit, silent_tile);
}

template <int SR>
cudaError_t launch_fused_sr(int lanes, const DevCSR& A, const DevCSR& B, int64_t* Crp, int32_t* Ccol,
                            void* Cval, int64_t cap, unsigned long long* tstat, int64_t tstat_cap,
                            unsigned* sync, int* status, cudaStream_t s, int sms, unsigned spin,
                            int64_t silent) {
  switch (lanes) {
    case 8: return launch_fused_t<SR, 8>(A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms, spin, silent);
    case 16: return launch_fused_t<SR, 16>(A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms, spin, silent);
    case 32: return launch_fused_t<SR, 32>(A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms, spin, silent);
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
                         int64_t tstat_cap, unsigned* sync, int* status, cudaStream_t s, int sms,
                         unsigned spin_limit, int64_t silent_tile) {
  switch (sr) {
#define CB_CASE(SRV) case SRV: return launch_fused_sr<SRV>(lanes, A, B, Crp, Ccol, Cval, cap, tstat, tstat_cap, sync, status, s, sms, spin_limit, silent_tile);
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
  }
  return cudaErrorInvalidValue;
}

CB_CHECK_READER(fused)

}  // namespace cb
