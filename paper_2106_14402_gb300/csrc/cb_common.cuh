// Device-side building blocks shared by the SpGEMM kernels: semiring
// traits, the shared-memory hash probe, team synchronisation and the
// tier limits that the host dispatcher and the kernels agree on.
#pragma once

#include <cstdint>
#include <climits>
#include <type_traits>
#include <cuda_runtime.h>

#include "cb_kernels.h"

namespace cb {

// ---------------------------------------------------------------------------
// Semirings (paper Sec. 1: user-defined (+) and (x) over up to three value
// types, two for the inputs and one for the output).  A semiring is one
// specialisation of Sem<SR> with
//   TA, TB  value types of A's and B's CSR arrays, TC of C's;
//   A       accumulator type (shared memory or L2), with ident() the
//           (+)-identity, mul(TA, TB) -> A the (x), add and atomic the (+),
//           out(A) -> TC the conversion of a finished entry;
//   kUsesA  false when (x) ignores A's value (A's values are not read);
// plus one entry in CB_FOR_EACH_SEMIRING and the value sizes in cb_api.cu.
// Every (+) here is commutative and associative on A, so products may be
// combined in any order with atomics; for fp64 that changes rounding only.
// ---------------------------------------------------------------------------
#define CB_FOR_EACH_SEMIRING(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7)

// ---------------------------------------------------------------------------
// Debug build (compiled with -DCB_CHECK, library libcb_check.so): the index
// of every CSR write and of every shared or global hash-table access is
// checked at run time.  A failed check records (code, index) in the check
// word of its translation unit (the first failure wins) and the access is
// skipped, so nothing is written out of bounds; the host reads the words
// after every call and fails it (CB_ERR_CUDA, "bounds check ...").  In the
// normal build chk() is constant true and guard() is the plain condition.
// ---------------------------------------------------------------------------
#ifdef CB_CHECK
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

namespace {
__device__ unsigned long long g_check_word[2];  // (code, index), one per translation unit
}

__device__ __forceinline__ void check_record(int code, int64_t index) {
  if (atomicCAS(&g_check_word[0], 0ull, (unsigned long long)code) == 0ull)
    g_check_word[1] = (unsigned long long)index;
}

// A check that only the debug build makes: true in the normal build.
__device__ __forceinline__ bool chk(bool ok, int code, int64_t index) {
  if constexpr (kChecked) {
    if (!ok) check_record(code, index);
    return ok;
  } else {
    return true;
  }
}

// A bound every build keeps (the access is skipped when it fails); the
// debug build also records the failure.
__device__ __forceinline__ bool guard(bool ok, int code, int64_t index) {
  if constexpr (kChecked) {
    if (!ok) check_record(code, index);
  }
  return ok;
}

// Host side, one per translation unit that includes this header: reads and
// clears the unit's check word on stream s (synchronises).  Returns the
// code (0: no failure) and the index in *index.  Always 0 in the normal build.
#define CB_CHECK_READER(NAME)                                                              \
  int64_t check_take_##NAME(cudaStream_t s, int64_t* index) {                              \
    *index = 0;                                                                            \
    if constexpr (!kChecked) {                                                             \
      return 0;                                                                            \
    } else {                                                                               \
      unsigned long long w[2] = {0, 0};                                                    \
      if (cudaMemcpyFromSymbolAsync(w, g_check_word, sizeof w, 0, cudaMemcpyDeviceToHost,  \
                                    s) != cudaSuccess)                                     \
        return -1;                                                                         \
      const unsigned long long z[2] = {0, 0};                                              \
      if (cudaMemcpyToSymbolAsync(g_check_word, z, sizeof z, 0, cudaMemcpyHostToDevice,    \
                                  s) != cudaSuccess ||                                     \
          cudaStreamSynchronize(s) != cudaSuccess)                                         \
        return -1;                                                                         \
      *index = (int64_t)w[1];                                                              \
      return (int64_t)w[0];                                                                \
    }                                                                                      \
  }

template <int SR> struct Sem;

// Read-only cached load of a value of any semiring type: integer types
// directly; floating-point values and 8-byte records (cb_wlabel) as their
// bits (an unsigned word of the same size), so that every bit pattern, NaN
// payloads included, arrives unchanged (a float load through __ldg lost NaN
// weights of the heterogeneous semiring).
template <class T>
__device__ __forceinline__ T ldg_val(const T* p) {
  if constexpr (std::is_integral<T>::value) {
    return __ldg(p);
  } else {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "values are 4 or 8 bytes");
    typedef typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned>::type U;
    const U u = __ldg(reinterpret_cast<const U*>(p));
    T r;
    memcpy(&r, &u, sizeof r);
    return r;
  }
}

// Store of a value written once and not read again by the kernel (C's
// entries, stored bitmaps): with kStreamOut an evict-first store, so that the
// output streaming through L2 does not push out the operands being gathered.
constexpr bool kStreamOut = true;
template <class T>
__device__ __forceinline__ void st_out(T* p, T v) {
  if constexpr (!kStreamOut) {
    *p = v;
  } else if constexpr (sizeof(T) == 8) {
    unsigned long long u;
    memcpy(&u, &v, sizeof u);
    __stcs(reinterpret_cast<unsigned long long*>(p), u);
  } else if constexpr (sizeof(T) == 4) {
    unsigned u;
    memcpy(&u, &v, sizeof u);
    __stcs(reinterpret_cast<unsigned*>(p), u);
  } else {
    static_assert(sizeof(T) == 1, "values of 1, 4 or 8 bytes");
    unsigned char u;
    memcpy(&u, &v, sizeof u);
    __stcs(reinterpret_cast<unsigned char*>(p), u);
  }
}

template <> struct Sem<1> {  // (+,x) over int64, wrapping
  typedef int64_t TA, TB, TC;
  typedef unsigned long long A;
  static constexpr bool kUsesA = true;
  __device__ static __forceinline__ A ident() { return 0ull; }
  __device__ static __forceinline__ A mul(TA a, TB b) { return (A)a * (A)b; }
  __device__ static __forceinline__ A add(A x, A y) { return x + y; }
  __device__ static __forceinline__ void atomic(A* p, A v) { atomicAdd(p, v); }
  __device__ static __forceinline__ TC out(A x) { return (TC)x; }
};

template <> struct Sem<2> {  // (+,x) over fp64
  typedef double TA, TB, TC;
  typedef double A;
  static constexpr bool kUsesA = true;
  __device__ static __forceinline__ A ident() { return 0.0; }
  __device__ static __forceinline__ A mul(TA a, TB b) { return __dmul_rn(a, b); }
  __device__ static __forceinline__ A add(A x, A y) { return __dadd_rn(x, y); }
  __device__ static __forceinline__ void atomic(A* p, A v) { atomicAdd(p, v); }
  __device__ static __forceinline__ TC out(A x) { return x; }
};

template <> struct Sem<3> {  // (min,+) over uint32, + saturating at UINT32_MAX
  typedef uint32_t TA, TB, TC;
  typedef unsigned A;
  static constexpr bool kUsesA = true;
  __device__ static __forceinline__ A ident() { return 0xFFFFFFFFu; }
  __device__ static __forceinline__ A mul(TA a, TB b) {
    unsigned s = a + b;
    return s < a ? 0xFFFFFFFFu : s;
  }
  __device__ static __forceinline__ A add(A x, A y) { return x < y ? x : y; }
  __device__ static __forceinline__ void atomic(A* p, A v) { atomicMin(p, v); }
  __device__ static __forceinline__ TC out(A x) { return x; }
};

template <> struct Sem<4> {  // (or,and) over bool (uint8 storage)
  typedef uint8_t TA, TB, TC;
  typedef unsigned A;
  static constexpr bool kUsesA = true;
  __device__ static __forceinline__ A ident() { return 0u; }
  __device__ static __forceinline__ A mul(TA a, TB b) { return (a != 0 && b != 0) ? 1u : 0u; }
  __device__ static __forceinline__ A add(A x, A y) { return x | y; }
  __device__ static __forceinline__ void atomic(A* p, A v) { if (v) atomicOr(p, v); }
  __device__ static __forceinline__ TC out(A x) { return x ? 1 : 0; }
};

template <> struct Sem<5> {  // (select2nd,min) over int32
  typedef int32_t TA, TB, TC;
  typedef int A;
  static constexpr bool kUsesA = false;
  __device__ static __forceinline__ A ident() { return INT_MAX; }
  __device__ static __forceinline__ A mul(TA, TB b) { return b; }
  __device__ static __forceinline__ A add(A x, A y) { return x < y ? x : y; }
  __device__ static __forceinline__ void atomic(A* p, A v) { atomicMin(p, v); }
  __device__ static __forceinline__ TC out(A x) { return x; }
};

// Heterogeneous (paper Sec. 1: three value types): A holds fp32 edge weights,
// B int32 labels, C (weight, label) pairs.  (x)(w, l) = (w, l); (+) keeps the
// pair with the larger weight in IEEE 754 totalOrder (-NaN < -inf < ... <
// -0 < +0 < ... < +inf < +NaN), and of equal weights the smaller label.  So
// C(i,j) is the label B(k,j) reached through the heaviest edge A(i,k).
// The accumulator packs both into one 64-bit key whose unsigned order is
// that order: high word = the weight's bits mapped monotonically (sign bit
// set: all bits flipped; clear: the sign bit flipped), low word =
// 0x7FFFFFFF - label (mod 2^32), which decreases with the label.
struct WLabel {
  float w;
  int32_t label;
};
template <> struct Sem<6> {
  typedef float TA;
  typedef int32_t TB;
  typedef WLabel TC;
  typedef unsigned long long A;
  static constexpr bool kUsesA = true;
  __device__ static __forceinline__ A ident() { return 0ull; }
  __device__ static __forceinline__ A mul(TA a, TB b) {
    const unsigned u = __float_as_uint(a);
    const unsigned hi = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    const unsigned lo = 0x7FFFFFFFu - (unsigned)b;
    return ((A)hi << 32) | lo;
  }
  __device__ static __forceinline__ A add(A x, A y) { return x > y ? x : y; }
  __device__ static __forceinline__ void atomic(A* p, A v) { atomicMax(p, v); }
  __device__ static __forceinline__ TC out(A x) {
    const unsigned hi = (unsigned)(x >> 32), lo = (unsigned)x;
    TC r;
    r.w = __uint_as_float((hi & 0x80000000u) ? (hi & 0x7FFFFFFFu) : ~hi);
    r.label = (int32_t)(0x7FFFFFFFu - lo);
    return r;
  }
  // the accumulator of a finished entry (used by the merge form below)
  __device__ static __forceinline__ A in(TC v) { return mul(v.w, v.label); }
};

// Merge form of Sem<6> (internal, not an ABI semiring): the selector product
// that (+)-combines partial results of Sem<6> has B and C of Sem<6>'s C
// type; (x)(selector, c) = c and (+) is Sem<6>'s.
template <> struct Sem<7> {
  typedef uint8_t TA;
  typedef WLabel TB, TC;
  typedef unsigned long long A;
  static constexpr bool kUsesA = false;
  __device__ static __forceinline__ A ident() { return Sem<6>::ident(); }
  __device__ static __forceinline__ A mul(TA, TB b) { return Sem<6>::in(b); }
  __device__ static __forceinline__ A add(A x, A y) { return Sem<6>::add(x, y); }
  __device__ static __forceinline__ void atomic(A* p, A v) { Sem<6>::atomic(p, v); }
  __device__ static __forceinline__ TC out(A x) { return Sem<6>::out(x); }
};

// ---------------------------------------------------------------------------
// Tier limits.  Symbolic tiers are chosen by u_i = min(flops_i, ncols) (an
// upper bound of nnz(C_i)); numeric tiers by the exact nnz(C_i).
//   * u <= 512: counted with a shared-memory hash table (warp or 256-thread
//     team); u > 512: counted with a dense bitmap per span of kSpanCols
//     columns, which also cuts the row into rank windows (below).
//   * nnz <= 512: numeric in a shared-memory hash table + bitonic sort;
//     nnz > 512: numeric per rank window.  Every such row has u > 512, so its
//     windows exist.
// A rank window is a run of whole bitmap words of one span holding at most
// NumLimits<SR>::kWcap output entries; inside it an output column's slot is
// its rank (popcount of the set bits before it), so a dense array of kWcap
// accumulators indexed by rank holds the window and reads out sorted.
// ---------------------------------------------------------------------------
constexpr int kEmptyKey = -1;

constexpr int kSymWarpMax = 128;     // warp team, table <= 256 slots
constexpr int kSymSmallMax = 512;    // 256-thread team, table <= 1024
constexpr int kSymHashMax = 512;     // default bound of the hash tiers (runtime-tunable)
constexpr int kSymLargeMax = 4096;   // largest bound the 1024-thread hash tier supports
constexpr int kSpanCols = 1 << 18;   // columns per bitmap span
constexpr int kSpanWords = kSpanCols / 32;
constexpr int kMaxWindowsPerSpan = 64;

constexpr int kNumWarpMax = 64;      // warp team, table <= 128
constexpr int kNumSmallMax = 512;    // 256-thread team, table <= 1024
template <int SR> struct NumLimits {
  static constexpr int kHashMax = kNumSmallMax;  // default bound of the hash tiers
  // largest bound the large hash tier supports (512-thread team, table of 2x slots)
  static constexpr int kLargeMax = 4096;
  // accumulators per rank window
  static constexpr int kWcap = sizeof(typename Sem<SR>::A) == 8 ? 16384 : 32768;
  // window cut: a window starts where the running count crosses a multiple
  // of kWcut, so it holds at most kWcut + 31 <= kWcap entries
  static constexpr int kWcut = kWcap - 32;
  // learned sizing: rows predicted to hold at most this many entries skip the
  // symbolic phase and are computed in one pass in a hash table of
  // 2^ceil(log2(2 cap)) slots (1024-thread team at most)
  static constexpr int kLearnHashMax = kLargeMax;
  // rank windows of 8-byte accumulators reduce into a per-CTA slice in L2
  // instead of shared memory (measured faster for int64 and fp64; slower for
  // the 4-byte ones, whose shared-memory atomics are cheap)
  static constexpr bool kL2Acc = sizeof(typename Sem<SR>::A) == 8;
};

// One rank window of a heavy row: row index h into the heavy-row list, the
// span, the word range [w_lo, w_hi) inside the span, its entry count and the
// rank of its first entry within the span.
struct Window {
  int32_t h, span, w_lo, w_hi, count, rank;
};

// Popcounts of the WPT consecutive bitmap words first .. first + WPT - 1 of
// a shared-memory bitmap (first a multiple of WPT, bits 16-byte aligned),
// words at or past nw counted as 0.  A thread's words are consecutive, so a
// load of one word per thread would put a warp's lanes 4*WPT bytes apart on
// a few banks (a WPT-way bank conflict); 16-byte loads of 4 words each take
// a quarter of the shared-memory wavefronts.
template <int WPT>
__device__ __forceinline__ void popc_words(const unsigned* bits, int first, int nw, int (&c)[WPT]) {
  static_assert(WPT % 4 == 0, "whole 16-byte vectors per thread");
  const uint4* v = reinterpret_cast<const uint4*>(bits + first);
#pragma unroll
  for (int q = 0; q < WPT / 4; ++q) {
    const int w = first + 4 * q;
    const uint4 x = w < nw ? v[q] : make_uint4(0u, 0u, 0u, 0u);
    c[4 * q + 0] = __popc(x.x);
    c[4 * q + 1] = w + 1 < nw ? __popc(x.y) : 0;
    c[4 * q + 2] = w + 2 < nw ? __popc(x.z) : 0;
    c[4 * q + 3] = w + 3 < nw ? __popc(x.w) : 0;
  }
}

// The running counts before each of those words, as 16-bit values (a
// window holds fewer than 2^16 entries), stored 8 per 16-byte vector:
// pre[first + j] = run + c[0] + ... + c[j - 1].  Vectors wholly past nw are
// not stored; counts past nw inside a stored vector are never read.
template <int WPT>
__device__ __forceinline__ void store_counts(unsigned short* pre, int first, int nw, int run,
                                             const int (&c)[WPT]) {
  static_assert(WPT % 8 == 0, "whole 16-byte vectors per thread");
  uint4* v = reinterpret_cast<uint4*>(pre + first);
#pragma unroll
  for (int q = 0; q < WPT / 8; ++q) {
    unsigned p[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const unsigned lo16 = (unsigned)run & 0xFFFFu;
      run += c[8 * q + 2 * h];
      const unsigned hi16 = (unsigned)run & 0xFFFFu;
      run += c[8 * q + 2 * h + 1];
      p[h] = lo16 | (hi16 << 16);
    }
    if (first + 8 * q < nw) v[q] = make_uint4(p[0], p[1], p[2], p[3]);
  }
}

// The set bits of a column bitmap, read out in column order: word w covers
// columns 32w .. 32w + 31 of the range, pre[w] counts the set bits of the
// words before it, and emit(j, c) receives the j-th set bit overall (c its
// column offset in the range), every j once.  Two walks, picked by the
// average number of set bits per word:
//   * dense (at least DENSE per word, DENSE > 0): one word per warp step; lane
//     l takes bit l, at the word's offset plus the bits set below it, so the
//     entries of one store instruction are consecutive (one or two L2
//     requests for up to 32 entries);
//   * sparse: one word per thread, its bits in turn.  A lane's entries are
//     consecutive and the lanes' words start a few entries apart.
// Walking a dense bitmap a word per thread places the 32 lanes' entries of
// one store a word's count apart, one L2 request per entry.
// The dense walk pays for that only where the kernel is bound by its
// requests to L2 (rank windows reducing in L2: R-MAT s18 fp64 numeric 55.7 ->
// 54.5 ms); where shared-memory accumulators bound it, its extra
// instructions and broadcast loads cost as much as they save (u32 and bool
// numeric unchanged at a bound of 8, 2-4 ms slower at 4), so those kernels
// pass DENSE = 0.
#ifndef CB_DENSE_WORD_BITS
#define CB_DENSE_WORD_BITS 8
#endif
constexpr int kDenseWordBits = CB_DENSE_WORD_BITS;
template <int DENSE, int CTA, class F>
__device__ __forceinline__ void for_bitmap_columns(const unsigned* bits, const unsigned short* pre,
                                                   int nw, int cnt, F&& emit) {
  const int tid = threadIdx.x;
  if (DENSE > 0 && (int64_t)cnt >= (int64_t)DENSE * nw) {  // uniform over the CTA
    const int lane = tid & 31;
    const unsigned below = (1u << lane) - 1u;
    for (int w = tid >> 5; w < nw; w += CTA / 32) {
      const unsigned word = bits[w];
      if ((word >> lane) & 1u) emit((int)pre[w] + __popc(word & below), 32 * w + lane);
    }
  } else {
    for (int w = tid; w < nw; w += CTA) {
      unsigned word = bits[w];
      int j = pre[w];
      while (word) {
        const int b = __ffs(word) - 1;
        word &= word - 1;
        emit(j, 32 * w + b);
        ++j;
      }
    }
  }
}

enum SymTier { kSymEmpty = 0, kSymWarp = 1, kSymSmall = 2, kSymLarge = 3, kSymHeavy = 4, kSymTiers = 5 };
enum NumTier { kNumEmpty = 0, kNumWarp = 1, kNumSmall = 2, kNumLarge = 3, kNumHeavy = 4, kNumTiers = 5 };

__device__ __forceinline__ int sym_tier(int64_t u, int64_t hash_max) {
  return u == 0 ? kSymEmpty : u <= kSymWarpMax ? kSymWarp : u <= kSymSmallMax ? kSymSmall
         : u <= hash_max ? kSymLarge : kSymHeavy;
}


// Smallest power of two >= x (x >= 1), as log2.
__host__ __device__ __forceinline__ int ceil_log2(int64_t x) {
  int l = 0;
  while ((int64_t(1) << l) < x) ++l;
  return l;
}

// Fibonacci hashing into a table of 2^bits slots (bits in [1, 31]).
__device__ __forceinline__ uint32_t hash_slot(int32_t c, int shift) {
  return ((uint32_t)c * 2654435769u) >> shift;
}

// Find the slot of key c in an open-addressing (linear probing) table of
// mask+1 slots, inserting it if absent.  Returns the slot, or -1 if the
// table is full (never happens for tables sized >= 2x the row bound).
// `inserted` reports whether this call created the key.
__device__ __forceinline__ int probe_insert(int* keys, uint32_t mask, int shift, int c,
                                           bool& inserted) {
  uint32_t s = hash_slot(c, shift);
  inserted = false;
  for (uint32_t n = 0; n <= mask; ++n) {
    int k = *(volatile int*)&keys[s];
    if (k == c) return (int)s;
    if (k == kEmptyKey) {
      int old = atomicCAS(&keys[s], kEmptyKey, c);
      if (old == kEmptyKey) { inserted = true; return (int)s; }
      if (old == c) return (int)s;
    }
    s = (s + 1) & mask;
  }
  return -1;
}

template <int TEAM>
__device__ __forceinline__ void team_sync() {
  if (TEAM == 32) __syncwarp();
  else __syncthreads();
}

// Group size (lanes per stored A entry) for a row: the power of two nearest
// below the mean B-row length, clamped to [1, TEAM_MAX].
template <int TEAM_MAX>
__device__ __forceinline__ int group_log2(int64_t flops, int64_t nnz_a) {
  if (nnz_a <= 0) return 0;
  int64_t avg = flops / nnz_a;
  int g = 0;
  while (g < 5 && (int64_t(2) << g) <= avg) ++g;
  int lim = TEAM_MAX >= 32 ? 5 : ceil_log2(TEAM_MAX);
  return g < lim ? g : lim;
}

// End offset of row k of a (possibly windowed) operand.
__device__ __forceinline__ int64_t row_end(const DevCSR& M, int64_t k) {
  return M.rpe ? M.rpe[k] : M.rp[k + 1];
}

// Output width of row i of A.B: A.rcols[i] when set (stacked batches, where
// each product keeps its own columns), else the width of B's view.
__device__ __forceinline__ int64_t row_width(const DevCSR& A, const DevCSR& B, int64_t i) {
  return A.rcols ? (int64_t)A.rcols[i] : B.ncols;
}

// Whether column c belongs to B's column window (always true unless filtering).
__device__ __forceinline__ bool in_window(const DevCSR& B, int c) {
  return !B.filter || (uint64_t)((int64_t)c - B.col_lo) < (uint64_t)B.ncols;
}

// Lane layout of a group of G = 2^gl lanes inside a warp (G <= 32).
struct Group {
  int G, gq, shift;
  unsigned mask;
  __device__ __forceinline__ Group(int gl, int thread) {
    G = 1 << gl;
    gq = thread & (G - 1);
    shift = (thread & 31) & ~(G - 1);
    mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << shift);
  }
  // ballot of the group's lanes, as G low bits
  __device__ __forceinline__ unsigned ballot(bool pred) const {
    return (__ballot_sync(mask, pred) & mask) >> shift;
  }
};

// First index in the sorted run col[q0, q1) whose column is >= x, found
// cooperatively by a lane group: each round lane j probes the (j+1)-th of
// G+1 equal cut points, and the number of probes below x narrows the run by
// a factor of about G+1.  Every lane of the group must call it.
__device__ __forceinline__ int64_t group_lower_bound(const int32_t* col, int64_t q0, int64_t q1,
                                                     int64_t x, const Group& g) {
  int64_t lo = q0, hi = q1;  // the answer lies in [lo, hi]
  while (hi - lo > g.G) {
    const int64_t len = hi - lo;
    const int64_t pos = lo + (len * (g.gq + 1)) / (g.G + 1);
    const int t = __popc(g.ballot((int64_t)col[pos] < x));
    const int64_t nlo = t > 0 ? lo + (len * t) / (g.G + 1) + 1 : lo;
    const int64_t nhi = t < g.G ? lo + (len * (t + 1)) / (g.G + 1) : hi;
    lo = nlo;
    hi = nhi;
  }
  const int64_t pos = lo + g.gq;
  return lo + __popc(g.ballot(pos < hi && (int64_t)col[pos] < x));
}

// Visit every product A(i,p) * B(p,q) of row i whose column lies in
// [lo, hi) (absolute columns): f(p, q, c) is called by the lane that owns
// it.  Lanes form groups of 2^gl per stored A entry (a team of TEAM
// threads, `thread` in [0, TEAM)).  `whole` means every entry of B's rows
// lies in [lo, hi) (no filter); `sorted` means B's rows are non-decreasing
// in column, so each B row's slice in [lo, hi) is located by a group search
// and walked to its end; otherwise whole B rows are read and filtered.
// Uniform per team.
template <int TEAM, class F>
__device__ __forceinline__ void for_row_products(const DevCSR& A, const DevCSR& B, int64_t i,
                                                 int64_t lo, int64_t hi, bool whole, bool sorted,
                                                 int gl, int thread, F&& f) {
  const Group g(gl, thread);
  const int groups = TEAM >> gl;
  const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
  const unsigned width = (unsigned)(hi - lo);
  if (whole || !sorted) {
    for (int64_t p = a0 + (thread >> gl); p < a1; p += groups) {
      const int k = A.col[p];
      const int64_t q1 = row_end(B, k);
      for (int64_t q = B.rp[k] + g.gq; q < q1; q += g.G) {
        const int c = B.col[q];
        if (whole || (unsigned)((int64_t)c - lo) < width) f(p, q, c);
      }
    }
    return;
  }
  for (int64_t p = a0 + (thread >> gl); p < a1; p += groups) {
    const int k = A.col[p];
    const int64_t q1 = row_end(B, k);
    int64_t q = group_lower_bound(B.col, B.rp[k], q1, lo, g);
    while (true) {
      const int64_t qq = q + g.gq;
      const int c = qq < q1 ? B.col[qq] : INT_MAX;
      const bool in = (int64_t)c < hi;
      const int n = __popc(g.ballot(in));
      if (in) f(p, qq, c);
      if (n < g.G) break;
      q += g.G;
    }
  }
}

// Exclusive scan of one int per thread across a team of TEAM threads.
template <int TEAM>
__device__ __forceinline__ int team_exclusive_scan(int x, int* scratch /* >= 33 ints */, int& total) {
  const int lane = threadIdx.x & 31;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (TEAM == 32) {
    total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - x;
  }
  const int w = threadIdx.x >> 5;
  constexpr int NW = TEAM / 32;
  if (lane == 31) scratch[w] = incl;
  __syncthreads();
  if (w == 0) {
    int v = lane < NW ? scratch[lane] : 0;
    int vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < NW) scratch[lane] = vi - v;
    if (lane == NW - 1) scratch[32] = vi;
  }
  __syncthreads();
  total = scratch[32];
  const int r = scratch[w] + incl - x;
  __syncthreads();
  return r;
}

// Exclusive scan of one int64 per thread across a CTA (blockDim.x threads,
// a multiple of 32, at most 1024).  scratch: >= 33 long longs.
__device__ __forceinline__ long long cta_exclusive_scan64(long long x, long long* scratch,
                                                         long long& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  long long incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) scratch[w] = incl;
  __syncthreads();
  if (w == 0) {
    long long v = lane < nw ? scratch[lane] : 0;
    long long vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < nw) scratch[lane] = vi - v;
    if (lane == nw - 1) scratch[32] = vi;
  }
  __syncthreads();
  total = scratch[32];
  const long long r = scratch[w] + incl - x;
  __syncthreads();
  return r;
}

// First index in the sorted run col[q0, q1) whose column is >= x (one thread).
__device__ __forceinline__ int64_t seq_lower_bound(const int32_t* col, int64_t q0, int64_t q1,
                                                   int64_t x) {
  while (q0 < q1) {
    const int64_t mid = q0 + ((q1 - q0) >> 1);
    if ((int64_t)col[mid] < x) q0 = mid + 1;
    else q1 = mid;
  }
  return q0;
}

// Shared memory used by for_row_products_balanced: per chunk entry with a
// nonempty product range, its product offset, its first B index and its A
// index (relative to the chunk), plus scan scratch.
struct BalancedSmem {
  long long* off;  // [blockDim.x]
  long long* b0;   // [blockDim.x]
  int* pa;         // [blockDim.x]
  long long* scan; // [33]
  int* iscan;      // [33]
};

// Load-balanced form of for_row_products for a whole CTA: the row's stored
// A entries are taken in chunks of blockDim.x; the chunk's nonempty product
// ranges (B row, or the B row's slice in [lo, hi) when `sorted` and not
// `whole`) are compacted and prefix-summed, every warp takes an equal
// contiguous share of the chunk's products and its lanes take consecutive
// products (coalesced B reads).  Short ranges (< kLongRange products) and
// long ones are done in two rounds:
//   * short: since ranges are nonempty, the 32 products of one warp step
//     start at most 31 new ranges: each lane reads one range start, the warp
//     ORs together the bits of the starts that fall inside the step, and a
//     lane's range is the step's first range plus the number of starts at or
//     before its product;
//   * long: the warp walks its share range by range, 32 * U consecutive
//     products of one range per iteration, with no per-product range
//     bookkeeping (the A entry is uniform over the warp).
// All threads of the CTA must call it.
constexpr int kLongRange = 128;
constexpr int kLongUnroll = 2;   // warp steps per iteration of the long round, in units of U

template <int U, class LD, class F>
__device__ __forceinline__ void for_row_products_balanced_u(const DevCSR& A, const DevCSR& B,
                                                            int64_t i, int64_t lo, int64_t hi,
                                                            bool whole, bool sorted,
                                                            const BalancedSmem& sm, LD&& ld, F&& f) {
  typedef decltype(ld(int64_t(0))) V;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x, nwarp = nthr >> 5;
  const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
  const bool filter = !whole && !sorted;
  const unsigned width = (unsigned)(hi - lo);
  for (int64_t c0 = a0; c0 < a1; c0 += nthr) {
    const int nch = (int)min((int64_t)nthr, a1 - c0);
    long long len = 0;
    int64_t q0 = 0;
    if (tid < nch) {
      const int k = A.col[c0 + tid];
      q0 = B.rp[k];
      int64_t q1 = row_end(B, k);
      if (!whole && sorted) {
        const int64_t s0 = seq_lower_bound(B.col, q0, q1, lo);
        q1 = seq_lower_bound(B.col, s0, q1, hi);
        q0 = s0;
      }
      len = q1 - q0;
    }
    // a round with no ranges of its kind in the chunk is skipped (uniform)
    const int any_short = __syncthreads_or(len > 0 && len < kLongRange);
    const int any_long = __syncthreads_or(len >= kLongRange);
    for (int round = 0; round < 2; ++round) {
      if (!(round == 0 ? any_short : any_long)) continue;
      const long long lr = (round == 0) == (len < kLongRange) ? len : 0;
      // one scan gives both the product offsets (high bits) and the slots of
      // the nonempty ranges (low 11 bits; at most 1024 of them)
      long long packed_total;
      const long long packed =
          cta_exclusive_scan64((lr << 11) | (lr > 0 ? 1 : 0), sm.scan, packed_total);
      const long long total = packed_total >> 11;
      const int ne = (int)(packed_total & 2047);
      if (lr > 0) {
        const int slot = (int)(packed & 2047);
        sm.off[slot] = packed >> 11;
        sm.b0[slot] = q0;
        sm.pa[slot] = tid;
      }
      __syncthreads();
      const long long t_beg = total * warp / nwarp, t_end = total * (warp + 1) / nwarp;
      if (round == 1 && t_beg < t_end) {
        // range holding the warp's first product
        int l = 0, r = ne - 1;
        while (l < r) {
          const int mid = (l + r + 1) >> 1;
          if (sm.off[mid] <= t_beg) l = mid;
          else r = mid - 1;
        }
        int j = l;
        constexpr int UL = U * kLongUnroll;
        for (long long t = t_beg; t < t_end; ++j) {  // uniform over the warp
          const long long r_end = j + 1 < ne ? sm.off[j + 1] : total;
          const long long e = r_end < t_end ? r_end : t_end;
          const int64_t qb = sm.b0[j] - sm.off[j];
          const int64_t pc = c0 + sm.pa[j];
          for (long long tt = t; tt < e; tt += 32 * UL) {
            int64_t qu[UL];
            bool vu[UL];
#pragma unroll
            for (int u = 0; u < UL; ++u) {
              const long long x = tt + 32 * u + lane;
              vu[u] = x < e;
              qu[u] = qb + x;
            }
            int cu[UL];
            V vv[UL];
#pragma unroll
            for (int u = 0; u < UL; ++u) {
              cu[u] = vu[u] ? __ldg(B.col + qu[u]) : 0;
              vv[u] = vu[u] ? ld(qu[u]) : V();
            }
#pragma unroll
            for (int u = 0; u < UL; ++u)
              if (vu[u] && (!filter || (unsigned)((int64_t)cu[u] - lo) < width)) f(pc, qu[u], cu[u], vv[u]);
          }
          t = e;
        }
      }
      if (round == 0 && t_beg < t_end) {
        // range holding the warp's first product (the same search in every lane)
        int l = 0, r = ne - 1;
        while (l < r) {
          const int mid = (l + r + 1) >> 1;
          if (sm.off[mid] <= t_beg) l = mid;
          else r = mid - 1;
        }
        int j0 = l;
        long long nxt = j0 + 1 < ne ? sm.off[j0 + 1] : LLONG_MAX;  // start of the next range
        int jc = -1;          // the lane's current range, its B offset and A entry
        int64_t qb = 0, pc = 0;
        // U warp steps per iteration: positions first, then all loads, then
        // the callbacks, so that U independent loads are in flight per lane
        for (long long tb = t_beg; tb < t_end; tb += 32 * U) {
          int64_t qu[U], pu[U];
          bool vu[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const long long ts = tb + 32 * u;
            int j = j0;
            if (nxt <= ts + 31) {  // the step crosses range starts (uniform over the warp)
              const int k = j0 + 1 + lane;
              const long long st = k < ne ? sm.off[k] : LLONG_MAX;
              const long long pos = st - ts;  // >= 1 by the choice of j0
              const unsigned bits = __reduce_or_sync(0xffffffffu, pos < 32 ? 1u << (int)pos : 0u);
              j = j0 + __popc(bits & ((2u << lane) - 1u));
              j0 += __popc(bits);
              nxt = j0 + 1 < ne ? sm.off[j0 + 1] : LLONG_MAX;
            }
            const long long t = ts + lane;
            vu[u] = t < t_end;
            if (vu[u] && j != jc) {
              jc = j;
              qb = sm.b0[j] - sm.off[j];
              pc = c0 + sm.pa[j];
            }
            qu[u] = qb + t;
            pu[u] = pc;
            // range holding product ts + 32 (ranges are nonempty, so at most one more start)
            if (nxt <= ts + 32) {
              ++j0;
              nxt = j0 + 1 < ne ? sm.off[j0 + 1] : LLONG_MAX;
            }
          }
          int cu[U];
          V vv[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            cu[u] = vu[u] ? __ldg(B.col + qu[u]) : 0;
            vv[u] = vu[u] ? ld(qu[u]) : V();
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (vu[u] && (!filter || (unsigned)((int64_t)cu[u] - lo) < width)) f(pu[u], qu[u], cu[u], vv[u]);
        }
      }
      __syncthreads();
    }
  }
}

// Piece-wise form for a whole CTA: the row's stored A entries are taken in
// chunks of blockDim.x; each entry's product range (its B row, or the B
// row's slice in [lo, hi) when `sorted` and not `whole`) is cut into pieces
// of at most 32 * U consecutive products, the chunk's pieces are numbered
// by one CTA scan, and every warp takes an equal contiguous run of pieces.
// Inside a piece the A entry is the same for the whole warp and lane l
// takes products l, l + 32, ...: no per-product bookkeeping, coalesced B
// reads, all loads of a piece in flight before the callbacks.
//   on_entry(p): called (warp-uniformly) when the warp reaches the pieces of
//                A entry p; returns a token (e.g. A's value) for them;
//   f(t, c, v):  one product: the token, column c and the value ld(q) of its
//                B entry.
// All threads of the CTA must call it.
// Whether full pieces take a path without per-product bounds checks.
constexpr bool kFullPieces = true;

struct PieceSmem {
  int* poff;        // [blockDim.x] first piece of each nonempty range (chunk numbering)
  long long* q0;    // [blockDim.x] first B index of the range
  long long* len;   // [blockDim.x] products in the range
  int* pa;          // [blockDim.x] A entry of the range (relative to the chunk)
  long long* scan;  // [33]
  static constexpr size_t kBytesPerThread = sizeof(int) + 2 * sizeof(long long) + sizeof(int);
};

template <int U, class LD, class FA, class F>
__device__ __forceinline__ void for_row_pieces(const DevCSR& A, const DevCSR& B, int64_t i,
                                               int64_t lo, int64_t hi, bool whole, bool sorted,
                                               const PieceSmem& sm, LD&& ld, FA&& on_entry, F&& f) {
  typedef decltype(ld(int64_t(0))) V;
  typedef decltype(on_entry(int64_t(0))) T;
  constexpr int P = 32 * U;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x, nwarp = nthr >> 5;
  const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
  const bool filter = !whole && !sorted;
  const unsigned width = (unsigned)(hi - lo);
  for (int64_t c0 = a0; c0 < a1; c0 += nthr) {
    const int nch = (int)min((int64_t)nthr, a1 - c0);
    long long len = 0;
    int64_t q0 = 0;
    if (tid < nch) {
      const int k = A.col[c0 + tid];
      q0 = B.rp[k];
      int64_t q1 = row_end(B, k);
      if (!whole && sorted) {
        const int64_t s0 = seq_lower_bound(B.col, q0, q1, lo);
        q1 = seq_lower_bound(B.col, s0, q1, hi);
        q0 = s0;
      }
      len = q1 - q0;
    }
    const long long np = (len + P - 1) / P;
    // one scan numbers the pieces (high bits) and the nonempty ranges (low 11 bits)
    long long packed_total;
    const long long packed = cta_exclusive_scan64((np << 11) | (np > 0 ? 1 : 0), sm.scan, packed_total);
    const long long npieces = packed_total >> 11;
    const int ne = (int)(packed_total & 2047);
    if (np > 0) {
      const int slot = (int)(packed & 2047);
      sm.poff[slot] = (int)(packed >> 11);
      sm.q0[slot] = q0;
      sm.len[slot] = len;
      sm.pa[slot] = tid;
    }
    __syncthreads();
    // equal runs of pieces per warp; nwarp is a power of two (512- and
    // 1024-thread CTAs), so the split needs no 64-bit division
    const int lgw = 31 - __clz(nwarp);
    const long long k_beg = (npieces * warp) >> lgw, k_end = (npieces * (warp + 1)) >> lgw;
    if (k_beg < k_end) {  // uniform over the warp
      int l = 0, r = ne - 1;  // range holding piece k_beg
      while (l < r) {
        const int mid = (l + r + 1) >> 1;
        if (sm.poff[mid] <= k_beg) l = mid;
        else r = mid - 1;
      }
      int j = l;
      long long pj = sm.poff[j];
      long long nxt = j + 1 < ne ? sm.poff[j + 1] : LLONG_MAX;
      int64_t qj = sm.q0[j];
      long long lj = sm.len[j];
      T tok = on_entry(c0 + sm.pa[j]);
      // one piece: its products' columns and values in registers
      struct Piece {
        int n;
        T tok;
        int c[U];
        V v[U];
      };
      const auto load = [&](long long k, Piece& pc) {
        if (k >= nxt) {  // the next range starts here (ranges are nonempty)
          ++j;
          pj = nxt;
          nxt = j + 1 < ne ? sm.poff[j + 1] : LLONG_MAX;
          qj = sm.q0[j];
          lj = sm.len[j];
          tok = on_entry(c0 + sm.pa[j]);
        }
        const long long s0 = (k - pj) * P;
        pc.n = (int)min((long long)P, lj - s0);
        pc.tok = tok;
        const int64_t qs = qj + s0;
        const int32_t* cp = B.col + qs;
        if (kFullPieces && pc.n == P) {  // a full piece: no bounds to check (uniform)
#pragma unroll
          for (int u = 0; u < U; ++u) {
            pc.c[u] = __ldg(cp + u * 32 + lane);
            pc.v[u] = ld(qs + u * 32 + lane);
          }
          return;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int x = u * 32 + lane;
          pc.c[u] = 0;
          pc.v[u] = V();
          if (u * 32 < pc.n && x < pc.n) {
            pc.c[u] = __ldg(cp + x);
            pc.v[u] = ld(qs + x);
          }
        }
      };
      const auto consume = [&](const Piece& pc) {
        if (kFullPieces && pc.n == P && !filter) {
#pragma unroll
          for (int u = 0; u < U; ++u) f(pc.tok, pc.c[u], pc.v[u]);
          return;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int x = u * 32 + lane;
          if (u * 32 < pc.n && x < pc.n && (!filter || (unsigned)((int64_t)pc.c[u] - lo) < width))
            f(pc.tok, pc.c[u], pc.v[u]);
        }
      };
      for (long long k = k_beg; k < k_end; ++k) {
        Piece cur;
        load(k, cur);
        consume(cur);
      }
    }
    __syncthreads();
  }
}

// The loop above with one warp step per iteration and no value loads.
template <class F>
__device__ __forceinline__ void for_row_products_balanced(const DevCSR& A, const DevCSR& B,
                                                          int64_t i, int64_t lo, int64_t hi,
                                                          bool whole, bool sorted,
                                                          const BalancedSmem& sm, F&& f) {
  for_row_products_balanced_u<1>(A, B, i, lo, hi, whole, sorted, sm,
                                 [](int64_t) { return 0; },
                                 [&](int64_t p, int64_t q, int c, int) { f(p, q, c); });
}

}  // namespace cb
