// K5-K7: numeric phase (paper Sec. 4.1, phase (3): the products are formed
// and combined in a hash-table accumulator), with the in-row sort that makes
// every output row strictly increasing in column.
//
// Tiers by the exact row size nz = nnz(C_i) from the symbolic phase:
//   * nz <= 64:   one warp per row, keys + accumulators in a per-warp table
//   * nz <= 512:  one 256-thread team per row
//   For these, the table has 2^ceil(log2 2nz) slots (load factor <= 1/2);
//   after accumulation the team compacts the occupied slots, bitonic-sorts
//   them by column in shared memory and writes the row with coalesced stores.
//   * heavier:    rank windows (cut by the symbolic phase).  One CTA per
//                 window takes the window's column bitmap (stored by the
//                 symbolic phase, or rebuilt from the row's products),
//                 prefix-counts it, and accumulates each product at its
//                 column's rank in a dense array (shared memory for 4-byte
//                 accumulators, a per-CTA slice in L2 for 8-byte ones); the
//                 window then reads out in column order without a sort.  The
//                 products are walked in pieces of 128 consecutive products
//                 of one B row per warp (for_row_pieces).
// Products are combined with the semiring's atomic (+).
#include "cb_common.cuh"
#include "cb_kernels.h"

namespace cb {

namespace {

__device__ __forceinline__ void flag_error(int64_t* err, int64_t code) {
  if (err) atomicCAS((unsigned long long*)err, 0ull, (unsigned long long)code);
}

// LEARNED: nnz holds each row's predicted capacity instead of its exact
// size; the row is written at Crp[i] (its staging slot) only when it fits,
// its size goes to cnt_out[i]; a row that overflows its capacity (full
// table or more entries than predicted) is marked learned[i] = 0 and
// recomputed later by the exact path.
//
// Accumulator by the row's compression ratio cf = flops_i / nnz(C_i) (paper
// Sec. 4.1: hash accumulators suit high compression, merging ones low
// compression, and a hybrid picks per output line), exact sizes only:
//   * cf <= cf_esc (and flops_i within the table): expand-sort-compress --
//     the products go to consecutive table slots in arrival order (one
//     shared-memory atomic per warp step reserves them), are sorted by column
//     with the bitonic network, and each column's run is combined;
//   * cf >= cf_pre: hash, with the products of each warp step that share a
//     column combined first (__match_any_sync groups them, the group's first
//     lane adds the others' products from a per-warp scratch), so that one
//     probe and one atomic serve the group;
//   * otherwise: hash, one probe and one atomic per product.
template <int SR, int CTA, int TEAM, int TABLE_MAX, bool LEARNED = false>
__global__ void __launch_bounds__(CTA) k_num_hash(DevCSR A, DevCSR B, const int32_t* rows,
                                                  int64_t nrows_tier, const int64_t* flops,
                                                  const int64_t* nnz, const int64_t* Crp,
                                                  int32_t* Ccol, typename Sem<SR>::TC* Cval,
                                                  int64_t* err, uint8_t* learned = nullptr,
                                                  int64_t* cnt_out = nullptr,
                                                  const int64_t* dcnt = nullptr, int tier = 0,
                                                  float cf_esc = 0.0f, float cf_pre = 1e30f) {
  typedef Sem<SR> S;
  typedef typename S::A Acc;
  typedef typename S::TA TA;
  typedef typename S::TB TB;
  constexpr int TEAMS = CTA / TEAM;
  constexpr int PER = TABLE_MAX / TEAM;
  if (dcnt) {  // tier sizes on the device (launch sequences without host synchronisation)
    int64_t beg = 0;
    for (int t = 1; t < tier; ++t) beg += dcnt[t];
    rows += beg;
    nrows_tier = dcnt[tier];
  }
  extern __shared__ __align__(16) unsigned char num_smem[];
  __shared__ int scan_scratch[TEAMS][33];
  __shared__ int overflow[TEAMS];
  __shared__ int esc_cnt[TEAMS];
  __shared__ typename Sem<SR>::A pre_scratch[CTA / 32][32];
  const int team = threadIdx.x / TEAM, lane = threadIdx.x % TEAM;
  Acc* vals = reinterpret_cast<Acc*>(num_smem) + team * TABLE_MAX;
  int* keys = reinterpret_cast<int*>(reinterpret_cast<Acc*>(num_smem) + TEAMS * TABLE_MAX) + team * TABLE_MAX;
  const TA* Aval = reinterpret_cast<const TA*>(A.val);
  const TB* Bval = reinterpret_cast<const TB*>(B.val);

  for (int64_t r = (int64_t)blockIdx.x * TEAMS + team; r < nrows_tier;
       r += (int64_t)gridDim.x * TEAMS) {
    const int i = rows[r];
    const int64_t nz = nnz[i];
    const int bits = max(ceil_log2(2 * nz), 5);
    const int tsize = 1 << bits;
    if (!chk(tsize <= TABLE_MAX, 30, i)) continue;  // uniform over the team
    const uint32_t mask = (uint32_t)tsize - 1;
    const int shift = 32 - bits;
    const int64_t f = flops[i];
    int mode = 0;  // 0 hash, 1 hash with warp pre-reduction, 2 expand-sort-compress
    if (!LEARNED) {
      if (f <= tsize && (float)f <= cf_esc * (float)nz) mode = 2;
      else if ((float)f >= cf_pre * (float)nz) mode = 1;
    }
    for (int s = lane; s < tsize; s += TEAM) {
      keys[s] = kEmptyKey;
      vals[s] = S::ident();
    }
    if (LEARNED && lane == 0) overflow[team] = 0;
    if (lane == 0) esc_cnt[team] = 0;
    team_sync<TEAM>();

    // accumulate every product of row i
    const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
    const int gl = group_log2<TEAM>(f, a1 - a0);
    const int G = 1 << gl, gq = lane & (G - 1), groups = TEAM >> gl;
    const int wl = threadIdx.x & 31;
    for (int64_t p = a0 + (lane >> gl); p < a1; p += groups) {
      const int k = A.col[p];
      const TA a = S::kUsesA ? Aval[p] : TA();
      const int64_t b1 = row_end(B, k);
      for (int64_t q = B.rp[k] + gq; q < b1; q += G) {
        const int c = B.col[q];
        if (!in_window(B, c)) continue;
        const Acc v = S::mul(a, Bval[q]);
        if (mode == 2) {  // the next free slots, one atomic per warp step
          const unsigned am = __activemask();
          const int leader = __ffs(am) - 1;
          int base = 0;
          if (wl == leader) base = atomicAdd(&esc_cnt[team], __popc(am));
          base = __shfl_sync(am, base, leader);
          const int t = base + __popc(am & ((1u << wl) - 1u));
          if (chk(t < tsize, 31, t)) {
            keys[t] = c;
            vals[t] = v;
          }
          continue;
        }
        Acc sum = v;
        bool lead = true;
        if (mode == 1) {  // combine the warp step's products of one column first
          const unsigned am = __activemask();
          const unsigned peers = __match_any_sync(am, c);
          lead = wl == __ffs(peers) - 1;
          pre_scratch[threadIdx.x >> 5][wl] = v;
          __syncwarp(am);
          if (lead)
            for (unsigned o = peers & (peers - 1); o; o &= o - 1)
              sum = S::add(sum, pre_scratch[threadIdx.x >> 5][__ffs(o) - 1]);
          __syncwarp(am);
        }
        if (lead) {
          bool ins;
          const int slot = probe_insert(keys, mask, shift, c, ins);
          if (slot >= 0) S::atomic(&vals[slot], sum);
          else if (LEARNED) overflow[team] = 1;
          else if (chk(false, 32, i)) flag_error(err, 20);
        }
      }
    }
    team_sync<TEAM>();

    // compact occupied slots (registers first, so the table can be overwritten)
    int mk[PER];
    Acc mv[PER];
    int mc = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int s = lane + j * TEAM;
      mk[j] = kEmptyKey;
      if (s < tsize) {
        mk[j] = keys[s];
        mv[j] = vals[s];
      }
      mc += mk[j] != kEmptyKey;
    }
    int total;
    int pos = team_exclusive_scan<TEAM>(mc, scan_scratch[team], total);
    team_sync<TEAM>();
    if (LEARNED && (overflow[team] || total > nz)) {  // uniform over the team
      if (lane == 0) {
        learned[i] = 0;
        cnt_out[i] = 0;
        if (err) atomicAdd((unsigned long long*)err, 1ull);  // overflow count
      }
      team_sync<TEAM>();
      continue;
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      if (mk[j] != kEmptyKey) {
        if (chk(pos < tsize, 33, pos)) {
          keys[pos] = mk[j];
          vals[pos] = mv[j];
        }
        ++pos;
      }
    }
    const int P = 1 << ceil_log2(total > 0 ? total : 1);
    for (int t = total + lane; t < P; t += TEAM) keys[t] = INT_MAX;
    team_sync<TEAM>();

    // bitonic sort of P (key, value) pairs by key
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = lane; t < (P >> 1); t += TEAM) {
          const int lo = ((t & ~(j - 1)) << 1) | (t & (j - 1));  // j is a power of two
          const int hi = lo + j;
          const bool asc = (lo & k) == 0;
          const int ka = keys[lo], kb = keys[hi];
          if ((ka > kb) == asc) {
            keys[lo] = kb;
            keys[hi] = ka;
            const Acc va = vals[lo];
            vals[lo] = vals[hi];
            vals[hi] = va;
          }
        }
        team_sync<TEAM>();
      }
    }

    if (mode == 2) {  // combine each column's run of the sorted products
      const int per = (total + TEAM - 1) / TEAM;
      const int t0 = lane * per, t1 = min(total, t0 + per);
      int h = 0;
      for (int t = t0; t < t1; ++t) h += t == 0 || keys[t] != keys[t - 1];
      int heads;
      int hpos = team_exclusive_scan<TEAM>(h, scan_scratch[team], heads);
      if (heads != nz && lane == 0) flag_error(err, 21);
      const int64_t off = Crp[i];
      for (int t = t0; t < t1; ++t) {
        if (t == 0 || keys[t] != keys[t - 1]) {
          Acc v = vals[t];
          for (int u = t + 1; u < total && keys[u] == keys[t]; ++u) v = S::add(v, vals[u]);
          if (guard(hpos < nz, 34, off + hpos)) {
            Ccol[off + hpos] = keys[t];
            Cval[off + hpos] = S::out(v);
          }
          ++hpos;
        }
      }
      team_sync<TEAM>();
      continue;
    }

    // write the sorted row
    if (!LEARNED && total != nz && lane == 0) flag_error(err, 21);
    if (lane == 0) chk(LEARNED || total <= nz, 35, i);
    if (LEARNED && lane == 0) cnt_out[i] = total;
    const int nw = total < nz ? total : (int)nz;
    const int64_t off = Crp[i];
    for (int t = lane; t < nw; t += TEAM) {
      Ccol[off + t] = keys[t];
      Cval[off + t] = S::out(vals[t]);
    }
    team_sync<TEAM>();
  }
}

// Rank windows of heavy rows (nnz > 512).  One CTA per window: take the
// window's column bitmap (stored by the symbolic phase, or rebuilt from the
// row's products), prefix-count its words, then accumulate every product
// into the dense accumulator at its column's rank and write the window's
// slice of the row in column order.
constexpr bool kRankInPlace = true;

// Launch shape of the rank windows per semiring: 512-thread CTAs, three per
// SM, when the accumulators take little or no shared memory (8-byte ones
// reduce in L2; (or,and) keeps one bit per slot), else one 1024-thread CTA
// per SM holding kWcap 4-byte shared accumulators.
template <int SR>
struct RankShape {
  static constexpr bool kBits = SR == 4;
  static constexpr int kCta = (NumLimits<SR>::kL2Acc || kBits) ? 512 : 1024;
  static constexpr size_t kAccBytes =
      NumLimits<SR>::kL2Acc ? 0
      : kBits ? (size_t)NumLimits<SR>::kWcap / 8
              : (size_t)NumLimits<SR>::kWcap * sizeof(typename Sem<SR>::A);
  static constexpr size_t kSmem = kAccBytes + kSpanWords * (sizeof(unsigned) + sizeof(unsigned short)) +
                                  (size_t)kCta * PieceSmem::kBytesPerThread;
};

// L2 residency of the windows that accumulate in C (fp64 and int64): the
// zeroing stores and the reductions carry an evict_last policy, so that the
// lines a window is still reducing into outlive the streaming traffic around
// them (stored bitmaps, columns written out, other windows' finished lines);
// when the window is complete its lines are set back to evict_normal.  At
// R-MAT s16 this cut the fp64 numeric phase's DRAM writes from 5.20 to 4.36 GB
// (C is 4.27 GB) at the same speed.
__device__ __forceinline__ unsigned long long policy_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void red_add_hint(double* a, double v, unsigned long long pol) {
  asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.f64 [%0], %1, %2;" :: "l"(a), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_add_hint(unsigned long long* a, unsigned long long v, unsigned long long pol) {
  asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.u64 [%0], %1, %2;" :: "l"(a), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(void* a, unsigned long long v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" :: "l"(a), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void demote_line(const void* a) {
  asm volatile("applypriority.global.L2::evict_normal [%0], 128;" :: "l"(a) : "memory");
}

template <int SR, int CTA>
__global__ void __launch_bounds__(CTA, CTA == 512 ? 3 : 1) k_num_rank(DevCSR A, DevCSR B, const int32_t* heavy_rows,
                                                      const Window* wins, int64_t n_wins,
                                                      const int32_t* span_counts, int64_t spans,
                                                      const unsigned* hbits, int b_sorted,
                                                      const int64_t* flops, const int64_t* nnz,
                                                      const int64_t* Crp, int32_t* Ccol,
                                                      typename Sem<SR>::TC* Cval, int64_t* err,
                                                      int64_t num_hash_max,
                                                      typename Sem<SR>::A* racc,
                                                      const int64_t* dcounters = nullptr) {
  typedef Sem<SR> S;
  typedef typename S::A Acc;
  typedef typename S::TA TA;
  typedef typename S::TB TB;
  typedef typename S::TC TC;
  constexpr int WCAP = NumLimits<SR>::kWcap;
  if (dcounters) {  // sizes on the device: heavy segment of the symbolic order, windows, sortedness
    heavy_rows += dcounters[kCntSym + 1] + dcounters[kCntSym + 2] + dcounters[kCntSym + 3];
    // a symbolic-phase error (e.g. window capacity) leaves the window list
    // unusable: do nothing then (the caller reads the error word)
    n_wins = dcounters[kError] ? 0 : dcounters[kUnits];
    b_sorted = dcounters[kUnsorted] == 0 ? 1 : 0;
  }
  // 8-byte accumulators reduce in L2 (a per-CTA slice of racc): shared-memory
  // 64-bit atomics cost more than L2 reductions, and without shared
  // accumulators three 512-thread CTAs share an SM (40 registers each).
  constexpr bool kL2 = NumLimits<SR>::kL2Acc;
  // (+,x) over int64 and fp64 accumulate in L2 directly in the window's
  // output entries (their accumulator bits are the output value's), so the
  // values need no copy out of a scratch slice; other 8-byte semirings use
  // the slice and convert on the way out.
  constexpr bool kInPlace = kL2 && kRankInPlace && (SR == 1 || SR == 2);
  constexpr int WPT = kSpanWords / CTA;
  static_assert(WCAP <= 65535, "a window's entry counts are kept in 16 bits");
  extern __shared__ __align__(16) unsigned char rank_smem[];
  // shared layout: [accumulators (shared-memory windows only)] [bx] [by] [iterator scratch]
  Acc* acc = reinterpret_cast<Acc*>(rank_smem);
  // word w of the window: bx[w] = its column bits, by[w] = entries of the
  // window before it (< 2^16: a window holds at most kWcap entries).  Two
  // arrays, not one of pairs: a product's lookup of both words then meets
  // fewer shared-memory bank conflicts; 16-bit counts leave room for a third
  // CTA per SM.
  constexpr bool kBits = RankShape<SR>::kBits;  // (or,and): one accumulator bit per slot
  unsigned* accbits = reinterpret_cast<unsigned*>(rank_smem);
  unsigned* bx = reinterpret_cast<unsigned*>(rank_smem + RankShape<SR>::kAccBytes);
  unsigned short* by = reinterpret_cast<unsigned short*>(bx + kSpanWords);
  long long* bal = reinterpret_cast<long long*>(by + kSpanWords);
  __shared__ int scratch[33];
  __shared__ long long scan64[33];
  const PieceSmem sm{reinterpret_cast<int*>(bal + 2 * CTA), bal, bal + CTA,
                     reinterpret_cast<int*>(bal + 2 * CTA) + CTA, scan64};
  __shared__ long long s_base;
  const int tid = threadIdx.x, lane = tid & 31;
  const TA* Aval = reinterpret_cast<const TA*>(A.val);
  const TB* Bval = reinterpret_cast<const TB*>(B.val);

  for (int64_t u = blockIdx.x; u < n_wins; u += gridDim.x) {
    const Window wd = wins[u];
    const int i = heavy_rows[wd.h];
    if (nnz[i] <= num_hash_max || wd.count <= 0) continue;  // hash tiers own these rows
    const int cnt = wd.count < WCAP ? wd.count : WCAP;
    const int64_t span_lo = B.col_lo + (int64_t)wd.span * kSpanCols;
    const int64_t lo = span_lo + 32 * (int64_t)wd.w_lo;
    const int64_t rw = row_width(A, B, i);
    const int64_t hi = min(span_lo + 32 * (int64_t)wd.w_hi, B.col_lo + rw);
    const bool whole = lo == B.col_lo && hi == B.col_lo + rw && !B.filter;
    const int nw = wd.w_hi - wd.w_lo;
    if (hbits) {
      const unsigned* src = hbits + (size_t)((int64_t)wd.h * spans + wd.span) * kSpanWords + wd.w_lo;
      for (int w = tid; w < nw; w += CTA) bx[w] = kStreamOut ? __ldcs(src + w) : src[w];
    } else {
      for (int w = tid; w < nw; w += CTA) bx[w] = 0u;
    }
    if (tid < 32) {
      long long o = 0;
      for (int64_t t = lane; t < wd.span; t += 32) o += span_counts[(int64_t)wd.h * spans + t];
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) o += __shfl_down_sync(0xffffffffu, o, d);
      if (lane == 0) s_base = o + wd.rank;
    }
    __syncthreads();
    // the window's slice of the row: C entries [out, out + cnt)
    const int64_t out = Crp[i] + s_base;
    const int64_t row_end = Crp[i + 1];
    Acc* wacc = kInPlace ? reinterpret_cast<Acc*>(Cval + out)
                         : (kL2 ? racc + (size_t)blockIdx.x * WCAP : acc);
    // slots past the row's end (an inconsistent count) are dropped
    const int lim = kInPlace ? (int)max((int64_t)0, min((int64_t)cnt, row_end - out)) : cnt;
    unsigned long long pol = 0;
    if constexpr (kInPlace) {
      pol = policy_evict_last();
      for (int t = tid; t < lim; t += CTA) {
        const Acc z = S::ident();
        unsigned long long zb;
        memcpy(&zb, &z, 8);
        st_hint(wacc + t, zb, pol);
      }
    } else if constexpr (kBits) {
      for (int t = tid; t < (lim + 31) / 32; t += CTA) accbits[t] = 0u;
    } else {
      for (int t = tid; t < lim; t += CTA) wacc[t] = S::ident();
    }

    if (!hbits) {  // pass 1: rebuild the window's columns
      for_row_pieces<2>(A, B, i, lo, hi, whole, b_sorted != 0, sm, [](int64_t) { return 0; },
                               [](int64_t) { return 0; }, [&](int, int c, int) {
                          const unsigned off = (unsigned)((int64_t)c - lo);
                          const unsigned bit = 1u << (off & 31);
                          if (chk(off < 32u * (unsigned)nw, 36, c)) atomicOr(&bx[off >> 5], bit);
                        });
      __syncthreads();
    }
    // exclusive prefix of word popcounts
    {
      int c[WPT];
      popc_words<WPT>(bx, tid * WPT, nw, c);
      int mine = 0;
#pragma unroll
      for (int j = 0; j < WPT; ++j) mine += c[j];
      int total;
      const int run = team_exclusive_scan<CTA>(mine, scratch, total);
      store_counts<WPT>(by, tid * WPT, nw, run, c);
      if (tid == 0 && total != wd.count) flag_error(err, 23);
    }
    __syncthreads();
    // pass 2: accumulate at the rank of each product's column (pieces of
    // 128 products of one B row per warp, loads first, then the atomics)
    const unsigned lo32 = (unsigned)lo;
    for_row_pieces<4>(A, B, i, lo, hi, whole, b_sorted != 0, sm,
                      [&](int64_t q) { return ldg_val(Bval + q); },
                      [&](int64_t p) { return S::kUsesA ? ldg_val(Aval + p) : TA(); },
                      [&](TA a_cur, int c, TB bv) {
                        const unsigned off = (unsigned)c - lo32;
                        if (!chk(off < 32u * (unsigned)nw, 36, c)) return;
                        const uint2 e = make_uint2(bx[off >> 5], by[off >> 5]);
                        const int slot = (int)e.y + __popc(e.x & ((1u << (off & 31)) - 1u));
                        if (guard(slot < lim, 37, out + slot)) {
                          if constexpr (kInPlace) {
                            red_add_hint(&wacc[slot], S::mul(a_cur, bv), pol);
                          } else if constexpr (kBits) {
                            if (S::mul(a_cur, bv)) atomicOr(&accbits[slot >> 5], 1u << (slot & 31));
                          } else {
                            S::atomic(&wacc[slot], S::mul(a_cur, bv));
                          }
                        }
                      });
    __syncthreads();
    if (kInPlace && lim > 0) {  // the window is complete: its lines back to normal priority
      const uintptr_t b0 = reinterpret_cast<uintptr_t>(wacc) & ~(uintptr_t)127;
      const uintptr_t b1 = reinterpret_cast<uintptr_t>(wacc + lim);
      for (uintptr_t a = b0 + (uintptr_t)tid * 128; a < b1; a += (uintptr_t)CTA * 128)
        demote_line(reinterpret_cast<const void*>(a));
    }
    // write the window: values by slot (coalesced; in place they are there
    // already), columns by word
    if constexpr (kBits) {
      for (int t = tid; t < cnt; t += CTA)
        if (guard(out + t < row_end, 38, out + t))
          st_out(Cval + out + t, (TC)((accbits[t >> 5] >> (t & 31)) & 1u));
    } else if constexpr (!kInPlace) {
      for (int t = tid; t < cnt; t += CTA)
        if (guard(out + t < row_end, 38, out + t))
          st_out(Cval + out + t, S::out(kL2 ? __ldcg(wacc + t) : wacc[t]));
    }
    for_bitmap_columns<kL2 ? kDenseWordBits : 0, CTA>(bx, by, nw, cnt, [&](int j, int c) {
      const int64_t o = out + j;
      if (guard(o < row_end, 39, o)) st_out(Ccol + o, (int32_t)(lo + c));
    });
    __syncthreads();
  }
}

template <class K>
void set_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

inline int capped(int64_t want, int64_t cap) {
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

template <int SR>
void numeric_sr(const DevCSR& A, const DevCSR& B, const int32_t* perm, const int64_t* seg_begin,
                const int64_t* seg_count, const int64_t* flops, const int64_t* nnz,
                const int32_t* heavy_rows, const Window* wins, int64_t n_wins,
                const int32_t* span_counts, int64_t spans, const unsigned* hbits, int b_sorted,
                const int64_t* Crp, int32_t* Ccol, void* Cval_, int64_t* err, cudaStream_t s,
                int sms, int* launches, int64_t num_hash_max, void* racc, CfBounds cf) {
  typedef typename Sem<SR>::A Acc;
  typedef typename Sem<SR>::TC TC;
  TC* Cval = reinterpret_cast<TC*>(Cval_);
  constexpr size_t slot = sizeof(Acc) + sizeof(int);
  if (seg_count[kNumWarp]) {
    constexpr int CTA = 256, TEAM = 32, TBL = 2 * kNumWarpMax;
    const size_t smem = (CTA / TEAM) * TBL * slot;
    k_num_hash<SR, CTA, TEAM, TBL><<<capped((seg_count[kNumWarp] + 7) / 8, sms * 8), CTA, smem, s>>>(
        A, B, perm + seg_begin[kNumWarp], seg_count[kNumWarp], flops, nnz, Crp, Ccol, Cval, err, nullptr,
        nullptr, nullptr, 0, cf.esc, cf.pre);
    ++*launches;
  }
  if (seg_count[kNumSmall]) {
    constexpr int CTA = 256, TEAM = 256, TBL = 2 * kNumSmallMax;
    const size_t smem = TBL * slot;
    k_num_hash<SR, CTA, TEAM, TBL><<<capped(seg_count[kNumSmall], sms * 8), CTA, smem, s>>>(
        A, B, perm + seg_begin[kNumSmall], seg_count[kNumSmall], flops, nnz, Crp, Ccol, Cval, err, nullptr,
        nullptr, nullptr, 0, cf.esc, cf.pre);
    ++*launches;
  }
  if (seg_count[kNumLarge]) {
    constexpr int CTA = 512, TEAM = 512, TBL = 2 * NumLimits<SR>::kLargeMax;
    const size_t smem = TBL * slot;
    set_smem(k_num_hash<SR, CTA, TEAM, TBL>, smem);
    k_num_hash<SR, CTA, TEAM, TBL><<<capped(seg_count[kNumLarge], sms * 4), CTA, smem, s>>>(
        A, B, perm + seg_begin[kNumLarge], seg_count[kNumLarge], flops, nnz, Crp, Ccol, Cval, err, nullptr,
        nullptr, nullptr, 0, cf.esc, cf.pre);
    ++*launches;
  }
  if (n_wins) {
    // windows whose accumulators take little or no shared memory run three
    // 512-thread CTAs per SM, three windows at once (RankShape)
    constexpr int CTA = RankShape<SR>::kCta;
    constexpr int PER_SM = CTA == 512 ? 3 : 1;
    constexpr size_t smem = RankShape<SR>::kSmem;
    set_smem(k_num_rank<SR, CTA>, smem);
    k_num_rank<SR, CTA><<<capped(n_wins, (int64_t)sms * PER_SM), CTA, smem, s>>>(
        A, B, heavy_rows, wins, n_wins, span_counts, spans, hbits, b_sorted, flops, nnz, Crp, Ccol,
        Cval, err, num_hash_max, static_cast<Acc*>(racc));
    ++*launches;
  }
}

// Hash tiers only, tier sizes read on the device (counters[kCntNum..]): the
// grids are sized for the worst case and the kernels stride over their tier.
template <int SR>
void numeric_dev_sr(const DevCSR& A, const DevCSR& B, const int32_t* perm, const int64_t* counters,
                    const int64_t* flops, const int64_t* nnz, const int64_t* Crp, int32_t* Ccol,
                    void* Cval_, int64_t* err, cudaStream_t s, int sms, int64_t m,
                    const int32_t* perm_sym, const Window* wins, const int32_t* span_counts,
                    int64_t spans, void* racc, int64_t num_hash_max, CfBounds cf) {
  typedef typename Sem<SR>::A Acc;
  typedef typename Sem<SR>::TC TC;
  TC* Cval = reinterpret_cast<TC*>(Cval_);
  constexpr size_t slot = sizeof(Acc) + sizeof(int);
  const int64_t* dc = counters + kCntNum;
  {
    constexpr int CTA = 256, TEAM = 32, TBL = 2 * kNumWarpMax;
    const size_t smem = (CTA / TEAM) * TBL * slot;
    k_num_hash<SR, CTA, TEAM, TBL><<<capped((m + 7) / 8, sms * 8), CTA, smem, s>>>(
        A, B, perm, 0, flops, nnz, Crp, Ccol, Cval, err, nullptr, nullptr, dc, kNumWarp, cf.esc, cf.pre);
  }
  {
    constexpr int CTA = 256, TEAM = 256, TBL = 2 * kNumSmallMax;
    k_num_hash<SR, CTA, TEAM, TBL><<<capped(m, sms * 8), CTA, TBL * slot, s>>>(
        A, B, perm, 0, flops, nnz, Crp, Ccol, Cval, err, nullptr, nullptr, dc, kNumSmall, cf.esc, cf.pre);
  }
  {  // shared-memory attribute set by prepare_dev_launchers
    constexpr int CTA = 512, TEAM = 512, TBL = 2 * NumLimits<SR>::kLargeMax;
    const size_t smem = TBL * slot;
    k_num_hash<SR, CTA, TEAM, TBL><<<capped(m, sms * 4), CTA, smem, s>>>(
        A, B, perm, 0, flops, nnz, Crp, Ccol, Cval, err, nullptr, nullptr, dc, kNumLarge, cf.esc, cf.pre);
  }
  {  // rank windows of the heavy rows (window count read on the device)
    constexpr int CTA = RankShape<SR>::kCta;
    constexpr int PER_SM = CTA == 512 ? 3 : 1;
    constexpr size_t smem = RankShape<SR>::kSmem;
    k_num_rank<SR, CTA><<<sms * PER_SM, CTA, smem, s>>>(
        A, B, perm_sym, wins, 0, span_counts, spans, nullptr, 0, flops, nnz, Crp, Ccol, Cval, err,
        num_hash_max, static_cast<Acc*>(racc), counters);
  }
}

template <int SR>
void learned_sr(const DevCSR& A, const DevCSR& B, const int32_t* perm, const int64_t* seg_begin,
                const int64_t* seg_count, const int64_t* flops, const int64_t* cap,
                const int64_t* stage_rp, int32_t* scol, void* sval_, uint8_t* learned,
                int64_t* cnt, int64_t* overflows, cudaStream_t s, int sms, int* launches) {
  typedef typename Sem<SR>::A Acc;
  typedef typename Sem<SR>::TC TC;
  TC* sval = reinterpret_cast<TC*>(sval_);
  constexpr size_t slot = sizeof(Acc) + sizeof(int);
  if (seg_count[1]) {
    constexpr int CTA = 256, TEAM = 32, TBL = 2 * kNumWarpMax;
    k_num_hash<SR, CTA, TEAM, TBL, true><<<capped((seg_count[1] + 7) / 8, sms * 8), CTA,
                                            (CTA / TEAM) * TBL * slot, s>>>(
        A, B, perm + seg_begin[1], seg_count[1], flops, cap, stage_rp, scol, sval, overflows,
        learned, cnt);
    ++*launches;
  }
  if (seg_count[2]) {
    constexpr int CTA = 256, TEAM = 256, TBL = 2 * kNumSmallMax;
    k_num_hash<SR, CTA, TEAM, TBL, true><<<capped(seg_count[2], sms * 8), CTA, TBL * slot, s>>>(
        A, B, perm + seg_begin[2], seg_count[2], flops, cap, stage_rp, scol, sval, overflows,
        learned, cnt);
    ++*launches;
  }
  if (seg_count[3]) {
    constexpr int CTA = 512, TEAM = 512, TBL = 2 * NumLimits<SR>::kLearnHashMax;
    const size_t smem = TBL * slot;
    set_smem(k_num_hash<SR, CTA, TEAM, TBL, true>, smem);
    k_num_hash<SR, CTA, TEAM, TBL, true><<<capped(seg_count[3], sms * 4), CTA, smem, s>>>(
        A, B, perm + seg_begin[3], seg_count[3], flops, cap, stage_rp, scol, sval, overflows,
        learned, cnt);
    ++*launches;
  }
}

}  // namespace

void launch_learned_numeric(int sr, const DevCSR& A, const DevCSR& B, const int32_t* perm,
                            const int64_t* seg_begin, const int64_t* seg_count,
                            const int64_t* flops, const int64_t* cap, const int64_t* stage_rp,
                            int32_t* scol, void* sval, uint8_t* learned, int64_t* cnt,
                            int64_t* overflows, cudaStream_t s, int sms, int* launches) {
#define CB_LRN(SRV)                                                                            \
  learned_sr<SRV>(A, B, perm, seg_begin, seg_count, flops, cap, stage_rp, scol, sval, learned, \
                  cnt, overflows, s, sms, launches)
  switch (sr) {
#define CB_CASE(SRV) case SRV: CB_LRN(SRV); break;
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
  }
#undef CB_LRN
}

int learn_hash_max(int sr) {
  switch (sr) {
#define CB_CASE(SRV) case SRV: return NumLimits<SRV>::kLearnHashMax;
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
    default: return 0;
  }
}

int num_window_cut(int sr) {
  switch (sr) {
#define CB_CASE(SRV) case SRV: return NumLimits<SRV>::kWcut;
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
    default: return 0;
  }
}

int num_large_max(int sr) {
  switch (sr) {
#define CB_CASE(SRV) case SRV: return NumLimits<SRV>::kLargeMax;
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
    default: return 0;
  }
}

void launch_numeric(int sr, const DevCSR& A, const DevCSR& B, const int32_t* perm,
                    const int64_t* seg_begin, const int64_t* seg_count, const int64_t* flops,
                    const int64_t* nnz, const int32_t* heavy_rows, const Window* wins,
                    int64_t n_wins, const int32_t* span_counts, int64_t spans,
                    const unsigned* hbits, int b_sorted, const int64_t* Crp, int32_t* Ccol,
                    void* Cval, int64_t* err, cudaStream_t s, int sms, int* launches,
                    int64_t num_hash_max, void* racc, CfBounds cf) {
#define CB_NUM(SRV)                                                                        \
  numeric_sr<SRV>(A, B, perm, seg_begin, seg_count, flops, nnz, heavy_rows, wins, n_wins,   \
                  span_counts, spans, hbits, b_sorted, Crp, Ccol, Cval, err, s, sms, launches, \
                  num_hash_max, racc, cf)
  switch (sr) {
#define CB_CASE(SRV) case SRV: CB_NUM(SRV); break;
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
  }
#undef CB_NUM
}

template <int SR>
size_t rank_scratch_bytes_sr(int sms) {
  // one slice of kWcap accumulators per resident CTA (three 512-thread CTAs per SM)
  return NumLimits<SR>::kL2Acc
             ? 3 * (size_t)sms * NumLimits<SR>::kWcap * sizeof(typename Sem<SR>::A)
             : 0;
}

template <int SR>
void prepare_numeric_dev_sr() {
  typedef typename Sem<SR>::A Acc;
  constexpr int CTA = 512, TEAM = 512, TBL = 2 * NumLimits<SR>::kLargeMax;
  set_smem(k_num_hash<SR, CTA, TEAM, TBL>, TBL * (sizeof(Acc) + sizeof(int)));
  constexpr int RCTA = RankShape<SR>::kCta;
  constexpr size_t rsmem = RankShape<SR>::kSmem;
  set_smem(k_num_rank<SR, RCTA>, rsmem);
}

void prepare_dev_launchers(int sr) {
  prepare_symbolic_dev();
  switch (sr) {
#define CB_CASE(SRV) case SRV: prepare_numeric_dev_sr<SRV>(); break;
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
  }
}

void launch_numeric_dev(int sr, const DevCSR& A, const DevCSR& B, const int32_t* perm,
                        const int64_t* counters, const int64_t* flops, const int64_t* nnz,
                        const int64_t* Crp, int32_t* Ccol, void* Cval, int64_t* err, cudaStream_t s,
                        int sms, const int32_t* perm_sym, const Window* wins,
                        const int32_t* span_counts, int64_t spans, void* racc, int64_t num_hash_max,
                        CfBounds cf) {
  const int64_t m = A.nrows;
  if (m == 0) return;
#define CB_NDEV(SRV)                                                                            \
  numeric_dev_sr<SRV>(A, B, perm, counters, flops, nnz, Crp, Ccol, Cval, err, s, sms, m, perm_sym, \
                      wins, span_counts, spans, racc, num_hash_max, cf)
  switch (sr) {
#define CB_CASE(SRV) case SRV: CB_NDEV(SRV); break;
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
  }
#undef CB_NDEV
}

size_t rank_scratch_bytes(int sr, int sms) {
  switch (sr) {
#define CB_CASE(SRV) case SRV: return rank_scratch_bytes_sr<SRV>(sms);
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
  }
  return 0;
}

CB_CHECK_READER(numeric)

}  // namespace cb
