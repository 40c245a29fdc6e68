// K3: symbolic phase (paper Sec. 4.1, phase (2): the pattern of C is found
// from the input patterns alone, which sizes C before any value is formed).  nnz(C_i) = |union over stored A(i,p) of cols(B(p,:))|.
//
// Rows are processed by tier of u_i = min(flops_i, ncols):
//   * u <= 128:  one warp per row, insert-only hash of 2^ceil(log2 2u) keys
//   * u <= 512:  one 256-thread team per row, same table shape
//   * heavier:   dense bitmap of the row's columns, one CTA per (row, span
//                of 2^18 columns); the span is also cut into rank windows
//                that the numeric phase processes one CTA each.
// Inside a team, lanes form groups of G = 2^g lanes (G ~ mean B-row length
// of the row); each group walks one stored A entry's B row with coalesced
// loads while the groups stride over A's row.
#include "cb_common.cuh"
#include "cb_kernels.h"

namespace cb {

namespace {

template <int CTA, int TEAM, int TABLE_MAX>
__global__ void __launch_bounds__(CTA) k_sym_hash(DevCSR A, DevCSR B, const int32_t* rows,
                                                  int64_t nrows_tier, const int64_t* flops,
                                                  int64_t* nnz, const int64_t* dcnt = nullptr,
                                                  int tier = 0) {
  extern __shared__ int sym_keys[];
  __shared__ int block_count;
  if (dcnt) {  // tier sizes on the device (launch sequences without host synchronisation)
    int64_t beg = 0;
    for (int t = 1; t < tier; ++t) beg += dcnt[t];
    rows += beg;
    nrows_tier = dcnt[tier];
  }
  constexpr int TEAMS = CTA / TEAM;
  const int team = threadIdx.x / TEAM, lane = threadIdx.x % TEAM;
  int* keys = sym_keys + team * TABLE_MAX;
  for (int64_t r = (int64_t)blockIdx.x * TEAMS + team; r < nrows_tier;
       r += (int64_t)gridDim.x * TEAMS) {
    const int i = rows[r];
    const int64_t f = flops[i];
    const int64_t u = min(f, row_width(A, B, i));
    const int bits = max(ceil_log2(2 * u), 5);
    const int tsize = 1 << bits;
    const uint32_t mask = (uint32_t)tsize - 1;
    const int shift = 32 - bits;
    for (int s = lane; s < tsize; s += TEAM) keys[s] = kEmptyKey;
    if (TEAM > 32 && threadIdx.x == 0) block_count = 0;
    team_sync<TEAM>();
    const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
    const int gl = group_log2<TEAM>(f, a1 - a0);
    const int G = 1 << gl, gq = lane & (G - 1), groups = TEAM >> gl;
    int cnt = 0;
    for (int64_t p = a0 + (lane >> gl); p < a1; p += groups) {
      const int k = A.col[p];
      const int64_t b1 = row_end(B, k);
      for (int64_t q = B.rp[k] + gq; q < b1; q += G) {
        const int c = B.col[q];
        if (!in_window(B, c)) continue;
        bool ins;
        chk(probe_insert(keys, mask, shift, c, ins) >= 0, 41, i);
        cnt += ins;
      }
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (TEAM == 32) {
      if (lane == 0) nnz[i] = cnt;
    } else {
      if ((threadIdx.x & 31) == 0) atomicAdd(&block_count, cnt);
      __syncthreads();
      if (threadIdx.x == 0) nnz[i] = block_count;
    }
    team_sync<TEAM>();
  }
}

// Heavy rows (u > 512): one CTA per (heavy row h, span) unit.  The bitmap
// covers the span's columns [lo, hi); after counting, the span is cut into
// rank windows of at most wcut + 31 entries (see cb_common.cuh), appended to
// `wins` (when non-null) for the numeric phase.
__global__ void __launch_bounds__(1024, 2) k_sym_bitmap(DevCSR A, DevCSR B, const int32_t* heavy_rows,
                                                     int64_t n_heavy, int64_t spans,
                                                     const int64_t* flops, int wcut, int64_t* nnz,
                                                     int32_t* span_counts, int2* span_wins,
                                                     Window* wins, int64_t win_cap,
                                                     unsigned* hbits, int b_sorted,
                                                     int64_t* counters) {
  extern __shared__ __align__(16) unsigned sym_bm[];
  __shared__ int scratch[33];
  __shared__ long long scan64[33];
  __shared__ int wstart[kMaxWindowsPerSpan];
  __shared__ int wrank[kMaxWindowsPerSpan];
  __shared__ long long wbase;
  constexpr int WPT = kSpanWords / 1024;  // bitmap words per thread in the scan
  const int tid = threadIdx.x;
  if (b_sorted < 0) {  // sizes on the device: heavy segment of perm, count, B's sortedness
    heavy_rows += counters[kCntSym + 1] + counters[kCntSym + 2] + counters[kCntSym + 3];
    n_heavy = counters[kCntSym + kSymHeavy];
    b_sorted = counters[kUnsorted] == 0 ? 1 : 0;
  }
  const int64_t units = n_heavy * spans;
  const int bm_words = (int)min((int64_t)kSpanWords, (B.ncols + 31) / 32);
  long long* bal = reinterpret_cast<long long*>(sym_bm + ((bm_words + 3) & ~3));
  const PieceSmem sm{reinterpret_cast<int*>(bal + 2048), bal, bal + 1024,
                     reinterpret_cast<int*>(bal + 2048) + 1024, scan64};
  // the bitmap starts clear; each unit clears the words it set once it has
  // read them, so no unit starts with a clearing pass of its own
  for (int w = tid; w < bm_words; w += 1024) sym_bm[w] = 0u;
  __syncthreads();
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t h = spans == 1 ? u : u / spans, sp = u - h * spans;
    const int i = heavy_rows[h];
    const int64_t lo = B.col_lo + sp * (int64_t)kSpanCols;
    const int64_t hi = min(lo + (int64_t)kSpanCols, B.col_lo + row_width(A, B, i));
    if (hi <= lo) {  // this row's columns end before the span: nothing to count
      if (tid == 0) {
        span_counts[h * spans + sp] = 0;
        if (span_wins) span_wins[h * spans + sp] = make_int2(0, 0);
      }
      continue;
    }
    const int nwords = (int)((hi - lo + 31) / 32);
    const unsigned lo32 = (unsigned)lo;
    for_row_pieces<4>(A, B, i, lo, hi, spans == 1 && !B.filter, b_sorted != 0, sm,
                             [](int64_t) { return 0; }, [](int64_t) { return 0; }, [&](int, int c, int) {
                        const unsigned off = (unsigned)c - lo32;
                        const unsigned bit = 1u << (off & 31);
                        if (chk(off < 32u * (unsigned)nwords, 40, c)) atomicOr(&sym_bm[off >> 5], bit);
                      });
    __syncthreads();
    if (hbits) {
      unsigned* dst = hbits + (size_t)(h * spans + sp) * kSpanWords;
      for (int w = tid; w < nwords; w += 1024) st_out(dst + w, sym_bm[w]);
    }

    // exclusive prefix of the word popcounts (WPT consecutive words per thread)
    int c[WPT];
    popc_words<WPT>(sym_bm, tid * WPT, nwords, c);
    int mine = 0;
#pragma unroll
    for (int j = 0; j < WPT; ++j) mine += c[j];
    int total;
    int run = team_exclusive_scan<1024>(mine, scratch, total);  // entries before my first word
    // Windows: word w belongs to window floor(before(w) / wcut), where
    // before(w) counts the entries in words < w.  Consecutive words differ by
    // at most 32 <= wcut entries, so window indices run 0..K-1 without gaps,
    // every window has a first word, and each holds at most wcut + 31 entries.
    const int last_before = total - __popc(sym_bm[nwords - 1]);
    int K = (wins && total > 0) ? last_before / wcut + 1 : 0;
    if (K > kMaxWindowsPerSpan) {  // wcut too small for this span width
      if (tid == 0) atomicCAS((unsigned long long*)&counters[kError], 0ull, 31ull);
      K = 0;
    }
    if (tid == 0) {
      wstart[0] = 0;
      wrank[0] = 0;
    }
    // kcur = the window of the word before the current one; one division
    // per thread, then a comparison per word (a word adds at most 32 <= wcut
    // entries, so it crosses at most one multiple of wcut)
    int kcur = 0, nextb = wcut;
    if (tid * WPT > 0 && tid * WPT < nwords) {
      kcur = (run - __popc(sym_bm[tid * WPT - 1])) / wcut;
      nextb = (kcur + 1) * wcut;
    }
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      const int w = tid * WPT + j;
      if (w > 0 && w < nwords && run >= nextb) {  // word w opens window kcur + 1
        ++kcur;
        nextb += wcut;
        if (kcur < K) {
          wstart[kcur] = w;
          wrank[kcur] = run;
        }
      }
      run += c[j];
    }
    if (tid == 0) {
      long long b = -1;
      if (K > 0) {
        b = (long long)atomicAdd((unsigned long long*)&counters[kUnits], (unsigned long long)K);
        if (b + K > win_cap) {
          atomicCAS((unsigned long long*)&counters[kError], 0ull, 30ull);
          b = -1;
        }
      }
      wbase = b;
      if (span_wins) span_wins[h * spans + sp] = make_int2((int)(b >= 0 ? b : 0), b >= 0 ? K : 0);
    }
    __syncthreads();
    if (tid < K && wbase >= 0) {
      Window wd;
      wd.h = (int32_t)h;
      wd.span = (int32_t)sp;
      wd.w_lo = wstart[tid];
      wd.w_hi = tid + 1 < K ? wstart[tid + 1] : nwords;
      wd.rank = wrank[tid];
      wd.count = (tid + 1 < K ? wrank[tid + 1] : total) - wrank[tid];
      wins[wbase + tid] = wd;
    }
    if (tid == 0) {
      span_counts[h * spans + sp] = total;
      if (total) atomicAdd((unsigned long long*)&nnz[i], (unsigned long long)total);
    }
    for (int w = tid; w < nwords; w += 1024) sym_bm[w] = 0u;  // every read of them is done
    __syncthreads();
  }
}

// Flags (counters[kUnsorted] > 0) when some row of B has a column smaller
// than its predecessor in the same row; when no row does, window passes may
// search B rows instead of filtering them.  One warp per row of B.
__global__ void __launch_bounds__(256) k_check_sorted(DevCSR B, int64_t* counters) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  int bad = 0;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < B.nrows;
       r += nwarps) {
    const int64_t q1 = row_end(B, r);
    for (int64_t q = B.rp[r] + lane; q + 1 < q1; q += 32) bad |= B.col[q + 1] < B.col[q] ? 1 : 0;
  }
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) atomicAdd((unsigned long long*)&counters[kUnsorted], 1ull);
}

template <class K>
void set_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

inline int capped(int64_t want, int64_t cap) {
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

}  // namespace

void launch_check_sorted(const DevCSR& B, int64_t* counters, cudaStream_t s, int sms) {
  if (B.nrows == 0) return;
  int64_t g = (B.nrows + 7) / 8;
  k_check_sorted<<<(int)(g < sms * 8 ? g : sms * 8), 256, 0, s>>>(B, counters);
}

void prepare_symbolic_dev() {
  constexpr int CTA = 512, TEAM = 512, TBL = 2 * kSymLargeMax;
  set_smem(k_sym_hash<CTA, TEAM, TBL>, TBL * sizeof(int));
  set_smem(k_sym_bitmap, (size_t)kSpanWords * sizeof(unsigned) + 1024 * PieceSmem::kBytesPerThread);
}

void launch_symbolic_dev(const DevCSR& A, const DevCSR& B, const int32_t* perm, int64_t* counters,
                         const int64_t* flops, int64_t* nnz, int32_t* span_counts, int2* span_wins,
                         int wcut, Window* wins, int64_t win_cap, cudaStream_t s, int sms) {
  const int64_t m = A.nrows;
  if (m == 0) return;
  {  // heavy rows (bitmaps, rank windows), count and B's sortedness read on the device
    const int64_t spans = (B.ncols + kSpanCols - 1) / kSpanCols;
    const int64_t width = B.ncols < kSpanCols ? B.ncols : kSpanCols;
    const size_t bm_words = (size_t)((width + 31) / 32);
    const size_t smem = ((bm_words + 3) & ~(size_t)3) * sizeof(unsigned) + 1024 * PieceSmem::kBytesPerThread;
    k_sym_bitmap<<<sms * 2, 1024, smem, s>>>(A, B, perm, 0, spans, flops, wcut, nnz, span_counts,
                                             span_wins, wins, win_cap, nullptr, -1, counters);
  }
  const int64_t* dc = counters + kCntSym;
  {
    constexpr int CTA = 256, TEAM = 32, TBL = 2 * kSymWarpMax;
    const size_t smem = (CTA / TEAM) * TBL * sizeof(int);
    k_sym_hash<CTA, TEAM, TBL><<<capped((m + 7) / 8, sms * 8), CTA, smem, s>>>(A, B, perm, 0, flops,
                                                                              nnz, dc, kSymWarp);
  }
  {
    constexpr int CTA = 256, TEAM = 256, TBL = 2 * kSymSmallMax;
    k_sym_hash<CTA, TEAM, TBL><<<capped(m, sms * 8), CTA, TBL * sizeof(int), s>>>(A, B, perm, 0, flops,
                                                                                 nnz, dc, kSymSmall);
  }
  {  // shared-memory attribute set by prepare_symbolic_dev
    constexpr int CTA = 512, TEAM = 512, TBL = 2 * kSymLargeMax;
    const size_t smem = TBL * sizeof(int);
    k_sym_hash<CTA, TEAM, TBL><<<capped(m, sms * 4), CTA, smem, s>>>(A, B, perm, 0, flops, nnz, dc,
                                                                    kSymLarge);
  }
}

void launch_symbolic(const DevCSR& A, const DevCSR& B, const int32_t* perm,
                     const int64_t* seg_begin, const int64_t* seg_count, const int64_t* flops,
                     int64_t* nnz, int32_t* span_counts, int2* span_wins, int wcut,
                     Window* wins, int64_t win_cap, unsigned* hbits, int b_sorted,
                     int64_t* counters, cudaStream_t s, int sms, int* launches) {
  if (seg_count[kSymWarp]) {
    constexpr int CTA = 256, TEAM = 32, TBL = 2 * kSymWarpMax;
    const size_t smem = (CTA / TEAM) * TBL * sizeof(int);
    k_sym_hash<CTA, TEAM, TBL><<<capped((seg_count[kSymWarp] + 7) / 8, sms * 8), CTA, smem, s>>>(
        A, B, perm + seg_begin[kSymWarp], seg_count[kSymWarp], flops, nnz);
    ++*launches;
  }
  if (seg_count[kSymSmall]) {
    constexpr int CTA = 256, TEAM = 256, TBL = 2 * kSymSmallMax;
    const size_t smem = TBL * sizeof(int);
    k_sym_hash<CTA, TEAM, TBL><<<capped(seg_count[kSymSmall], sms * 8), CTA, smem, s>>>(
        A, B, perm + seg_begin[kSymSmall], seg_count[kSymSmall], flops, nnz);
    ++*launches;
  }
  if (seg_count[kSymLarge]) {
    constexpr int CTA = 512, TEAM = 512, TBL = 2 * kSymLargeMax;
    const size_t smem = TBL * sizeof(int);
    set_smem(k_sym_hash<CTA, TEAM, TBL>, smem);
    k_sym_hash<CTA, TEAM, TBL><<<capped(seg_count[kSymLarge], sms * 4), CTA, smem, s>>>(
        A, B, perm + seg_begin[kSymLarge], seg_count[kSymLarge], flops, nnz);
    ++*launches;
  }
  if (seg_count[kSymHeavy]) {
    const int64_t spans = (B.ncols + kSpanCols - 1) / kSpanCols;
    const int64_t width = B.ncols < kSpanCols ? B.ncols : kSpanCols;
    const size_t bm_words = (size_t)((width + 31) / 32);
    const size_t smem = ((bm_words + 3) & ~(size_t)3) * sizeof(unsigned) + 1024 * PieceSmem::kBytesPerThread;
    set_smem(k_sym_bitmap, smem);
    k_sym_bitmap<<<capped(seg_count[kSymHeavy] * spans, (int64_t)sms * 2), 1024, smem, s>>>(
        A, B, perm + seg_begin[kSymHeavy], seg_count[kSymHeavy], spans, flops, wcut, nnz,
        span_counts, span_wins, wins, win_cap, hbits, b_sorted, counters);
    ++*launches;
  }
}

CB_CHECK_READER(symbolic)

}  // namespace cb
