// K3: symbolic phase (paper Sec. 4.1, phase (2): the pattern of C is found
// from the input patterns alone, which sizes C before any value is formed).  nnz(C_i) = |union over stored A(i,p) of cols(B(p,:))|.
//
// Rows are processed by tier of u_i = min(flops_i, ncols):
//   * u <= 128:  one warp per row, insert-only hash of 2^ceil(log2 2u) keys
//   * u <= 1024: one 256-thread team per row, same table shape
//   * u <= 4096: one 1024-thread team per row
//   * heavier:   dense bitmap of the row's columns, one CTA per (row, slice
//                of 2^20 columns); popcounts are also recorded per numeric
//                column slice so the numeric phase can place its output.
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
                                                  int64_t* nnz) {
  extern __shared__ int sym_keys[];
  __shared__ int block_count;
  constexpr int TEAMS = CTA / TEAM;
  const int team = threadIdx.x / TEAM, lane = threadIdx.x % TEAM;
  int* keys = sym_keys + team * TABLE_MAX;
  for (int64_t r = (int64_t)blockIdx.x * TEAMS + team; r < nrows_tier;
       r += (int64_t)gridDim.x * TEAMS) {
    const int i = rows[r];
    const int64_t f = flops[i];
    const int64_t u = min(f, B.ncols);
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
      const int64_t b1 = B.rp[k + 1];
      for (int64_t q = B.rp[k] + gq; q < b1; q += G) {
        bool ins;
        probe_insert(keys, mask, shift, B.col[q], ins);
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

// Heavy rows: one CTA per (heavy row h, symbolic slice ss) unit.  The bitmap
// covers columns [lo, hi) of the slice; counts are recorded per numeric
// slice of wnum columns (wnum divides kSymSliceBits and is a multiple of 32).
__global__ void __launch_bounds__(1024) k_sym_heavy(DevCSR A, DevCSR B, const int32_t* heavy_rows,
                                                    int64_t n_heavy, int64_t sym_slices,
                                                    const int64_t* flops, int64_t wnum,
                                                    int64_t num_slices, int64_t* nnz,
                                                    int32_t* slice_counts) {
  extern __shared__ unsigned sym_bm[];
  __shared__ int total;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t units = n_heavy * sym_slices;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t h = u / sym_slices, ss = u - h * sym_slices;
    const int i = heavy_rows[h];
    const int64_t lo = ss * (int64_t)kSymSliceBits;
    const int64_t hi = min(lo + (int64_t)kSymSliceBits, B.ncols);
    const unsigned width = (unsigned)(hi - lo);
    const int nwords = (int)((width + 31) / 32);
    for (int w = tid; w < nwords; w += 1024) sym_bm[w] = 0u;
    if (tid == 0) total = 0;
    __syncthreads();
    const int64_t a0 = A.rp[i], a1 = A.rp[i + 1];
    const int gl = group_log2<1024>(flops[i], a1 - a0);
    const int G = 1 << gl, gq = tid & (G - 1), groups = 1024 >> gl;
    for (int64_t p = a0 + (tid >> gl); p < a1; p += groups) {
      const int k = A.col[p];
      const int64_t b1 = B.rp[k + 1];
      for (int64_t q = B.rp[k] + gq; q < b1; q += G) {
        const unsigned off = (unsigned)((int64_t)B.col[q] - lo);
        if (off < width) {
          const unsigned bit = 1u << (off & 31);
          if (!(sym_bm[off >> 5] & bit)) atomicOr(&sym_bm[off >> 5], bit);
        }
      }
    }
    __syncthreads();
    const int64_t s0 = lo / wnum;
    const int nsub = (int)((width + wnum - 1) / wnum);
    const int wpw = (int)(wnum / 32);
    for (int t = warp; t < nsub; t += 32) {
      int c = 0;
      const int wend = min((t + 1) * wpw, nwords);
      for (int w = t * wpw + lane; w < wend; w += 32) c += __popc(sym_bm[w]);
      c = __reduce_add_sync(0xffffffffu, c);
      if (lane == 0) {
        slice_counts[h * num_slices + s0 + t] = c;
        if (c) atomicAdd(&total, c);
      }
    }
    __syncthreads();
    if (tid == 0 && total) atomicAdd((unsigned long long*)&nnz[i], (unsigned long long)total);
    __syncthreads();
  }
}

template <class K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

inline int capped(int64_t want, int64_t cap) {
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

}  // namespace

void launch_symbolic(const DevCSR& A, const DevCSR& B, const int32_t* perm,
                     const int64_t* seg_begin, const int64_t* seg_count, const int64_t* flops,
                     int64_t* nnz, int32_t* slice_counts, int64_t num_slice_w,
                     int64_t num_slices, cudaStream_t s, int sms, int* launches) {
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
    constexpr int CTA = 1024, TEAM = 1024, TBL = 2 * kSymHashMax;
    const size_t smem = TBL * sizeof(int);
    set_smem(k_sym_hash<CTA, TEAM, TBL>, smem);
    k_sym_hash<CTA, TEAM, TBL><<<capped(seg_count[kSymLarge], sms * 2), CTA, smem, s>>>(
        A, B, perm + seg_begin[kSymLarge], seg_count[kSymLarge], flops, nnz);
    ++*launches;
  }
  if (seg_count[kSymHeavy]) {
    const int64_t ncols = B.ncols;
    const int64_t sym_slices = (ncols + kSymSliceBits - 1) / kSymSliceBits;
    const int64_t width = ncols < kSymSliceBits ? ncols : kSymSliceBits;
    const size_t smem = (size_t)((width + 31) / 32) * sizeof(unsigned);
    set_smem(k_sym_heavy, smem);
    const int per_sm = smem <= 64 * 1024 ? 2 : 1;
    k_sym_heavy<<<capped(seg_count[kSymHeavy] * sym_slices, (int64_t)sms * per_sm), 1024, smem, s>>>(
        A, B, perm + seg_begin[kSymHeavy], seg_count[kSymHeavy], sym_slices, flops, num_slice_w,
        num_slices, nnz, slice_counts);
    ++*launches;
  }
}

}  // namespace cb
