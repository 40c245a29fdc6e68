// Semiring SpMSpV, row form for CSR matrices: y^T = x^T A, i.e.
//   y_c = (+) over stored x entries (i, x_i) and stored A(i, c) of x_i (x) A(i, c)
// (paper Sec. 4.3: SpMSpV merges the matrix lines selected by the vector's
// nonzeros; Sec. 4.5 compares its accumulators).  The GPU form is a push
// into a dense accumulator (the SPA of Sec. 4.3) that lives in device memory
// across calls:
//   K1  per x entry: the number of 256-product chunks of its A row;
//   K2  exclusive scan of those counts (k_rows.cu);
//   K3  every warp takes chunks (one binary search over the chunk prefix per
//       chunk), its lanes read the chunk's A entries coalesced and combine
//       x_i (x) A(i, c) into spa[c] with the semiring's atomic in L2, setting
//       bit c of a touched-bitmap;
//   K4  popcounts of the bitmap words, scanned (k_rows.cu), give nnz(y) and
//       each word's output offset;
//   K5  every touched entry is written in column order and its SPA slot and
//       bitmap word are reset, so the next call starts clean without an O(n)
//       initialisation.
// The bucket form (Sec. 4.3: the column-partitioned SpMSpV merges through
// buckets that block y, i.e. propagation blocking) keeps no O(n) state:
//   B1  products per bucket of kBucketCols output columns (lanes of one
//       bucket counted together; per-CTA counters in shared memory when the
//       buckets fit, then a scan over CTAs), scanned into bucket offsets;
//   B2  every product (c, x_i (x) A(i, c)) is appended to its bucket (from
//       its CTA's own block of the bucket);
//   B3  one CTA per bucket (+)-combines the bucket's products in a shared-
//       memory accumulator with a touched bitmap and writes the bucket's
//       entries, in column order, to a staging area at the bucket's offset,
//       and the bucket's entry count;
//   B4  after a scan of the counts, each bucket's entries are copied to y.
#include "cb_common.cuh"
#include "cb_kernels.h"

namespace cb {
namespace {

constexpr int kChunk = 256;

// K1.  An index outside [0, A.nrows) gets no chunks and sets *err.
__global__ void __launch_bounds__(256) k_spmspv_chunks(DevCSR A, const int32_t* x_idx, int64_t nx,
                                                      int64_t* chunks, int64_t* err) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nx;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int i = x_idx[p];
    if (i < 0 || (int64_t)i >= A.nrows) {
      chunks[p] = 0;
      atomicMax(reinterpret_cast<unsigned long long*>(err), 1ull);
      continue;
    }
    const int64_t len = A.rp[i + 1] - A.rp[i];
    chunks[p] = (len + kChunk - 1) / kChunk;
  }
}

template <int SR>
__global__ void __launch_bounds__(256) k_spa_init(typename Sem<SR>::A* spa, int64_t n) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    spa[c] = Sem<SR>::ident();
}

// K3.  cpre[p] = first chunk of x entry p, cpre[nx] = number of chunks.
template <int SR>
__global__ void __launch_bounds__(256) k_spmspv_push(DevCSR A, const int32_t* x_idx,
                                                    const typename Sem<SR>::TA* x_val, int64_t nx,
                                                    const int64_t* cpre, typename Sem<SR>::A* spa,
                                                    unsigned* touched) {
  typedef Sem<SR> S;
  typedef typename S::TA TA;
  typedef typename S::TB TB;
  const int lane = threadIdx.x & 31;
  const int64_t total = cpre[nx];
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const TB* Aval = reinterpret_cast<const TB*>(A.val);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < total; w += nwarps) {
    // x entry owning chunk w: the last p with cpre[p] <= w
    int64_t lo = 0, hi = nx - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (__ldg(cpre + mid) <= w) lo = mid;
      else hi = mid - 1;
    }
    const int64_t p = lo;
    const int i = __ldg(x_idx + p);
    const TA xv = S::kUsesA ? ldg_val(x_val + p) : TA();
    const int64_t r0 = __ldg(A.rp + i), r1 = __ldg(A.rp + i + 1);
    const int64_t q0 = r0 + (w - __ldg(cpre + p)) * kChunk;
    const int64_t q1 = min(q0 + kChunk, r1);
    for (int64_t q = q0 + lane; q < q1; q += 32) {
      const int c = __ldg(A.col + q);
      S::atomic(&spa[c], S::mul(xv, ldg_val(Aval + q)));
      const unsigned bit = 1u << (c & 31);
      if (!(touched[c >> 5] & bit)) atomicOr(&touched[c >> 5], bit);
    }
  }
}

__global__ void __launch_bounds__(256) k_word_popc(const unsigned* touched, int64_t nw, int64_t* cnt) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw;
       w += (int64_t)gridDim.x * blockDim.x)
    cnt[w] = __popc(touched[w]);
}

// K5: entries of word w go to out + wpre[w], in column order; SPA and
// bitmap are reset.  Nothing is written past cap (the caller's capacity).
template <int SR>
__global__ void __launch_bounds__(256) k_spmspv_compact(unsigned* touched, int64_t nw,
                                                       const int64_t* wpre,
                                                       typename Sem<SR>::A* spa, int32_t* y_idx,
                                                       typename Sem<SR>::TC* y_val, int64_t cap) {
  typedef Sem<SR> S;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw;
       w += (int64_t)gridDim.x * blockDim.x) {
    unsigned word = touched[w];
    if (!word) continue;
    int64_t o = wpre[w];
    while (word) {
      const int b = __ffs(word) - 1;
      word &= word - 1;
      const int64_t c = 32 * w + b;
      if (o < cap) {
        y_idx[o] = (int32_t)c;
        y_val[o] = S::out(spa[c]);
      }
      spa[c] = S::ident();
      ++o;
    }
    touched[w] = 0u;
  }
}

constexpr int kBucketLog = 10;
constexpr int kBucketCols = 1 << kBucketLog;  // output columns per bucket

// The x entry owning chunk w: the last p with cpre[p] <= w.
__device__ __forceinline__ int64_t chunk_owner(const int64_t* cpre, int64_t nx, int64_t w) {
  int64_t lo = 0, hi = nx - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (__ldg(cpre + mid) <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// B1 (PASS 0) and B2 (PASS 1): every warp takes chunks; in each step of 32
// products the lanes of one bucket are counted together (one atomic per
// bucket and step).  PASS 1 appends (column, product) to the bucket at the
// slot taken from cur[bucket].
template <int SR, int PASS>
__global__ void __launch_bounds__(256) k_bucket_fill(DevCSR A, const int32_t* x_idx,
                                                    const typename Sem<SR>::TA* x_val, int64_t nx,
                                                    const int64_t* cpre,
                                                    unsigned long long* cur, int32_t* bcol,
                                                    typename Sem<SR>::A* bval) {
  typedef Sem<SR> S;
  typedef typename S::TA TA;
  typedef typename S::TB TB;
  const int lane = threadIdx.x & 31;
  const int64_t total = cpre[nx];
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const TB* Aval = reinterpret_cast<const TB*>(A.val);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < total; w += nwarps) {
    const int64_t p = chunk_owner(cpre, nx, w);
    const int i = __ldg(x_idx + p);
    const int64_t r0 = __ldg(A.rp + i), r1 = __ldg(A.rp + i + 1);
    const int64_t q0 = r0 + (w - __ldg(cpre + p)) * kChunk;
    const int64_t q1 = min(q0 + kChunk, r1);
    const TA xv = (PASS == 1 && S::kUsesA) ? ldg_val(x_val + p) : TA();
    for (int64_t base = q0; base < q1; base += 32) {  // uniform over the warp
      const int64_t q = base + lane;
      const bool v = q < q1;
      const int c = v ? __ldg(A.col + q) : 0;
      const int b = v ? (c >> kBucketLog) : -1;
      const unsigned same = __match_any_sync(0xffffffffu, b);
      const int leader = __ffs(same) - 1;
      unsigned long long slot = 0;
      if (v && lane == leader) slot = atomicAdd(cur + b, (unsigned long long)__popc(same));
      slot = __shfl_sync(0xffffffffu, slot, leader);
      if (PASS == 1 && v) {
        const unsigned long long at = slot + __popc(same & ((1u << lane) - 1u));
        bcol[at] = c;
        bval[at] = S::mul(xv, ldg_val(Aval + q));
      }
    }
  }
}

// B1/B2 with per-CTA bucket counters in shared memory (nb <= kPrivBuckets):
// PASS 0 counts each CTA's products per bucket into ccnt[b][cta]; after a
// scan over CTAs (k_bucket_cta_scan) PASS 1 places them from the CTA's own
// block of each bucket, so no global atomic is taken per product.  Both
// passes give every CTA the same chunks (same grid).
constexpr int kPrivBuckets = 2048;

template <int SR, int PASS>
__global__ void __launch_bounds__(256) k_bucket_fill_priv(DevCSR A, const int32_t* x_idx,
                                                         const typename Sem<SR>::TA* x_val, int64_t nx,
                                                         const int64_t* cpre, int64_t nb,
                                                         int64_t* ccnt, const int64_t* bpre,
                                                         int32_t* bcol, typename Sem<SR>::A* bval) {
  typedef Sem<SR> S;
  typedef typename S::TA TA;
  typedef typename S::TB TB;
  __shared__ long long s_base[kPrivBuckets];
  __shared__ unsigned s_rel[kPrivBuckets];
  for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) {
    s_rel[b] = 0u;
    s_base[b] = PASS == 1 ? bpre[b] + ccnt[b * (int64_t)gridDim.x + blockIdx.x] : 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t total = cpre[nx];
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const TB* Aval = reinterpret_cast<const TB*>(A.val);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < total; w += nwarps) {
    const int64_t p = chunk_owner(cpre, nx, w);
    const int i = __ldg(x_idx + p);
    const int64_t r0 = __ldg(A.rp + i), r1 = __ldg(A.rp + i + 1);
    const int64_t q0 = r0 + (w - __ldg(cpre + p)) * kChunk;
    const int64_t q1 = min(q0 + kChunk, r1);
    const TA xv = (PASS == 1 && S::kUsesA) ? ldg_val(x_val + p) : TA();
    for (int64_t base = q0; base < q1; base += 32) {  // uniform over the warp
      const int64_t q = base + lane;
      const bool v = q < q1;
      const int c = v ? __ldg(A.col + q) : 0;
      const int b = v ? (c >> kBucketLog) : -1;
      const unsigned same = __match_any_sync(0xffffffffu, b);
      const int leader = __ffs(same) - 1;
      unsigned rel = 0;
      if (v && lane == leader) rel = atomicAdd(&s_rel[b], (unsigned)__popc(same));
      rel = __shfl_sync(0xffffffffu, rel, leader);
      if (PASS == 1 && v) {
        const long long at = s_base[b] + rel + __popc(same & ((1u << lane) - 1u));
        bcol[at] = c;
        bval[at] = S::mul(xv, ldg_val(Aval + q));
      }
    }
  }
  if (PASS == 0) {
    __syncthreads();
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) ccnt[b * (int64_t)gridDim.x + blockIdx.x] = s_rel[b];
  }
}

// ccnt[b][c] becomes the exclusive prefix over CTAs c of bucket b's counts;
// tot[b] the bucket's total.  One warp per bucket.
__global__ void __launch_bounds__(256) k_bucket_cta_scan(int64_t* ccnt, int64_t nb, int ncta,
                                                        int64_t* tot) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += nwarps) {
    int64_t* row = ccnt + b * ncta;
    long long run = 0;
    for (int c0 = 0; c0 < ncta; c0 += 32) {  // uniform over the warp
      const int c = c0 + lane;
      const long long v = c < ncta ? row[c] : 0;
      long long inc = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
      }
      if (c < ncta) row[c] = run + inc - v;
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) tot[b] = run;
  }
}

// B3: one CTA (256 threads) per bucket (kBucketCols = 1024 columns: 32
// words of bitmap, one warp scans them).
template <int SR>
__global__ void __launch_bounds__(256) k_bucket_reduce(const int64_t* bpre, int64_t nb, int64_t n,
                                                      const int32_t* bcol,
                                                      const typename Sem<SR>::A* bval,
                                                      int32_t* scol, typename Sem<SR>::TC* sval,
                                                      int64_t* bnnz) {
  typedef Sem<SR> S;
  typedef typename S::A Acc;
  __shared__ Acc acc[kBucketCols];
  __shared__ unsigned bits[kBucketCols / 32];
  __shared__ int wscan[kBucketCols / 32 + 1];
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    for (int t = threadIdx.x; t < kBucketCols; t += blockDim.x) acc[t] = S::ident();
    for (int t = threadIdx.x; t < kBucketCols / 32; t += blockDim.x) bits[t] = 0u;
    __syncthreads();
    const int64_t e0 = bpre[b], e1 = bpre[b + 1];
    const int64_t lo = b << kBucketLog;
    constexpr int UR = 4;  // entries per thread per iteration, loaded before any is combined
    for (int64_t e = e0 + threadIdx.x; e < e1; e += (int64_t)UR * blockDim.x) {
      int oc[UR];
      Acc ov[UR];
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        const int64_t eu = e + (int64_t)u * blockDim.x;
        oc[u] = eu < e1 ? (int)(__ldg(bcol + eu) - lo) : -1;
        ov[u] = eu < e1 ? bval[eu] : S::ident();
      }
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        if (oc[u] < 0) continue;
        const int o = oc[u];
        S::atomic(&acc[o], ov[u]);
        const unsigned bit = 1u << (o & 31);
        if (!(bits[o >> 5] & bit)) atomicOr(&bits[o >> 5], bit);
      }
    }
    __syncthreads();
    // word offsets: exclusive scan of the 128 word popcounts (thread t < 128)
    constexpr int NWD = kBucketCols / 32;
    if (threadIdx.x < 32) {
      int run = 0;
      int cnt[NWD / 32];
#pragma unroll
      for (int j = 0; j < NWD / 32; ++j) {
        cnt[j] = __popc(bits[threadIdx.x * (NWD / 32) + j]);
        run += cnt[j];
      }
      int inc = run;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, d);
        if ((int)threadIdx.x >= d) inc += y;
      }
      int off = inc - run;
#pragma unroll
      for (int j = 0; j < NWD / 32; ++j) {
        wscan[threadIdx.x * (NWD / 32) + j] = off;
        off += cnt[j];
      }
      if (threadIdx.x == 31) wscan[NWD] = inc;
    }
    __syncthreads();
    // the bucket's entries in column order at the staging offset e0
    for (int wd = threadIdx.x; wd < NWD; wd += blockDim.x) {
      unsigned word = bits[wd];
      int64_t o = e0 + wscan[wd];
      while (word) {
        const int bt = __ffs(word) - 1;
        word &= word - 1;
        const int c = wd * 32 + bt;
        scol[o] = (int32_t)(lo + c);
        sval[o] = S::out(acc[c]);
        ++o;
      }
    }
    if (threadIdx.x == 0) bnnz[b] = wscan[NWD];
    (void)n;
    __syncthreads();
  }
}

// B4: bucket b's staged entries [bpre[b], bpre[b] + bnnz[b]) to y at ypre[b].
template <int SR>
__global__ void __launch_bounds__(256) k_bucket_copy(const int64_t* bpre, const int64_t* bnnz,
                                                    const int64_t* ypre, int64_t nb,
                                                    const int32_t* scol,
                                                    const typename Sem<SR>::TC* sval,
                                                    int32_t* y_idx, typename Sem<SR>::TC* y_val,
                                                    int64_t cap) {
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const int64_t s0 = bpre[b], cnt = bnnz[b], d0 = ypre[b];
    for (int64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
      if (d0 + t < cap) {
        y_idx[d0 + t] = scol[s0 + t];
        y_val[d0 + t] = sval[s0 + t];
      }
    }
  }
}

inline unsigned grid_of(int64_t n, int threads, int cap) {
  const int64_t g = (n + threads - 1) / threads;
  return (unsigned)(g < 1 ? 1 : (g < cap ? g : cap));
}

template <int SR>
void spmspv_sr(int step, const DevCSR& A, const int32_t* x_idx, const void* x_val, int64_t nx,
               int64_t* chunks, const int64_t* cpre, void* spa, unsigned* touched, int64_t n,
               int64_t* wcnt, const int64_t* wpre, int32_t* y_idx, void* y_val, int64_t cap,
               int64_t* err, cudaStream_t s, int sms) {
  typedef typename Sem<SR>::A Acc;
  typedef typename Sem<SR>::TA TA;
  typedef typename Sem<SR>::TC TC;
  const int64_t nw = (n + 31) / 32;
  switch (step) {
    case 0:
      k_spa_init<SR><<<grid_of(n, 256, sms * 8), 256, 0, s>>>(static_cast<Acc*>(spa), n);
      break;
    case 1:
      k_spmspv_chunks<<<grid_of(nx, 256, sms * 8), 256, 0, s>>>(A, x_idx, nx, chunks, err);
      break;
    case 2:
      k_spmspv_push<SR><<<sms * 8, 256, 0, s>>>(A, x_idx, static_cast<const TA*>(x_val), nx, cpre,
                                               static_cast<Acc*>(spa), touched);
      break;
    case 3:
      k_word_popc<<<grid_of(nw, 256, sms * 8), 256, 0, s>>>(touched, nw, wcnt);
      break;
    case 4:
      k_spmspv_compact<SR><<<grid_of(nw, 256, sms * 8), 256, 0, s>>>(
          touched, nw, wpre, static_cast<Acc*>(spa), y_idx, static_cast<TC*>(y_val), cap);
      break;
  }
}

template <int SR>
void bucket_sr(int step, const DevCSR& A, const int32_t* x_idx, const void* x_val, int64_t nx,
               const int64_t* cpre, unsigned long long* cur, int32_t* bcol, void* bval,
               const int64_t* bpre, int64_t nb, int64_t n, int32_t* scol, void* sval, int64_t* bnnz,
               const int64_t* ypre, int32_t* y_idx, void* y_val, int64_t cap, cudaStream_t s, int sms) {
  typedef typename Sem<SR>::A Acc;
  typedef typename Sem<SR>::TA TA;
  typedef typename Sem<SR>::TC TC;
  switch (step) {
    case 0:
      k_bucket_fill<SR, 0><<<sms * 8, 256, 0, s>>>(A, x_idx, static_cast<const TA*>(x_val), nx, cpre,
                                                   cur, nullptr, nullptr);
      break;
    case 1:
      k_bucket_fill<SR, 1><<<sms * 8, 256, 0, s>>>(A, x_idx, static_cast<const TA*>(x_val), nx, cpre,
                                                   cur, bcol, static_cast<Acc*>(bval));
      break;
    case 2:
      k_bucket_reduce<SR><<<grid_of(nb, 1, sms * 4), 256, 0, s>>>(
          bpre, nb, n, bcol, static_cast<const Acc*>(bval), scol, static_cast<TC*>(sval), bnnz);
      break;
    case 3:
      k_bucket_copy<SR><<<grid_of(nb, 1, sms * 8), 256, 0, s>>>(
          bpre, bnnz, ypre, nb, scol, static_cast<const TC*>(sval), y_idx, static_cast<TC*>(y_val), cap);
      break;
  }
}

}  // namespace

int64_t spmspv_buckets(int64_t n) { return (n + kBucketCols - 1) / kBucketCols; }

int spmspv_priv_ctas(int64_t nb, int sms) { return nb <= kPrivBuckets ? sms * 4 : 0; }

void launch_spmspv_bucket_priv(int sr, int pass, const DevCSR& A, const int32_t* x_idx,
                               const void* x_val, int64_t nx, const int64_t* cpre, int64_t nb,
                               int64_t* ccnt, const int64_t* bpre, int64_t* tot, int32_t* bcol,
                               void* bval, cudaStream_t s, int sms) {
  const int ncta = spmspv_priv_ctas(nb, sms);
  if (pass == 2) {
    k_bucket_cta_scan<<<grid_of(nb, 8, sms * 4), 256, 0, s>>>(ccnt, nb, ncta, tot);
    return;
  }
  switch (sr) {
#define CB_CASE(SRV)                                                                               \
  case SRV:                                                                                        \
    if (pass == 0)                                                                                 \
      k_bucket_fill_priv<SRV, 0><<<ncta, 256, 0, s>>>(                                             \
          A, x_idx, static_cast<const Sem<SRV>::TA*>(x_val), nx, cpre, nb, ccnt, bpre, nullptr,  \
          nullptr);                                                                                \
    else                                                                                           \
      k_bucket_fill_priv<SRV, 1><<<ncta, 256, 0, s>>>(                                             \
          A, x_idx, static_cast<const Sem<SRV>::TA*>(x_val), nx, cpre, nb, ccnt, bpre, bcol,     \
          static_cast<Sem<SRV>::A*>(bval));                                                        \
    break;
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
  }
}

void launch_spmspv_bucket_step(int sr, int step, const DevCSR& A, const int32_t* x_idx,
                               const void* x_val, int64_t nx, const int64_t* cpre,
                               unsigned long long* cur, int32_t* bcol, void* bval, const int64_t* bpre,
                               int64_t nb, int64_t n, int32_t* scol, void* sval, int64_t* bnnz,
                               const int64_t* ypre, int32_t* y_idx, void* y_val, int64_t cap,
                               cudaStream_t s, int sms) {
  switch (sr) {
#define CB_CASE(SRV)                                                                             \
  case SRV:                                                                                      \
    bucket_sr<SRV>(step, A, x_idx, x_val, nx, cpre, cur, bcol, bval, bpre, nb, n, scol, sval, bnnz, \
                   ypre, y_idx, y_val, cap, s, sms);                                             \
    break;
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
  }
}

size_t spa_value_size(int sr) {
  switch (sr) {
#define CB_CASE(SRV) case SRV: return sizeof(Sem<SRV>::A);
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
  }
  return 0;
}

void launch_spmspv_step(int sr, int step, const DevCSR& A, const int32_t* x_idx, const void* x_val,
                        int64_t nx, int64_t* chunks, const int64_t* cpre, void* spa,
                        unsigned* touched, int64_t n, int64_t* wcnt, const int64_t* wpre,
                        int32_t* y_idx, void* y_val, int64_t cap, int64_t* err, cudaStream_t s,
                        int sms) {
#define CB_SPV(SRV)                                                                           \
  spmspv_sr<SRV>(step, A, x_idx, x_val, nx, chunks, cpre, spa, touched, n, wcnt, wpre, y_idx, \
                 y_val, cap, err, s, sms)
  switch (sr) {
#define CB_CASE(SRV) case SRV: CB_SPV(SRV); break;
    CB_FOR_EACH_SEMIRING(CB_CASE)
#undef CB_CASE
  }
#undef CB_SPV
}

}  // namespace cb
