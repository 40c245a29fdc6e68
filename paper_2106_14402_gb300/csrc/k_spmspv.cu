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

}  // namespace

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
