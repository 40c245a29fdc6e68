// Stacking kernels for batched SpGEMM: many independent products C_i = A_i B_i
// are laid out as one block-diagonal product.  A_i's rows are appended to a
// stacked A whose column indices are shifted by the first stacked row of
// B_i; B_i's rows are appended to a stacked B that keeps B_i's own column
// indices.  Every row of the stacked A therefore only meets rows of its own
// B_i, and the stacked C holds C_i's rows, in order, with local columns.
#include "cb_common.cuh"
#include "cb_kernels.h"

namespace cb {
namespace {

// One product's part of the stacked operand.
struct StackPart {
  const int64_t* rp;   // source row pointers (nrows + 1)
  const int32_t* col;  // source columns
  const void* val;     // source values
  int64_t nrows, row_off, nnz_off;
  int32_t col_add;     // added to every column (row offset of B_i in the stacked B for A)
  int32_t width;       // output width of the part's rows (k_i)
};

// blockIdx.y = part; x-blocks stride over the part's rows and entries.  The
// last part also writes the closing row pointer.
template <class T>
__global__ void __launch_bounds__(256) k_stack(const StackPart* parts, int nparts, int64_t* rp_out,
                                               int32_t* col_out, T* val_out, int32_t* rcols_out) {
  const StackPart pt = parts[blockIdx.y];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t base = pt.rp[0];
  for (int64_t r = t0; r < pt.nrows; r += stride) {
    rp_out[pt.row_off + r] = pt.nnz_off + pt.rp[r] - base;
    if (rcols_out) rcols_out[pt.row_off + r] = pt.width;
  }
  const int64_t nnz = pt.rp[pt.nrows] - base;
  if (t0 == 0 && (int)blockIdx.y == nparts - 1) rp_out[pt.row_off + pt.nrows] = pt.nnz_off + nnz;
  const T* src = static_cast<const T*>(pt.val) + base;
  for (int64_t q = t0; q < nnz; q += stride) {
    col_out[pt.nnz_off + q] = pt.col[base + q] + pt.col_add;
    val_out[pt.nnz_off + q] = src[q];
  }
}

// Selector of the merge: row i holds k entries, at columns l*m + i
// (l = 0..k-1) with the semiring's multiplicative identity, so that
// (selector (+).(x) [P_0; ...; P_{k-1}]) = P_0 (+) ... (+) P_{k-1}.
template <class T>
__global__ void __launch_bounds__(256) k_merge_selector(int64_t m, int k, int64_t* rp, int32_t* col,
                                                        T* val, T one) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    rp[i] = i * k;
    for (int l = 0; l < k; ++l) {
      col[i * k + l] = (int32_t)(l * m + i);
      val[i * k + l] = one;
    }
    if (i == m - 1) rp[m] = m * k;
  }
}

// ---------------------------------------------------------------------------
// Per-product digests of a wave's stacked output (cb_opts.digests): a check
// of transient batched outputs (graph mode included) that needs no copy of C.
//   sm(x) = splitmix64 output function;
//   D0 = sum over rows r of sm(sm(2r) + len_r)
//      + sum over entries (r, j, c, v) of sm(sm(sm(sm(2r + 1) + j) + c) + bits(v))   (mod 2^64)
//     (r the product's own row, j the position in the row, c the column,
//      bits(v) the value's bytes zero-extended; 0 for fp64, whose D0 covers
//      the pattern only);
//   D1 (fp64 only) = bits of sum over entries of v * w(r, c),
//     w(r, c) = 1 + 2^-53 (sm(sm(2r + 1) ^ c) >> 11), in compensated
//     (Neumaier) summation in a fixed order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sm64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Neumaier step: (s, c) += x.
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
  const double t = __dadd_rn(s, x);
  c = __dadd_rn(c, fabs(s) >= fabs(x) ? __dadd_rn(__dsub_rn(s, t), x) : __dadd_rn(__dsub_rn(x, t), s));
  s = t;
}

// Lane-ordered compensated combination of the warp's (s, c) pairs (lane 0
// returns the total; deterministic).
__device__ __forceinline__ double warp_neumaier_total(double s, double c) {
  double ts = 0.0, tc = 0.0;
  for (int l = 0; l < 32; ++l) {
    const double ls = __shfl_sync(0xffffffffu, s, l), lc = __shfl_sync(0xffffffffu, c, l);
    neumaier(ts, tc, ls);
    neumaier(ts, tc, lc);
  }
  return __dadd_rn(ts, tc);
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
  return x;
}

// Product of stacked row g: the last p with prow[p] <= g (prow ascending, nprod + 1 entries).
__device__ __forceinline__ int product_of_row(const int64_t* prow, int nprod, int64_t g) {
  int lo = 0, hi = nprod - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prow[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One warp per row of the wave: the row's D0 terms and its fp64 checksum.
template <class V, bool F64>
__global__ void __launch_bounds__(256) k_digest_rows(const int64_t* rp, const int32_t* col, const V* val,
                                                     int64_t m, const int64_t* prow, int nprod,
                                                     int64_t row_base, uint64_t* rdig, double* rsum) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < m; r += nwarps) {
    const int64_t g = row_base + r;
    const int p = product_of_row(prow, nprod, g);
    const uint64_t lr = (uint64_t)(g - prow[p]);  // row index within the product
    const int64_t q0 = rp[r], q1 = rp[r + 1];
    const uint64_t hr = sm64(2 * lr + 1);
    uint64_t d = 0;
    double s = 0.0, c = 0.0;
    for (int64_t q = q0 + lane; q < q1; q += 32) {
      const uint64_t cc = (uint64_t)(uint32_t)col[q];
      const V v = val[q];
      uint64_t bits = 0;
      if (!F64) memcpy(&bits, &v, sizeof(V));
      d += sm64(sm64(sm64(hr + (uint64_t)(q - q0)) + cc) + bits);
      if (F64) {
        const double w = 1.0 + (double)(sm64(hr ^ cc) >> 11) * 0x1.0p-53;
        double x;
        memcpy(&x, &v, sizeof x);
        neumaier(s, c, __dmul_rn(x, w));
      }
    }
    d = warp_sum_u64(d);
    double tot = 0.0;
    if (F64) tot = warp_neumaier_total(s, c);
    if (lane == 0) {
      rdig[r] = d + sm64(sm64(2 * lr) + (uint64_t)(q1 - q0));
      rsum[r] = tot;
    }
  }
}

// One warp per product of the wave: D0 = sum of its rows' terms, D1 the
// compensated sum of its rows' checksums in row order.
__global__ void __launch_bounds__(256) k_digest_products(const int64_t* prow, int nprod, int64_t row_base,
                                                         const uint64_t* rdig, const double* rsum, bool f64,
                                                         uint64_t* out) {
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < nprod; p += nwarps) {
    const int64_t r0 = prow[p] - row_base, r1 = prow[p + 1] - row_base;
    uint64_t d = 0;
    double s = 0.0, c = 0.0;
    for (int64_t r = r0 + lane; r < r1; r += 32) {
      d += rdig[r];
      if (f64) neumaier(s, c, rsum[r]);
    }
    d = warp_sum_u64(d);
    double tot = 0.0;
    if (f64) tot = warp_neumaier_total(s, c);  // f64 is uniform over the grid
    if (lane == 0) {
      out[2 * (int64_t)p] = d;
      uint64_t b = 0;
      if (f64) memcpy(&b, &tot, sizeof b);
      out[2 * (int64_t)p + 1] = b;
    }
  }
}

}  // namespace

void launch_digest(int vsz, bool f64, const int64_t* rp, const int32_t* col, const void* val, int64_t m,
                   const int64_t* prow, int nprod, int64_t row_base, uint64_t* rdig, double* rsum,
                   uint64_t* out, cudaStream_t s, int sms) {
  if (nprod <= 0) return;
  if (m > 0) {
    const int64_t g = (m + 7) / 8;
    const unsigned grid = (unsigned)(g < (int64_t)sms * 16 ? g : (int64_t)sms * 16);
    if (f64)
      k_digest_rows<double, true><<<grid, 256, 0, s>>>(rp, col, static_cast<const double*>(val), m, prow,
                                                       nprod, row_base, rdig, rsum);
    else if (vsz == 8)
      k_digest_rows<uint64_t, false><<<grid, 256, 0, s>>>(rp, col, static_cast<const uint64_t*>(val), m,
                                                          prow, nprod, row_base, rdig, rsum);
    else if (vsz == 4)
      k_digest_rows<uint32_t, false><<<grid, 256, 0, s>>>(rp, col, static_cast<const uint32_t*>(val), m,
                                                          prow, nprod, row_base, rdig, rsum);
    else
      k_digest_rows<uint8_t, false><<<grid, 256, 0, s>>>(rp, col, static_cast<const uint8_t*>(val), m,
                                                         prow, nprod, row_base, rdig, rsum);
  }
  const unsigned pg = (unsigned)((nprod + 7) / 8);
  k_digest_products<<<pg, 256, 0, s>>>(prow, nprod, row_base, rdig, rsum, f64, out);
}

void launch_merge_selector(int64_t m, int k, int vsz, uint64_t one_bits, int64_t* rp, int32_t* col,
                           void* val, cudaStream_t s, int sms) {
  if (m <= 0) return;
  const int64_t g = (m + 255) / 256;
  const unsigned grid = (unsigned)(g < sms * 8 ? g : sms * 8);
  switch (vsz) {
    case 8: k_merge_selector<uint64_t><<<grid, 256, 0, s>>>(m, k, rp, col, static_cast<uint64_t*>(val), one_bits); break;
    case 4: k_merge_selector<uint32_t><<<grid, 256, 0, s>>>(m, k, rp, col, static_cast<uint32_t*>(val), (uint32_t)one_bits); break;
    default: k_merge_selector<uint8_t><<<grid, 256, 0, s>>>(m, k, rp, col, static_cast<uint8_t*>(val), (uint8_t)one_bits);
  }
}

void launch_stack(const void* parts_dev, int nparts, int vsz, int64_t* rp_out, int32_t* col_out,
                  void* val_out, int32_t* rcols_out, cudaStream_t s, int sms) {
  if (nparts <= 0) return;
  dim3 grid((unsigned)(nparts < 64 ? sms * 4 : 8), (unsigned)nparts);
  const StackPart* pp = static_cast<const StackPart*>(parts_dev);
  switch (vsz) {
    case 8: k_stack<uint64_t><<<grid, 256, 0, s>>>(pp, nparts, rp_out, col_out, static_cast<uint64_t*>(val_out), rcols_out); break;
    case 4: k_stack<uint32_t><<<grid, 256, 0, s>>>(pp, nparts, rp_out, col_out, static_cast<uint32_t*>(val_out), rcols_out); break;
    default: k_stack<uint8_t><<<grid, 256, 0, s>>>(pp, nparts, rp_out, col_out, static_cast<uint8_t*>(val_out), rcols_out);
  }
}

size_t stack_part_size() { return sizeof(StackPart); }

void fill_stack_part(void* dst, const int64_t* rp, const int32_t* col, const void* val, int64_t nrows,
                     int64_t row_off, int64_t nnz_off, int32_t col_add, int32_t width) {
  StackPart* p = static_cast<StackPart*>(dst);
  p->rp = rp;
  p->col = col;
  p->val = val;
  p->nrows = nrows;
  p->row_off = row_off;
  p->nnz_off = nnz_off;
  p->col_add = col_add;
  p->width = width;
}

}  // namespace cb
