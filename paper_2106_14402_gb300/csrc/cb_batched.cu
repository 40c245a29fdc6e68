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

}  // namespace

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
