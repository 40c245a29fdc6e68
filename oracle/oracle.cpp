// CPU oracle for the semiring SpGEMM C = A (+).(x) B -- TEST INFRASTRUCTURE ONLY.
//
// This file is the plain, slow, obviously-correct statement of what the GPU
// path computes.  Only the test suite, the smoke check and the benchmark's
// CPU-baseline leg may load it; the library's product path never does.  It
// shares no code, header, table or constant with the CUDA sources.
//
// Definition followed (paper Sec. 3.1 and Sec. 4.1):
//   * C = A B with A in S^{m x n}, B in S^{n x k}, C in S^{m x k} (Sec. 3.1).
//   * Gustavson's formulation (Sec. 4.1, multithreaded SpGEMM): output
//     line i of C is the merge of the B lines selected by the nonzeros of
//     A's line i.  The paper states it column-wise on CSC; on CSR rows the
//     same statement holds for C^T = B^T A^T, so here rows play the role of
//     the paper's columns.
//   * The pattern of C is structural (the symbolic phase of Sec. 4.1 derives
//     it from the input patterns alone): (i,j) is stored iff some stored
//     A(i,p) meets some stored B(p,j).  An entry is kept even when its value
//     equals the (+)-identity or zero.
//   * Every stored pair (A(i,p), B(p,j)) contributes one (x)-product; the
//     products of an entry are (+)-combined in storage order: A's row i in
//     storage order, and for each of its entries, B's row in storage order.
//     Duplicate coordinates in A or B therefore contribute separately.
//   * flops (Table 1: the count of arithmetic operations on nonzeros) is the
//     number of (x)-products, flops_i = sum over A(i,p) of nnz(B(p,:)).
//
// Semirings (the paper allows any; these six are the ones exercised):
//   1 (+,x)   over int64: wrapping two's-complement multiply and add.
//   2 (+,x)   over fp64 : IEEE multiply (no contraction into FMA), and the
//                          products of one entry summed with Neumaier's
//                          compensated summation so the reference is near
//                          exact; the sum of |products| is returned beside
//                          each entry for the tolerance test.
//   3 (min,+) over uint32: (x) = addition saturating at UINT32_MAX (= +inf),
//                          (+) = min.
//   4 (or,and) over bool : stored as uint8; nonzero = true; output 0/1.
//   5 (select2nd,min) over int32: (x)(a,b) = b, (+) = signed min.
//   6 heterogeneous (Sec. 1: two input types and one output type): A holds
//     float32 weights, B int32 labels, C (weight, label) pairs; (x)(w, l) =
//     (w, l); (+) keeps the pair whose weight is larger in IEEE 754
//     totalOrder, and of equal weights the one with the smaller label.
//
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -shared -fPIC
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>
#include <omp.h>

namespace {

enum { S_I64 = 1, S_F64 = 2, S_U32 = 3, S_BOOL = 4, S_S2M = 5, S_WL = 6 };

struct AccI64 {
  typedef int64_t T;
  typedef T TA, TB, TC;
  uint64_t s;
  void first(T a, T b) { s = (uint64_t)a * (uint64_t)b; }
  void next(T a, T b) { s += (uint64_t)a * (uint64_t)b; }
  T value() const { return (T)s; }
  double absum() const { return 0.0; }
};

struct AccF64 {
  typedef double T;
  typedef T TA, TB, TC;
  double s, c, abs_s;
  void first(T a, T b) {
    double p = a * b;
    s = p; c = 0.0; abs_s = std::fabs(p);
  }
  void next(T a, T b) {
    double p = a * b;
    double t = s + p;
    if (std::fabs(s) >= std::fabs(p)) c += (s - t) + p;
    else c += (p - t) + s;
    s = t;
    abs_s += std::fabs(p);
  }
  T value() const { return s + c; }
  double absum() const { return abs_s; }
};

struct AccU32 {
  typedef uint32_t T;
  typedef T TA, TB, TC;
  uint32_t s;
  static uint32_t mul(T a, T b) {
    uint64_t w = (uint64_t)a + (uint64_t)b;
    return w > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)w;
  }
  void first(T a, T b) { s = mul(a, b); }
  void next(T a, T b) { uint32_t p = mul(a, b); if (p < s) s = p; }
  T value() const { return s; }
  double absum() const { return 0.0; }
};

struct AccBool {
  typedef uint8_t T;
  typedef T TA, TB, TC;
  bool s;
  void first(T a, T b) { s = (a != 0) && (b != 0); }
  void next(T a, T b) { s = s || ((a != 0) && (b != 0)); }
  T value() const { return s ? 1 : 0; }
  double absum() const { return 0.0; }
};

struct AccS2M {
  typedef int32_t T;
  typedef T TA, TB, TC;
  int32_t s;
  void first(T, T b) { s = b; }
  void next(T, T b) { if (b < s) s = b; }
  T value() const { return s; }
  double absum() const { return 0.0; }
};

// IEEE 754 totalOrder, strict: x before y.  Negative-signed values (-NaN,
// -inf, ..., -0) come before positive-signed ones; among negative-signed
// values a larger magnitude encoding comes first, among positive-signed ones
// a smaller one (the binary encodings order magnitudes, NaNs above inf).
bool total_order_before(float x, float y) {
  uint32_t bx, by;
  std::memcpy(&bx, &x, sizeof bx);
  std::memcpy(&by, &y, sizeof by);
  const bool nx = (bx >> 31) != 0, ny = (by >> 31) != 0;
  if (nx != ny) return nx;
  const uint32_t mx = bx & 0x7FFFFFFFu, my = by & 0x7FFFFFFFu;
  return nx ? mx > my : mx < my;
}

struct WLabel {
  float w;
  int32_t label;
};

struct AccWL {
  typedef float TA;
  typedef int32_t TB;
  typedef WLabel TC;
  WLabel s;
  void first(TA a, TB b) { s = WLabel{a, b}; }
  void next(TA a, TB b) {
    const bool heavier = total_order_before(s.w, a);
    const bool same = !total_order_before(s.w, a) && !total_order_before(a, s.w);
    if (heavier || (same && b < s.label)) s = WLabel{a, b};
  }
  TC value() const { return s; }
  double absum() const { return 0.0; }
};

template <class Acc>
int run(int64_t m, const int64_t* Arp, const int32_t* Acol, const void* Aval_,
        const int64_t* Brp, const int32_t* Bcol, const void* Bval_,
        int64_t nsel, const int64_t* rows, int threads,
        int64_t** out_rp, int32_t** out_col, void** out_val, double** out_abs) {
  typedef typename Acc::TA TA;
  typedef typename Acc::TB TB;
  typedef typename Acc::TC TC;
  const TA* Aval = (const TA*)Aval_;
  const TB* Bval = (const TB*)Bval_;
  std::vector<std::vector<std::pair<int32_t, Acc>>> res((size_t)nsel);
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads)
  for (int64_t r = 0; r < nsel; ++r) {
    int64_t i = rows ? rows[r] : r;
    std::map<int32_t, Acc> acc;
    for (int64_t p = Arp[i]; p < Arp[i + 1]; ++p) {
      int32_t kk = Acol[p];
      TA a = Aval[p];
      for (int64_t q = Brp[kk]; q < Brp[kk + 1]; ++q) {
        int32_t j = Bcol[q];
        auto it = acc.find(j);
        if (it == acc.end()) {
          Acc x;
          x.first(a, Bval[q]);
          acc.emplace(j, x);
        } else {
          it->second.next(a, Bval[q]);
        }
      }
    }
    res[r].assign(acc.begin(), acc.end());
  }
  int64_t* rp = (int64_t*)std::malloc(sizeof(int64_t) * (size_t)(nsel + 1));
  if (!rp) return 2;
  rp[0] = 0;
  for (int64_t r = 0; r < nsel; ++r) rp[r + 1] = rp[r] + (int64_t)res[r].size();
  int64_t nnz = rp[nsel];
  int32_t* col = (int32_t*)std::malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  TC* val = (TC*)std::malloc(sizeof(TC) * (size_t)(nnz > 0 ? nnz : 1));
  double* ab = (double*)std::malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!col || !val || !ab) return 2;
#pragma omp parallel for schedule(dynamic, 64) num_threads(threads)
  for (int64_t r = 0; r < nsel; ++r) {
    int64_t o = rp[r];
    for (const auto& e : res[r]) {
      col[o] = e.first;
      val[o] = e.second.value();
      ab[o] = e.second.absum();
      ++o;
    }
  }
  *out_rp = rp;
  *out_col = col;
  *out_val = val;
  *out_abs = ab;
  return 0;
}

}  // namespace

extern "C" {

// Per-row statistics of the product A.B (Sec. 4.1, phase (1); Table 1):
// flops[i] = sum over stored A(i,p) of nnz(B(p,:)); maxb[i] = max of those
// nnz(B(p,:)) (0 for an empty row).
int orc_row_stats(int64_t m, const int64_t* Arp, const int32_t* Acol,
                  const int64_t* Brp, int64_t* flops, int64_t* maxb) {
  for (int64_t i = 0; i < m; ++i) {
    int64_t f = 0, mx = 0;
    for (int64_t p = Arp[i]; p < Arp[i + 1]; ++p) {
      int64_t len = Brp[Acol[p] + 1] - Brp[Acol[p]];
      f += len;
      if (len > mx) mx = len;
    }
    flops[i] = f;
    maxb[i] = mx;
  }
  return 0;
}

// C = A.B restricted to the rows listed in `rows` (all m rows when rows is
// NULL, then nsel must equal m).  Results are malloc'ed and returned through
// the out pointers (row pointers over the selected rows, sorted unique
// columns, values, and per-entry sum of |products| for fp64, else zeros);
// release them with orc_free.  Returns 0, 1 (bad semiring) or 2 (no memory).
int orc_spgemm(int semiring, int64_t m, const int64_t* Arp, const int32_t* Acol,
               const void* Aval, const int64_t* Brp, const int32_t* Bcol,
               const void* Bval, int64_t nsel, const int64_t* rows, int threads,
               int64_t** out_rp, int32_t** out_col, void** out_val,
               double** out_abs) {
  switch (semiring) {
    case S_I64: return run<AccI64>(m, Arp, Acol, Aval, Brp, Bcol, Bval, nsel, rows, threads, out_rp, out_col, out_val, out_abs);
    case S_F64: return run<AccF64>(m, Arp, Acol, Aval, Brp, Bcol, Bval, nsel, rows, threads, out_rp, out_col, out_val, out_abs);
    case S_U32: return run<AccU32>(m, Arp, Acol, Aval, Brp, Bcol, Bval, nsel, rows, threads, out_rp, out_col, out_val, out_abs);
    case S_BOOL: return run<AccBool>(m, Arp, Acol, Aval, Brp, Bcol, Bval, nsel, rows, threads, out_rp, out_col, out_val, out_abs);
    case S_S2M: return run<AccS2M>(m, Arp, Acol, Aval, Brp, Bcol, Bval, nsel, rows, threads, out_rp, out_col, out_val, out_abs);
    case S_WL: return run<AccWL>(m, Arp, Acol, Aval, Brp, Bcol, Bval, nsel, rows, threads, out_rp, out_col, out_val, out_abs);
  }
  return 1;
}

void orc_free(void* p) { std::free(p); }

int orc_max_threads(void) { return omp_get_max_threads(); }

}  // extern "C"
