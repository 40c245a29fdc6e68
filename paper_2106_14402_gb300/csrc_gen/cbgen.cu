// Seeded synthetic inputs generated on the device (libcbgen.so).  Input
// generation only: nothing here computes a product.  The same counter-based
// definition is restated in numpy (paper_2106_14402_gb300/gen.py) so the CPU
// side can regenerate any sampled matrix bit for bit.
//
// Counter-based draw: for a stream seed s and counter c (64-bit),
//   draw(s, c) = mix(s + 0x9E3779B97F4A7C15 * (c + 1))
// where mix is the splitmix64 output function (Steele, Lea, Flood 2014).
// Exact-degree ER row r of a matrix with `ncols` columns and degree d takes
// the candidates  col_t = (draw(s, (r << 32) | t) >> 32) * ncols >> 32  for
// t = 0, 1, ... and keeps the first d distinct ones, sorted.  Values of
// entry q: uniform integers lo + ((draw(s, q) >> 32) * (hi - lo + 1) >> 32),
// or doubles lo + (hi - lo) * (draw(s, q) >> 11) * 2^-53.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t s, uint64_t c) {
  return mix64(s + 0x9E3779B97F4A7C15ull * (c + 1));
}

constexpr int kMaxDeg = 128;
constexpr uint32_t kMaxTries = 1u << 20;

__global__ void k_er_rows(uint64_t seed, int64_t nrows, int64_t ncols, int deg, int32_t* col,
                          int* err) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int32_t got[kMaxDeg];
  int n = 0;
  for (uint32_t t = 0; n < deg; ++t) {
    if (t >= kMaxTries) {  // cannot happen for ncols >> deg; bounded all the same
      atomicExch(err, 1);
      break;
    }
    const uint64_t x = draw(seed, ((uint64_t)r << 32) | t);
    const int32_t c = (int32_t)(((x >> 32) * (uint64_t)ncols) >> 32);
    bool dup = false;
    for (int k = 0; k < n; ++k) dup |= got[k] == c;
    if (!dup) got[n++] = c;
  }
  for (int k = 1; k < n; ++k) {  // insertion sort
    const int32_t v = got[k];
    int p = k - 1;
    while (p >= 0 && got[p] > v) {
      got[p + 1] = got[p];
      --p;
    }
    got[p + 1] = v;
  }
  int32_t* dst = col + r * deg;
  for (int k = 0; k < deg; ++k) dst[k] = k < n ? got[k] : 0;
}

__global__ void k_row_ptr(int64_t nrows, int deg, int64_t* rp) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= nrows;
       r += (int64_t)gridDim.x * blockDim.x)
    rp[r] = r * deg;
}

__global__ void k_values_u32(uint64_t seed, int64_t n, uint32_t lo, uint32_t hi, uint32_t* out) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = lo + (uint32_t)(((draw(seed, (uint64_t)q) >> 32) * ((uint64_t)hi - lo + 1)) >> 32);
}

__global__ void k_values_f64(uint64_t seed, int64_t n, double lo, double hi, double* out) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = lo + (hi - lo) * ((double)(draw(seed, (uint64_t)q) >> 11) * 0x1.0p-53);
}

}  // namespace

extern "C" {

// Exact-degree ER pattern: row_ptr int64[nrows+1] = r*deg, col int32[nrows*deg]
// (device).  Returns 0, or 1 for bad arguments, 2 for a CUDA error.
int cbgen_er(uint64_t seed, int64_t nrows, int64_t ncols, int deg, int64_t* row_ptr, int32_t* col,
             int* err_dev, void* stream) {
  if (nrows < 0 || ncols <= 0 || deg < 0 || deg > kMaxDeg || deg > ncols) return 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_row_ptr<<<256, 256, 0, s>>>(nrows, deg, row_ptr);
  if (nrows > 0 && deg > 0)
    k_er_rows<<<(unsigned)((nrows + 127) / 128), 128, 0, s>>>(seed, nrows, ncols, deg, col, err_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int cbgen_values_u32(uint64_t seed, int64_t n, uint32_t lo, uint32_t hi, uint32_t* out, void* stream) {
  if (n < 0 || hi < lo) return 1;
  if (n) k_values_u32<<<1024, 256, 0, static_cast<cudaStream_t>(stream)>>>(seed, n, lo, hi, out);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int cbgen_values_f64(uint64_t seed, int64_t n, double lo, double hi, double* out, void* stream) {
  if (n < 0) return 1;
  if (n) k_values_f64<<<1024, 256, 0, static_cast<cudaStream_t>(stream)>>>(seed, n, lo, hi, out);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
