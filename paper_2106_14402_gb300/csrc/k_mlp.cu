// K8/K9: the learned row-size predictor (paper Sec. 5: the GPU path estimates
// the output's memory needs with approximate algorithms instead of an exact
// symbolic pass; Sec. 7.4: the batch count of batched SpGEMM comes from
// such an estimate).
//
// Model: 3 -> 64 -> 64 -> 1 MLP over the row features f = (nnz(A_i), flops_i,
// max_p nnz(B_p)), the last two taken relative to the row's output width w_i
// (the column count of B), so that the same network serves products of any
// size:
//   l  = (log2(1 + f_0), log2(1 + f_1) - log2(w_i), log2(1 + f_2) - log2(w_i))
//   x  = bf16((l - mu) / sigma)
//   h1 = bf16(relu(W1 x + b1)),  h2 = bf16(relu(W2 h1 + b2)),  z = w3 . h2 + b3
//   rho = sigmoid(z) ~ nnz(C_i) / flops_i,
//   pred = clamp(ceil(rho * flops_i), maxB_i, min(flops_i, w_i))
// Feature rows are float32 [4]: nnz(A_i), flops_i, maxB_i, w_i.
// Weights are used as bf16 copies of fp32 master weights; every product is
// accumulated in fp32.  Training minimises the pinball loss (tau) on
// e = log2(nnz/flops) - log2(rho) with Adam on the fp32 master weights.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "../../include/cb.h"
#include "cb_common.cuh"

namespace cb {
namespace {

constexpr int H = CB_MLP_HIDDEN;
// offsets into the flat parameter vector
constexpr int oW1 = 0, ob1 = oW1 + H * 3, oW2 = ob1 + H, ob2 = oW2 + H * H, ow3 = ob2 + H,
              ob3 = ow3 + H, kNP = ob3 + 1;
static_assert(kNP == CB_MLP_NPARAM, "parameter layout");

constexpr int kFwdThreads = 256;
constexpr int kBwdThreads = 128;
constexpr int kPad = H + 1;  // padded row stride of per-row activation tiles

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Weights staged in shared memory as floats holding bf16 values.
struct SmemWeights {
  float W1[H * 3], b1[H], W2[H * H], b2[H], w3[H], b3, mu[3], sg[3];
};

__device__ __forceinline__ void stage_weights(SmemWeights& w, const __nv_bfloat16* wb,
                                              const float* master, const float* norm) {
  for (int t = threadIdx.x; t < H * 3; t += blockDim.x) w.W1[t] = __bfloat162float(wb[oW1 + t]);
  for (int t = threadIdx.x; t < H * H; t += blockDim.x) w.W2[t] = __bfloat162float(wb[oW2 + t]);
  for (int t = threadIdx.x; t < H; t += blockDim.x) {
    w.b1[t] = master[ob1 + t];
    w.b2[t] = master[ob2 + t];
    w.w3[t] = __bfloat162float(wb[ow3 + t]);
  }
  if (threadIdx.x == 0) w.b3 = master[ob3];
  if (threadIdx.x < 3) {
    w.mu[threadIdx.x] = norm[threadIdx.x];
    w.sg[threadIdx.x] = norm[3 + threadIdx.x];
  }
}

constexpr int kNF = CB_MLP_NFEAT;  // floats per feature row

__device__ __forceinline__ void features(const SmemWeights& w, const float* f, float x[3]) {
  const float lw = log2f(fmaxf(f[3], 1.0f));
  float l[3] = {log2f(1.0f + f[0]), log2f(1.0f + f[1]) - lw, log2f(1.0f + f[2]) - lw};
#pragma unroll
  for (int d = 0; d < 3; ++d) x[d] = bf16r((l[d] - w.mu[d]) / w.sg[d]);
}

// Forward pass of one row; h1/h2 receive the bf16-rounded activations.
__device__ __forceinline__ float forward_row(const SmemWeights& w, const float x[3], float* h1,
                                             float* h2) {
#pragma unroll 4
  for (int j = 0; j < H; ++j) {
    float a = w.b1[j];
    a = fmaf(w.W1[j * 3 + 0], x[0], a);
    a = fmaf(w.W1[j * 3 + 1], x[1], a);
    a = fmaf(w.W1[j * 3 + 2], x[2], a);
    h1[j] = bf16r(fmaxf(a, 0.0f));
  }
  float z = w.b3;
  for (int j = 0; j < H; ++j) {
    float a = w.b2[j];
#pragma unroll 8
    for (int k = 0; k < H; ++k) a = fmaf(w.W2[j * H + k], h1[k], a);
    const float v = bf16r(fmaxf(a, 0.0f));
    h2[j] = v;
    z = fmaf(w.w3[j], v, z);
  }
  return z;
}

__device__ __forceinline__ int64_t size_from_logit(float z, int64_t flops, int64_t maxb,
                                                   int64_t width, int64_t ncols) {
  if (flops <= 0) return 0;
  const double rho = 1.0 / (1.0 + exp(-(double)z));
  int64_t est = (int64_t)ceil(rho * (double)flops);
  int64_t hi = flops < width ? flops : width;
  if (ncols > 0 && ncols < hi) hi = ncols;
  if (est < maxb) est = maxb;
  if (est > hi) est = hi;
  return est;
}

// K8: one thread per row.
__global__ void __launch_bounds__(kFwdThreads) k_mlp_predict(const __nv_bfloat16* wb,
                                                             const float* master, const float* norm,
                                                             const float* feat, int64_t m,
                                                             int64_t ncols, float* z_out,
                                                             int64_t* pred_out) {
  __shared__ SmemWeights w;
  __shared__ float h1s[kFwdThreads * kPad];
  stage_weights(w, wb, master, norm);
  __syncthreads();
  float h2[H];
  float* h1 = h1s + threadIdx.x * kPad;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    float x[3];
    const float* f = feat + kNF * r;
    features(w, f, x);
    const float z = forward_row(w, x, h1, h2);
    if (z_out) z_out[r] = z;
    if (pred_out) pred_out[r] = size_from_logit(z, (int64_t)f[1], (int64_t)f[2], (int64_t)f[3], ncols);
  }
}

// K9: forward + pinball loss + backward for rows [r0, r0 + n).  Gradient sums
// (not yet divided by the number of live rows) are added to grad[0..kNP),
// the loss sum to stat[0] and the live-row count to stat[1].
__global__ void __launch_bounds__(kBwdThreads) k_mlp_grad(const __nv_bfloat16* wb,
                                                          const float* master, const float* norm,
                                                          const float* feat, const int64_t* nnz,
                                                          int64_t r0, int64_t n, float tau,
                                                          float* grad, double* stat) {
  constexpr int T = kBwdThreads;
  __shared__ SmemWeights w;
  extern __shared__ float tiles[];  // h1, h2, dh2, dh1: [T][kPad] each; x: [T][3]; dz: [T]
  float* h1 = tiles;
  float* h2 = h1 + T * kPad;
  float* dh2 = h2 + T * kPad;
  float* dh1 = dh2 + T * kPad;
  float* xs = dh1 + T * kPad;
  float* dzs = xs + T * 3;
  __shared__ float loss_part[T];
  __shared__ int live_part[T];
  stage_weights(w, wb, master, norm);
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t base = r0 + (int64_t)blockIdx.x * T;
  const int64_t r = base + t;
  float dz = 0.0f, loss = 0.0f;
  int live = 0;
  float* my1 = h1 + t * kPad;
  float* my2 = h2 + t * kPad;
  if (r < r0 + n) {
    float x[3];
    features(w, feat + kNF * r, x);
    xs[t * 3 + 0] = x[0];
    xs[t * 3 + 1] = x[1];
    xs[t * 3 + 2] = x[2];
    const float z = forward_row(w, x, my1, my2);
    const float fl = feat[kNF * r + 1];
    if (fl > 0.0f) {
      live = 1;
      const float ls = -(fmaxf(-z, 0.0f) + log1pf(expf(-fabsf(z))));  // log sigmoid(z)
      const float e = log2f((float)nnz[r] / fl) - ls * 1.4426950408889634f;
      loss = e >= 0.0f ? tau * e : (tau - 1.0f) * e;
      const float sig = 1.0f / (1.0f + expf(-z));
      dz = (e >= 0.0f ? tau : tau - 1.0f) * (-(1.0f - sig) * 1.4426950408889634f);
    }
  } else {
    for (int j = 0; j < H; ++j) my1[j] = my2[j] = 0.0f;
    xs[t * 3 + 0] = xs[t * 3 + 1] = xs[t * 3 + 2] = 0.0f;
  }
  dzs[t] = dz;
  loss_part[t] = loss;
  live_part[t] = live;
  float* myd2 = dh2 + t * kPad;
  for (int j = 0; j < H; ++j) myd2[j] = my2[j] > 0.0f ? dz * w.w3[j] : 0.0f;
  float* myd1 = dh1 + t * kPad;
  for (int k = 0; k < H; ++k) {
    float a = 0.0f;
#pragma unroll 8
    for (int j = 0; j < H; ++j) a = fmaf(myd2[j], w.W2[j * H + k], a);
    myd1[k] = my1[k] > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  // weight-gradient reductions over the block's rows
  {
    // W2: thread pair (j, half) sums 32 entries over T rows
    const int j = t >> 1, k0 = (t & 1) * (H / 2);
    float acc[H / 2];
#pragma unroll
    for (int q = 0; q < H / 2; ++q) acc[q] = 0.0f;
    for (int rr = 0; rr < T; ++rr) {
      const float d = dh2[rr * kPad + j];
#pragma unroll
      for (int q = 0; q < H / 2; ++q) acc[q] = fmaf(d, h1[rr * kPad + k0 + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < H / 2; ++q) atomicAdd(&grad[oW2 + j * H + k0 + q], acc[q]);
  }
  if (t < H) {
    float gw3 = 0.0f, gb2 = 0.0f, gb1 = 0.0f, g1[3] = {0.0f, 0.0f, 0.0f};
    for (int rr = 0; rr < T; ++rr) {
      gw3 = fmaf(dzs[rr], h2[rr * kPad + t], gw3);
      gb2 += dh2[rr * kPad + t];
      const float d1 = dh1[rr * kPad + t];
      gb1 += d1;
      g1[0] = fmaf(d1, xs[rr * 3 + 0], g1[0]);
      g1[1] = fmaf(d1, xs[rr * 3 + 1], g1[1]);
      g1[2] = fmaf(d1, xs[rr * 3 + 2], g1[2]);
    }
    atomicAdd(&grad[ow3 + t], gw3);
    atomicAdd(&grad[ob2 + t], gb2);
    atomicAdd(&grad[ob1 + t], gb1);
    atomicAdd(&grad[oW1 + t * 3 + 0], g1[0]);
    atomicAdd(&grad[oW1 + t * 3 + 1], g1[1]);
    atomicAdd(&grad[oW1 + t * 3 + 2], g1[2]);
  }
  if (t == H) {
    float gb3 = 0.0f, ls = 0.0f;
    int lv = 0;
    for (int rr = 0; rr < T; ++rr) {
      gb3 += dzs[rr];
      ls += loss_part[rr];
      lv += live_part[rr];
    }
    atomicAdd(&grad[ob3], gb3);
    atomicAdd(&stat[0], (double)ls);
    atomicAdd(&stat[1], (double)lv);
  }
}

// Divide gradient sums by the live-row count (gradient output form).
__global__ void k_mlp_scale(const float* grad, const double* stat, float* out, float* loss) {
  const double inv = stat[1] > 0 ? 1.0 / stat[1] : 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < kNP; t += gridDim.x * blockDim.x)
    out[t] = (float)(grad[t] * inv);
  if (blockIdx.x == 0 && threadIdx.x == 0 && loss) *loss = (float)(stat[0] * inv);
}

// Adam step on the master weights with the mean gradient, refresh the bf16
// copies, clear the gradient sums and the batch statistics.  One block (it
// clears the statistics that all threads read first).
__global__ void k_mlp_adam(float* master, __nv_bfloat16* wb, float* mom, float* vel, float* grad,
                           double* stat, double* epoch_loss, float lr, float b1c, float b2c,
                           int64_t step) {
  const double live = stat[1];
  const float inv = live > 0 ? (float)(1.0 / live) : 0.0f;
  const float c1 = 1.0f - powf(b1c, (float)step), c2 = 1.0f - powf(b2c, (float)step);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < kNP; t += gridDim.x * blockDim.x) {
    const float g = grad[t] * inv;
    const float mt = b1c * mom[t] + (1.0f - b1c) * g;
    const float vt = b2c * vel[t] + (1.0f - b2c) * g * g;
    mom[t] = mt;
    vel[t] = vt;
    const float wnew = master[t] - lr * (mt / c1) / (sqrtf(vt / c2) + 1e-8f);
    master[t] = wnew;
    wb[t] = __float2bfloat16_rn(wnew);
    grad[t] = 0.0f;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (epoch_loss) {
      epoch_loss[0] += stat[0];
      epoch_loss[1] += stat[1];
    }
    stat[0] = 0.0;
    stat[1] = 0.0;
  }
}

__global__ void k_mlp_round(const float* master, __nv_bfloat16* wb) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < kNP; t += gridDim.x * blockDim.x)
    wb[t] = __float2bfloat16_rn(master[t]);
}

// raw features (nnz(A_i), flops_i, maxB_i) as floats
__global__ void k_row_features(DevCSR A, const int64_t* flops, const int32_t* maxb, int64_t ncols,
                               float* feat) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.nrows;
       i += (int64_t)gridDim.x * blockDim.x) {
    feat[kNF * i + 0] = (float)(A.rp[i + 1] - A.rp[i]);
    feat[kNF * i + 1] = (float)flops[i];
    feat[kNF * i + 2] = (float)maxb[i];
    feat[kNF * i + 3] = (float)(A.rcols ? (int64_t)A.rcols[i] : ncols);
  }
}

constexpr size_t kGradSmem = (size_t)kBwdThreads * (4 * kPad + 4) * sizeof(float);

}  // namespace

void launch_row_features(const DevCSR& A, const int64_t* flops, const int32_t* maxb, int64_t ncols,
                         float* feat, cudaStream_t s, int sms) {
  if (A.nrows == 0) return;
  int64_t g = (A.nrows + 255) / 256;
  k_row_features<<<(int)(g < sms * 8 ? g : sms * 8), 256, 0, s>>>(A, flops, maxb, ncols, feat);
}

void launch_mlp_predict(const void* wb, const float* master, const float* norm, const float* feat,
                        int64_t m, int64_t ncols, float* z, int64_t* pred, cudaStream_t s, int sms) {
  if (m == 0) return;
  int64_t g = (m + kFwdThreads - 1) / kFwdThreads;
  k_mlp_predict<<<(int)(g < sms * 4 ? g : sms * 4), kFwdThreads, 0, s>>>(
      static_cast<const __nv_bfloat16*>(wb), master, norm, feat, m, ncols, z, pred);
}

}  // namespace cb

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

struct cb_mlp {
  int device = 0;
  float* master = nullptr;     // kNP fp32
  __nv_bfloat16* wb = nullptr; // kNP bf16 copies
  float* mom = nullptr;
  float* vel = nullptr;
  float* grad = nullptr;
  float* norm = nullptr;       // mu[3], sigma[3]
  double* stat = nullptr;      // loss sum, live rows; then epoch loss sum, epoch live rows
  int64_t step = 0;
};

namespace {
int mlp_free(cb_mlp* m) {
  if (!m) return CB_OK;
  cudaFree(m->master);
  cudaFree(m->wb);
  cudaFree(m->mom);
  cudaFree(m->vel);
  cudaFree(m->grad);
  cudaFree(m->norm);
  cudaFree(m->stat);
  delete m;
  return CB_OK;
}
}  // namespace

extern "C" {

int cb_mlp_create(cb_mlp** out, const float* params, const float* norm) {
  using namespace cb;
  if (!out || !params || !norm) return CB_ERR_ARG;
  *out = nullptr;
  cb_mlp* m = new (std::nothrow) cb_mlp();
  if (!m) return CB_ERR_OOM;
  cudaGetDevice(&m->device);
  bool ok = cudaMalloc(&m->master, kNP * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->wb, kNP * sizeof(__nv_bfloat16)) == cudaSuccess &&
            cudaMalloc(&m->mom, kNP * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->vel, kNP * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->grad, kNP * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->norm, 6 * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->stat, 4 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    mlp_free(m);
    return CB_ERR_OOM;
  }
  ok = cudaMemcpy(m->master, params, kNP * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(m->norm, norm, 6 * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(m->mom, 0, kNP * sizeof(float)) == cudaSuccess &&
       cudaMemset(m->vel, 0, kNP * sizeof(float)) == cudaSuccess &&
       cudaMemset(m->grad, 0, kNP * sizeof(float)) == cudaSuccess &&
       cudaMemset(m->stat, 0, 4 * sizeof(double)) == cudaSuccess;
  if (ok) {
    k_mlp_round<<<8, 256>>>(m->master, m->wb);
    ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
  }
  if (!ok) {
    mlp_free(m);
    return CB_ERR_CUDA;
  }
  *out = m;
  return CB_OK;
}

void cb_mlp_destroy(cb_mlp* m) {
  if (m) cudaDeviceSynchronize();
  mlp_free(m);
}

int cb_mlp_get(const cb_mlp* m, float* params, float* norm, int64_t* step) {
  using namespace cb;
  if (!m) return CB_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return CB_ERR_CUDA;
  if (params && cudaMemcpy(params, m->master, kNP * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CB_ERR_CUDA;
  if (norm && cudaMemcpy(norm, m->norm, 6 * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CB_ERR_CUDA;
  if (step) *step = m->step;
  return CB_OK;
}

}  // extern "C"

// Device-side accessors used by the SpGEMM dispatcher (learned sizing).
namespace cb {
const void* mlp_bf16(const cb_mlp* m) { return m->wb; }
const float* mlp_master(const cb_mlp* m) { return m->master; }
const float* mlp_norm(const cb_mlp* m) { return m->norm; }
}  // namespace cb

extern "C" {

int cb_mlp_predict(cb_ctx* ctx, const cb_mlp* m, const float* feat, int64_t nrows, int64_t ncols,
                   float* z, int64_t* pred);
int cb_mlp_grad(cb_ctx* ctx, const cb_mlp* m, const float* feat, const int64_t* nnz, int64_t nrows,
                float tau, float* grad, float* loss);
int cb_mlp_train(cb_ctx* ctx, cb_mlp* m, const float* feat, const int64_t* nnz, int64_t nrows,
                 int epochs, int64_t batch, float lr, float tau, float* epoch_loss);

}  // extern "C"

// Shared with the context-owning file.
namespace cb {
cudaStream_t ctx_stream(cb_ctx* ctx);
int ctx_sms(cb_ctx* ctx);
}  // namespace cb

extern "C" int cb_mlp_predict(cb_ctx* ctx, const cb_mlp* m, const float* feat, int64_t nrows,
                              int64_t ncols, float* z, int64_t* pred) {
  if (!ctx || !m || nrows < 0 || (nrows > 0 && !feat) || ncols < 0) return CB_ERR_ARG;
  cb::launch_mlp_predict(m->wb, m->master, m->norm, feat, nrows, ncols, z, pred, cb::ctx_stream(ctx),
                         cb::ctx_sms(ctx));
  return cudaGetLastError() == cudaSuccess ? CB_OK : CB_ERR_CUDA;
}

extern "C" int cb_mlp_grad(cb_ctx* ctx, const cb_mlp* m, const float* feat, const int64_t* nnz,
                           int64_t nrows, float tau, float* grad, float* loss) {
  using namespace cb;
  if (!ctx || !m || nrows < 0 || (nrows > 0 && (!feat || !nnz)) || !grad) return CB_ERR_ARG;
  cudaStream_t s = ctx_stream(ctx);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
    attr = true;
  }
  if (cudaMemsetAsync(m->grad, 0, kNP * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(m->stat, 0, 2 * sizeof(double), s) != cudaSuccess)
    return CB_ERR_CUDA;
  if (nrows > 0) {
    const int64_t blocks = (nrows + kBwdThreads - 1) / kBwdThreads;
    k_mlp_grad<<<(unsigned)blocks, kBwdThreads, kGradSmem, s>>>(m->wb, m->master, m->norm, feat, nnz,
                                                                 0, nrows, tau, m->grad, m->stat);
  }
  k_mlp_scale<<<8, 256, 0, s>>>(m->grad, m->stat, grad, loss);
  const bool ok = cudaGetLastError() == cudaSuccess &&
                  cudaMemsetAsync(m->grad, 0, kNP * sizeof(float), s) == cudaSuccess &&
                  cudaMemsetAsync(m->stat, 0, 2 * sizeof(double), s) == cudaSuccess;
  return ok ? CB_OK : CB_ERR_CUDA;
}

extern "C" int cb_mlp_train(cb_ctx* ctx, cb_mlp* m, const float* feat, const int64_t* nnz,
                            int64_t nrows, int epochs, int64_t batch, float lr, float tau,
                            float* epoch_loss) {
  using namespace cb;
  if (!ctx || !m || nrows <= 0 || !feat || !nnz || epochs < 0 || batch <= 0 || !(lr > 0.0f))
    return CB_ERR_ARG;
  cudaStream_t s = ctx_stream(ctx);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
    attr = true;
  }
  if (batch % kBwdThreads) batch += kBwdThreads - batch % kBwdThreads;
  if (cudaMemsetAsync(m->grad, 0, kNP * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(m->stat, 0, 4 * sizeof(double), s) != cudaSuccess)
    return CB_ERR_CUDA;
  for (int ep = 0; ep < epochs; ++ep) {
    // each epoch starts the batch sequence at a different offset
    const int64_t shift = ((int64_t)ep * 7919 * kBwdThreads) % nrows;
    for (int64_t done = 0; done < nrows; done += batch) {
      const int64_t start = (shift + done) % nrows;
      int64_t n = batch < nrows - done ? batch : nrows - done;
      // a batch that runs past the end wraps to the front in two launches
      const int64_t n1 = n < nrows - start ? n : nrows - start;
      k_mlp_grad<<<(unsigned)((n1 + kBwdThreads - 1) / kBwdThreads), kBwdThreads, kGradSmem, s>>>(
          m->wb, m->master, m->norm, feat, nnz, start, n1, tau, m->grad, m->stat);
      if (n > n1)
        k_mlp_grad<<<(unsigned)((n - n1 + kBwdThreads - 1) / kBwdThreads), kBwdThreads, kGradSmem,
                     s>>>(m->wb, m->master, m->norm, feat, nnz, 0, n - n1, tau, m->grad, m->stat);
      ++m->step;
      k_mlp_adam<<<1, 1024, 0, s>>>(m->master, m->wb, m->mom, m->vel, m->grad, m->stat,
                                    m->stat + 2, lr, 0.9f, 0.999f, m->step);
    }
    if (epoch_loss) {
      double h[2];
      if (cudaMemcpyAsync(h, m->stat + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess ||
          cudaMemsetAsync(m->stat + 2, 0, 2 * sizeof(double), s) != cudaSuccess)
        return CB_ERR_CUDA;
      epoch_loss[ep] = h[1] > 0 ? (float)(h[0] / h[1]) : 0.0f;
    }
  }
  return cudaGetLastError() == cudaSuccess ? CB_OK : CB_ERR_CUDA;
}
