// k_mlp.cu -- the learned tile-cost model: a 16 -> 128 -> 128 -> 1 MLP with
// exact GELU, trained with MSE and Adam, all on the GPU in FP32.
//
// It ranks candidate tile schedules (tile sizes, stages, cluster, split-K) so
// that only a few are timed -- a model-guided replacement for the black-box
// tile/unroll search of Sec. 4.3.  Forward: y = W3 g(W2 g(W1 x + b1) + b2) + b3
// with g(z) = z * Phi(z).  Backward follows the chain rule; each block of 32
// rows writes its partial gradient sums to the workspace and one pass adds
// the blocks in a fixed order (run-to-run identical), then Adam (Kingma & Ba
// 2015, Algorithm 1) updates the parameters.
//
// Parameter layout (one FP32 buffer, 18817 values): W1 [128][16], b1 [128],
// W2 [128][128], b2 [128], W3 [128], b3 [1].
#include <cuda_runtime.h>

#include "../../include/nk_tune.h"
#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int D0 = 16, D1 = 128, D2 = 128;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + D1 * D0, OFF_W2 = OFF_B1 + D1, OFF_B2 = OFF_W2 + D2 * D1,
              OFF_W3 = OFF_B2 + D2, OFF_B3 = OFF_W3 + D2, NPARAM = OFF_B3 + 1;
constexpr int ROWS = 32;     // batch rows per block
constexpr int THREADS = 128; // one thread per hidden unit

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  const float Phi = 0.5f * (1.f + erff(z * 0.70710678118654752f));
  const float phi = 0.39894228040143268f * expf(-0.5f * z * z);
  return Phi + z * phi;
}

struct Smem {
  float w2t[D1][D2 + 1];  // W2 transposed, padded: w2t[i][j] = W2[j][i]
  float w1[D1][D0 + 1];
  float x[ROWS][D0];
  float z1[ROWS][D1];
  float h1[ROWS][D1];
  float z2[ROWS][D2];
  float h2[ROWS][D2];
  float y[ROWS];
  float dy[ROWS];
};

// Forward for the block's rows; fills s.z1, h1, z2, h2, y.  Thread j owns
// hidden unit j.
__device__ void forward_rows(const float* __restrict__ P, const float* __restrict__ X, int64_t B,
                             int64_t r0, Smem& s) {
  const int j = threadIdx.x;
  for (int e = j; e < D1 * D2; e += THREADS) {
    const int jj = e / D1, ii = e % D1;      // W2[jj][ii]
    s.w2t[ii][jj] = P[OFF_W2 + e];
  }
  for (int e = j; e < D1 * D0; e += THREADS) s.w1[e / D0][e % D0] = P[OFF_W1 + e];
  for (int e = j; e < ROWS * D0; e += THREADS) {
    const int r = e / D0;
    s.x[r][e % D0] = (r0 + r < B) ? X[(r0 + r) * D0 + e % D0] : 0.f;
  }
  __syncthreads();
  const float b1 = P[OFF_B1 + j], b2 = P[OFF_B2 + j];
  for (int r = 0; r < ROWS; ++r) {
    float z = b1;
#pragma unroll
    for (int i = 0; i < D0; ++i) z = fmaf(s.x[r][i], s.w1[j][i], z);
    s.z1[r][j] = z;
    s.h1[r][j] = gelu(z);
  }
  __syncthreads();
  for (int r = 0; r < ROWS; ++r) {
    float z = b2;
#pragma unroll 8
    for (int i = 0; i < D1; ++i) z = fmaf(s.h1[r][i], s.w2t[i][j], z);
    s.z2[r][j] = z;
    s.h2[r][j] = gelu(z);
  }
  __syncthreads();
  // y[r] = b3 + sum_j h2[r][j] W3[j]: warp w reduces rows w, w+4, ...
  const int warp = j / 32, lane = j % 32;
  for (int r = warp; r < ROWS; r += THREADS / 32) {
    float a = 0.f;
    for (int i = lane; i < D2; i += 32) a = fmaf(s.h2[r][i], P[OFF_W3 + i], a);
#pragma unroll
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) s.y[r] = a + P[OFF_B3];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(THREADS) mlp_forward_kernel(const float* __restrict__ P,
                                                              const float* __restrict__ X, int64_t B,
                                                              float* __restrict__ y) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  extern __shared__ __align__(16) uint8_t raw[];
  Smem& s = *reinterpret_cast<Smem*>(raw);
  const int64_t r0 = (int64_t)blockIdx.x * ROWS;
  forward_rows(P, X, B, r0, s);
  for (int r = threadIdx.x; r < ROWS; r += THREADS)
    if (r0 + r < B) y[r0 + r] = s.y[r];
}

// Forward + backward of the MSE loss for the block's rows; writes this
// block's partial gradient sums (and sum of squared errors) to part[block].
__global__ void __launch_bounds__(THREADS) mlp_grad_kernel(const float* __restrict__ P,
                                                           const float* __restrict__ X,
                                                           const float* __restrict__ T, int64_t B,
                                                           float* __restrict__ part) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  extern __shared__ __align__(16) uint8_t raw[];
  Smem& s = *reinterpret_cast<Smem*>(raw);
  const int64_t r0 = (int64_t)blockIdx.x * ROWS;
  forward_rows(P, X, B, r0, s);
  const int j = threadIdx.x;
  float* g = part + (int64_t)blockIdx.x * (NPARAM + 1);
  const float inv2b = 2.f / (float)B;
  if (j < ROWS) {
    const bool ok = r0 + j < B;
    const float d = ok ? s.y[j] - T[r0 + j] : 0.f;
    s.dy[j] = ok ? inv2b * d : 0.f;
    // squared-error partial: reduced by the first warp below
    float sq = d * d;
#pragma unroll
    for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (j == 0) g[NPARAM] = sq;
  }
  __syncthreads();
  // dZ2 (into z2), grads of W3, b3
  const float w3 = P[OFF_W3 + j];
  float gw3 = 0.f, gb2 = 0.f;
  for (int r = 0; r < ROWS; ++r) {
    gw3 = fmaf(s.dy[r], s.h2[r][j], gw3);
    const float dz = s.dy[r] * w3 * gelu_grad(s.z2[r][j]);
    s.z2[r][j] = dz;
    gb2 += dz;
  }
  g[OFF_W3 + j] = gw3;
  g[OFF_B2 + j] = gb2;
  if (j == 0) {
    float gb3 = 0.f;
    for (int r = 0; r < ROWS; ++r) gb3 += s.dy[r];
    g[OFF_B3] = gb3;
  }
  __syncthreads();
  // gW2[jj][j] = sum_r dZ2[r][jj] h1[r][j]; thread j owns column j (coalesced stores)
  for (int jj = 0; jj < D2; ++jj) {
    float a = 0.f;
#pragma unroll 8
    for (int r = 0; r < ROWS; ++r) a = fmaf(s.z2[r][jj], s.h1[r][j], a);
    g[OFF_W2 + jj * D1 + j] = a;
  }
  // dH1[r][i] = sum_jj dZ2[r][jj] W2[jj][i]; thread j owns column i = j
  __syncthreads();
  const int i = j;
  float gb1 = 0.f;
  for (int r = 0; r < ROWS; ++r) {
    float a = 0.f;
#pragma unroll 8
    for (int jj = 0; jj < D2; ++jj) a = fmaf(s.z2[r][jj], s.w2t[i][jj], a);
    const float dz1 = a * gelu_grad(s.z1[r][i]);
    s.h1[r][i] = dz1;          // h1 is no longer needed: reuse it for dZ1
    gb1 += dz1;
  }
  g[OFF_B1 + i] = gb1;
  __syncthreads();
  // gW1[j][k] = sum_r dZ1[r][j] x[r][k]
#pragma unroll
  for (int k = 0; k < D0; ++k) {
    float a = 0.f;
    for (int r = 0; r < ROWS; ++r) a = fmaf(s.h1[r][j], s.x[r][k], a);
    g[OFF_W1 + j * D0 + k] = a;
  }
}

// grad[p] = sum_b part[b][p] in block order; loss = sum_b part[b][NPARAM] / B.
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int nblocks, int64_t B,
                                  float* __restrict__ grad, float* __restrict__ loss) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > NPARAM) return;
  float a = 0.f;
  for (int b = 0; b < nblocks; ++b) a += part[(int64_t)b * (NPARAM + 1) + p];
  if (p < NPARAM) grad[p] = a;
  else if (loss) *loss = a / (float)B;
}

__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                                float bc1, float bc2) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.f - b1) * gp;
  const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float mh = mp / bc1;
  const float vh = vp / bc2;
  P[p] -= lr * mh / (sqrtf(vh) + eps);
}

nk_status set_smem(const void* fn) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  return e == cudaSuccess ? NK_OK : cuda_fail(e, "cudaFuncSetAttribute(mlp)");
}

}  // namespace
}  // namespace nk

using namespace nk;

extern "C" {

size_t nk_mlp_param_count(void) { return NPARAM; }

size_t nk_mlp_workspace_size(int64_t B) {
  const int64_t nb = (B + ROWS - 1) / ROWS;
  return (size_t)nb * (NPARAM + 1) * sizeof(float);
}

nk_status nk_mlp_forward(const float* params, const float* X, int64_t B, float* y, void* stream) {
  nk::NvtxRange nvtx_range_("nk_mlp_forward");
  nk_status s = require_device();
  if (s != NK_OK) return s;
  if (B < 0) return fail(NK_ERR_INVALID_ARG, "negative batch");
  if (B == 0) return NK_OK;
  if (!params || !X || !y) return fail(NK_ERR_INVALID_ARG, "null pointer");
  if ((s = set_smem(reinterpret_cast<const void*>(mlp_forward_kernel))) != NK_OK) return s;
  const int64_t nb = (B + ROWS - 1) / ROWS;
  (void)nk::launch_k(mlp_forward_kernel, dim3((unsigned)nb), dim3(THREADS), sizeof(Smem), static_cast<cudaStream_t>(stream), 1, params, X, B, y);
  return check_launch("mlp_forward_kernel");
}

nk_status nk_mlp_grad(const float* params, const float* X, const float* t, int64_t B, float* grad, float* loss,
                      void* ws, size_t ws_bytes, void* stream) {
  nk::NvtxRange nvtx_range_("nk_mlp_grad");
  nk_status s = require_device();
  if (s != NK_OK) return s;
  if (B <= 0) return fail(NK_ERR_INVALID_ARG, "batch must be positive");
  if (!params || !X || !t || !grad) return fail(NK_ERR_INVALID_ARG, "null pointer");
  if (!ws || ws_bytes < nk_mlp_workspace_size(B))
    return fail(NK_ERR_WORKSPACE, "mlp gradient needs %zu bytes of workspace", nk_mlp_workspace_size(B));
  if ((s = set_smem(reinterpret_cast<const void*>(mlp_grad_kernel))) != NK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nb = (B + ROWS - 1) / ROWS;
  float* part = static_cast<float*>(ws);
  (void)nk::launch_k(mlp_grad_kernel, dim3((unsigned)nb), dim3(THREADS), sizeof(Smem), st, 1, params, X, t, B, part);
  if ((s = check_launch("mlp_grad_kernel")) != NK_OK) return s;
  (void)nk::launch_k(mlp_reduce_kernel, dim3((NPARAM + 1 + 255) / 256), dim3(256), 0, st, 1, part, (int)nb, B, grad, loss);
  return check_launch("mlp_reduce_kernel");
}

nk_status nk_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t step, float lr, float beta1,
                      float beta2, float eps, void* stream) {
  nk::NvtxRange nvtx_range_("nk_mlp_adam");
  nk_status s = require_device();
  if (s != NK_OK) return s;
  if (step < 1) return fail(NK_ERR_INVALID_ARG, "Adam step counts from 1");
  if (!params || !grad || !m || !v) return fail(NK_ERR_INVALID_ARG, "null pointer");
  const float bc1 = 1.f - powf(beta1, (float)step);
  const float bc2 = 1.f - powf(beta2, (float)step);
  (void)nk::launch_k(mlp_adam_kernel, dim3((NPARAM + 255) / 256), dim3(256), 0, static_cast<cudaStream_t>(stream), 1, 
      params, grad, m, v, NPARAM, lr, beta1, beta2, eps, bc1, bc2);
  return check_launch("mlp_adam_kernel");
}

}  // extern "C"
