// k_prep.cu -- operand preparation and the validation norm.
//
// Operand prep turns FP32 operands into what the tensor cores read:
//   BF16     x -> bf16_rn(x)
//   FP8      s = 448/amax(|x|) (1 if amax is 0 or not finite), q = e4m3_rn_sat(x*s)
//   BF16x3   hi = bf16_rn(x), lo = bf16_rn(x - hi)
// optionally transposing [rows, cols] -> [cols, rows] so that a [K,N] operand
// becomes K-major.  These passes are HBM-bound: 128-bit loads, one read and
// one write of every element, 64x64 shared-memory tiles for the transpose.
// Rounding uses CUDA's own conversion intrinsics (RNE; satfinite for E4M3).
//
// The validation norm sums (C-R)^2 and R^2 in FP64 over a fixed partition
// (fixed block count, fixed tree), so its result is identical run to run.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int kAmaxBlocks = 1024;
constexpr int kNormBlocks = 1024;

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Prologue program on four consecutive elements starting at offset `off`.
template <bool PRO>
__device__ __forceinline__ void pro4(const EwProg& e, float* v, int64_t off) {
  if constexpr (PRO) {
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = ew_run(e, v[j], off + j);
  }
}

// amax over a [rows, cols] matrix with row stride ld.  Stage 1: one partial
// per block; stage 2: one block folds the partials.  NaN inputs make the
// result NaN (the scale then falls back to 1).  PRO: the amax of the values
// after the prologue program `pro`.
template <bool PRO>
__global__ void amax_stage1(const float* __restrict__ x, int64_t rows, int64_t cols, int64_t ld,
                            float* __restrict__ partial, const __grid_constant__ EwProg pro) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  float m = 0.f;
  bool nan = false;
  const bool al = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  if (al && ld == cols && (rows * cols) % 4 == 0) {
    // dense: one flat run of float4, no index arithmetic per element
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const int64_t n4 = rows * cols / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
      float4 v = __ldg(x4 + i);
      if constexpr (PRO) {
        float w[4] = {v.x, v.y, v.z, v.w};
        pro4<PRO>(pro, w, 4 * i);
        v = make_float4(w[0], w[1], w[2], w[3]);
      }
      nan |= (v.x != v.x) | (v.y != v.y) | (v.z != v.z) | (v.w != v.w);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
  } else {
    // strided rows: blocks stride over rows, threads over the row
    const bool vec = al && (cols % 4 == 0) && (ld % 4 == 0);
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
      const float* row = x + r * ld;
      if (vec) {
        for (int64_t c = threadIdx.x; c < cols / 4; c += blockDim.x) {
          float4 v = __ldg(reinterpret_cast<const float4*>(row) + c);
          if constexpr (PRO) {
            float w[4] = {v.x, v.y, v.z, v.w};
            pro4<PRO>(pro, w, r * ld + 4 * c);
            v = make_float4(w[0], w[1], w[2], w[3]);
          }
          nan |= (v.x != v.x) | (v.y != v.y) | (v.z != v.z) | (v.w != v.w);
          m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
      } else {
        for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) {
          float v = row[c];
          if constexpr (PRO) v = ew_run(pro, v, r * ld + c);
          nan |= (v != v);
          m = fmaxf(m, fabsf(v));
        }
      }
    }
  }
  if (__any_sync(0xffffffffu, nan)) m = __int_as_float(0x7fc00000);
  __shared__ float sm[32];
  float w = warp_max(m);
  bool wn = __any_sync(0xffffffffu, m != m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x / 32] = wn ? __int_as_float(0x7fc00000) : w;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x / 32;
    float v = threadIdx.x < nw ? sm[threadIdx.x] : 0.f;
    bool bn = __any_sync(0xffffffffu, v != v);
    v = warp_max(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = bn ? __int_as_float(0x7fc00000) : v;
  }
}

__global__ void amax_stage2(const float* __restrict__ partial, int n, float* __restrict__ out) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  float m = 0.f;
  bool nan = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float v = partial[i];
    nan |= (v != v);
    m = fmaxf(m, v);
  }
  __shared__ float sm[32];
  __shared__ int sn;
  if (threadIdx.x == 0) sn = 0;
  __syncthreads();
  if (nan) atomicOr(&sn, 1);
  float w = warp_max(m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x / 32] = w;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (int)(blockDim.x / 32) ? sm[threadIdx.x] : 0.f;
    v = warp_max(v);
    if (threadIdx.x == 0) *out = sn ? __int_as_float(0x7fc00000) : v;
  }
}

__device__ __forceinline__ float fp8_scale_of(const float* amax) {
  const float a = *amax;
  return (a > 0.f && a <= 3.402823466e38f) ? __fdiv_rn(448.f, a) : 1.f;
}

// One element of each cast kind.  kind 0: bf16, 1: e4m3, 2: bf16 hi/lo.
template <int KIND>
struct Caster;

template <>
struct Caster<0> {
  using T = __nv_bfloat16;
  __device__ static void cvt(float x, float, T& o0, T&) { o0 = __float2bfloat16_rn(x); }
};
template <>
struct Caster<1> {
  using T = __nv_fp8_storage_t;
  __device__ static void cvt(float x, float s, T& o0, T&) {
    o0 = __nv_cvt_float_to_fp8(__fmul_rn(x, s), __NV_SATFINITE, __NV_E4M3);
  }
};
template <>
struct Caster<2> {
  using T = __nv_bfloat16;
  __device__ static void cvt(float x, float, T& o0, T& o1) {
    o0 = __float2bfloat16_rn(x);
    o1 = __float2bfloat16_rn(__fsub_rn(x, __bfloat162float(o0)));
  }
};

// Row-major cast without transpose: four elements per thread per step.
// PRO: the prologue program `pro` runs on each element before the cast.
template <int KIND, bool PRO>
__global__ void cast_rows(const float* __restrict__ in, int64_t rows, int64_t cols, int64_t ld_in,
                          const float* __restrict__ amax, typename Caster<KIND>::T* __restrict__ o0,
                          typename Caster<KIND>::T* __restrict__ o1, int64_t ld_out,
                          float* scale_out, const __grid_constant__ EwProg pro) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  using T = typename Caster<KIND>::T;
  const float s = KIND == 1 ? fp8_scale_of(amax) : 1.f;
  if (scale_out && blockIdx.x == 0 && threadIdx.x == 0) *scale_out = s;
  const int64_t cq = (cols + 3) / 4;
  const int64_t total = rows * cq;
  const bool vec = (cols % 4 == 0) && (ld_in % 4 == 0) &&
                   ((reinterpret_cast<uintptr_t>(in) & 15) == 0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cq, c = (i % cq) * 4;
    float v[4];
    if (vec) {
      float4 q = __ldg(reinterpret_cast<const float4*>(in + r * ld_in + c));
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = (c + j < cols) ? in[r * ld_in + c + j] : 0.f;
    }
    if constexpr (PRO) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (c + j < cols) v[j] = ew_run(pro, v[j], r * ld_in + c + j);
    }
    T a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) Caster<KIND>::cvt(v[j], s, a[j], b[j]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (c + j < cols) {
        o0[r * ld_out + c + j] = a[j];
        if (KIND == 2) o1[r * ld_out + c + j] = b[j];
      }
    }
  }
}

// Transposing cast: a 64 x 64 tile through shared memory.  Reads are 128-bit
// along the input rows; writes pack 8 BF16 (or 16 E4M3) consecutive output
// elements into one 16-byte store, so both sides move whole sectors.
template <int KIND, bool PRO>
__global__ void __launch_bounds__(256) cast_transpose(const float* __restrict__ in, int64_t rows, int64_t cols,
                                                      int64_t ld_in, const float* __restrict__ amax,
                                                      typename Caster<KIND>::T* __restrict__ o0,
                                                      typename Caster<KIND>::T* __restrict__ o1, int64_t ld_out,
                                                      float* scale_out, const __grid_constant__ EwProg pro) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  using T = typename Caster<KIND>::T;
  constexpr int TS = 64;
  constexpr int VEC = sizeof(T) == 1 ? 16 : 8;      // output elements per 16-byte store
  __shared__ float tile[TS][TS + 1];
  const float s = KIND == 1 ? fp8_scale_of(amax) : 1.f;
  if (scale_out && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *scale_out = s;
  const int t = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * TS, c0 = (int64_t)blockIdx.x * TS;
  const bool vin = (ld_in % 4 == 0) && ((reinterpret_cast<uintptr_t>(in) & 15) == 0) && c0 + TS <= cols;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = t / 16 + 16 * i, cc = (t % 16) * 4;
    const int64_t r = r0 + rr, c = c0 + cc;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (r < rows) {
      if (vin) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(in + r * ld_in + c));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (c + j < cols) v[j] = in[r * ld_in + c + j];
      }
      if constexpr (PRO) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (c + j < cols) v[j] = ew_run(pro, v[j], r * ld_in + c + j);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) tile[rr][cc + j] = v[j];
  }
  __syncthreads();
  // output row c0 + oc holds input column oc; its elements are input rows r0 ..
  constexpr int CHUNKS = TS / VEC;
  const bool vout = ((ld_out * (int64_t)sizeof(T)) % 16 == 0) &&
                    ((reinterpret_cast<uintptr_t>(o0) & 15) == 0) &&
                    (KIND != 2 || (reinterpret_cast<uintptr_t>(o1) & 15) == 0);
  for (int idx = t; idx < TS * CHUNKS; idx += 256) {
    const int oc = idx / CHUNKS, rc = (idx % CHUNKS) * VEC;
    const int64_t orow = c0 + oc, ocol = r0 + rc;
    if (orow >= cols) continue;
    T a[VEC], b[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) Caster<KIND>::cvt(tile[rc + j][oc], s, a[j], b[j]);
    T* d0 = o0 + orow * ld_out + ocol;
    if (vout && ocol + VEC <= rows) {
      *reinterpret_cast<uint4*>(d0) = *reinterpret_cast<const uint4*>(a);
      if (KIND == 2) *reinterpret_cast<uint4*>(o1 + orow * ld_out + ocol) = *reinterpret_cast<const uint4*>(b);
    } else {
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        if (ocol + j < rows) {
          d0[j] = a[j];
          if (KIND == 2) o1[orow * ld_out + ocol + j] = b[j];
        }
      }
    }
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order FP64 block sums: thread i of block b visits elements
// b*blockDim + i + k*gridDim*blockDim; warp tree, then a tree over warps.
__global__ void norm_stage1(const float* __restrict__ C, int64_t ldc, const double* __restrict__ R,
                            int64_t ldr, int64_t M, int64_t N, double* __restrict__ partial) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  double e = 0.0, r2 = 0.0;
  const int64_t total = M * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = i / N, n = i % N;
    const double r = R[m * ldr + n];
    const double d = (double)C[m * ldc + n] - r;
    e = fma(d, d, e);
    r2 = fma(r, r, r2);
  }
  __shared__ double se[32], sr[32];
  e = warp_sum_d(e);
  r2 = warp_sum_d(r2);
  if ((threadIdx.x & 31) == 0) { se[threadIdx.x / 32] = e; sr[threadIdx.x / 32] = r2; }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x / 32;
    double a = threadIdx.x < nw ? se[threadIdx.x] : 0.0;
    double b = threadIdx.x < nw ? sr[threadIdx.x] : 0.0;
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    if (threadIdx.x == 0) { partial[2 * blockIdx.x] = a; partial[2 * blockIdx.x + 1] = b; }
  }
}

__global__ void norm_stage2(const double* __restrict__ partial, int n, double* __restrict__ out) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  double e = 0.0, r2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) { e += partial[2 * i]; r2 += partial[2 * i + 1]; }
  __shared__ double se[32], sr[32];
  e = warp_sum_d(e);
  r2 = warp_sum_d(r2);
  if ((threadIdx.x & 31) == 0) { se[threadIdx.x / 32] = e; sr[threadIdx.x / 32] = r2; }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x / 32;
    double a = threadIdx.x < nw ? se[threadIdx.x] : 0.0;
    double b = threadIdx.x < nw ? sr[threadIdx.x] : 0.0;
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    if (threadIdx.x == 0) { out[0] = a; out[1] = b; }
  }
}

template <int KIND, bool PRO>
nk_status launch_cast(const float* in, int64_t rows, int64_t cols, int64_t ld_in,
                      const float* amax, void* out0, void* out1, int64_t ld_out, int transpose,
                      float* scale_out, cudaStream_t st, int sms, const EwProg& pro) {
  using T = typename Caster<KIND>::T;
  T* o0 = static_cast<T*>(out0);
  T* o1 = static_cast<T*>(out1);
  if (transpose) {
    dim3 grid((unsigned)((cols + 63) / 64), (unsigned)((rows + 63) / 64));
    if (grid.y > 65535) return fail(NK_ERR_UNSUPPORTED, "too many rows for the transposing cast");
    (void)nk::launch_k(cast_transpose<KIND, PRO>, dim3(grid), dim3(256), 0, st, 1, in, rows, cols, ld_in, amax, o0, o1, ld_out, scale_out, pro);
  } else {
    const int64_t work = rows * ((cols + 3) / 4);
    int64_t blocks = (work + 255) / 256;
    const int64_t cap = (int64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    (void)nk::launch_k(cast_rows<KIND, PRO>, dim3((unsigned)blocks), dim3(256), 0, st, 1, in, rows, cols, ld_in, amax, o0, o1, ld_out,
                                                            scale_out, pro);
  }
  return check_launch("cast kernel");
}

template <int KIND>
nk_status launch_cast(const float* in, int64_t rows, int64_t cols, int64_t ld_in, const float* amax,
                      void* out0, void* out1, int64_t ld_out, int transpose, float* scale_out, cudaStream_t st,
                      int sms, const EwProg* pro) {
  if (pro && pro->n)
    return launch_cast<KIND, true>(in, rows, cols, ld_in, amax, out0, out1, ld_out, transpose, scale_out, st, sms,
                                   *pro);
  return launch_cast<KIND, false>(in, rows, cols, ld_in, amax, out0, out1, ld_out, transpose, scale_out, st, sms,
                                  EwProg{});
}

// Y = prog(X) over a rank-4 (padded) strided tensor: one element per thread
// per step, grid-stride.  `dense`: X, Y and the operands are one contiguous
// run, handled as float4 (the element offset is the flat index).
__global__ void ew_dense_kernel(const float* x, float* y, int64_t n,
                                const __grid_constant__ EwProg prog) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  const int64_t n4 = n / 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 v = reinterpret_cast<const float4*>(x)[i];
    float4 o;
    o.x = ew_run(prog, v.x, 4 * i);
    o.y = ew_run(prog, v.y, 4 * i + 1);
    o.z = ew_run(prog, v.z, 4 * i + 2);
    o.w = ew_run(prog, v.w, 4 * i + 3);
    reinterpret_cast<float4*>(y)[i] = o;
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = ew_run(prog, x[i], i);
}

struct Strided4 {
  int64_t shape[4];
  int64_t sx[4], sy[4];
};

__global__ void ew_strided_kernel(const float* x, float* y, int64_t n, const __grid_constant__ Strided4 g,
                                  const __grid_constant__ EwProg prog) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i, ox = 0, oy = 0;
#pragma unroll
    for (int d = 3; d >= 0; --d) {
      const int64_t id = r % g.shape[d];
      r /= g.shape[d];
      ox += id * g.sx[d];
      oy += id * g.sy[d];
    }
    y[oy] = ew_run(prog, x[ox], oy);
  }
}

}  // namespace

size_t prep_amax_ws(int64_t) { return kAmaxBlocks * sizeof(float); }

nk_status prep_amax(const float* x, int64_t rows, int64_t cols, int64_t ld, float* amax, void* ws,
                    size_t ws_bytes, cudaStream_t st, const EwProg* pro) {
  if (!amax) return fail(NK_ERR_INVALID_ARG, "amax: null pointer");
  if (rows * cols == 0) {   // max over nothing: 0 (the scale then falls back to 1)
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(float), st);
    return e == cudaSuccess ? NK_OK : cuda_fail(e, "cudaMemsetAsync(amax)");
  }
  if (!x) return fail(NK_ERR_INVALID_ARG, "amax: null pointer");
  if (!ws || ws_bytes < prep_amax_ws(rows * cols))
    return fail(NK_ERR_WORKSPACE, "amax needs %zu bytes of workspace", prep_amax_ws(rows * cols));
  if (pro && pro->n)
    (void)nk::launch_k(amax_stage1<true>, dim3(kAmaxBlocks), dim3(256), 0, st, 1, x, rows, cols, ld, static_cast<float*>(ws), *pro);
  else
    (void)nk::launch_k(amax_stage1<false>, dim3(kAmaxBlocks), dim3(256), 0, st, 1, x, rows, cols, ld, static_cast<float*>(ws), EwProg{});
  nk_status s = check_launch("amax_stage1");
  if (s != NK_OK) return s;
  (void)nk::launch_k(amax_stage2, dim3(1), dim3(1024), 0, st, 1, static_cast<float*>(ws), kAmaxBlocks, amax);
  return check_launch("amax_stage2");
}

nk_status prep_cast(int kind, const float* in, int64_t rows, int64_t cols, int64_t ld_in,
                    const float* amax, void* out0, void* out1, int64_t ld_out, int transpose,
                    float* scale_out, cudaStream_t st, const EwProg* pro) {
  int sms = 0;
  nk_status s = require_device(&sms);
  if (s != NK_OK) return s;
  if (rows <= 0 || cols <= 0) return NK_OK;
  switch (kind) {
    case 0: return launch_cast<0>(in, rows, cols, ld_in, amax, out0, out1, ld_out, transpose, scale_out, st, sms, pro);
    case 1: return launch_cast<1>(in, rows, cols, ld_in, amax, out0, out1, ld_out, transpose, scale_out, st, sms, pro);
    case 2: return launch_cast<2>(in, rows, cols, ld_in, amax, out0, out1, ld_out, transpose, scale_out, st, sms, pro);
    default: return fail(NK_ERR_INVALID_ARG, "unknown cast kind %d", kind);
  }
}

nk_status ew_tensor(const float* x, const int64_t* sx, float* y, const int64_t* sy, const int64_t* shape, int rank,
                    const EwProg& prog, cudaStream_t st) {
  int sms = 0;
  nk_status s = require_device(&sms);
  if (s != NK_OK) return s;
  Strided4 g{};
  int64_t n = 1;
  for (int d = 0; d < 4; ++d) {
    const int src = d - (4 - rank);   // leading dimensions pad to extent 1
    g.shape[d] = src >= 0 ? shape[src] : 1;
    g.sx[d] = src >= 0 ? sx[src] : 0;
    g.sy[d] = src >= 0 ? sy[src] : 0;
    n *= g.shape[d];
  }
  if (n == 0) return NK_OK;
  // dense row-major X and Y with the same strides: one flat run
  bool dense = true;
  int64_t run = 1;
  for (int d = 3; d >= 0; --d) {
    if (g.shape[d] != 1 && (g.sx[d] != run || g.sy[d] != run)) dense = false;
    run *= g.shape[d];
  }
  const int64_t per = dense ? (n + 3) / 4 : n;
  int64_t blocks = (per + 255) / 256;
  if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
  if (blocks < 1) blocks = 1;
  const bool al = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
  if (dense && al) (void)nk::launch_k(ew_dense_kernel, dim3((unsigned)blocks), dim3(256), 0, st, 1, x, y, n, prog);
  else (void)nk::launch_k(ew_strided_kernel, dim3((unsigned)blocks), dim3(256), 0, st, 1, x, y, n, g, prog);
  return check_launch("elementwise kernel");
}

size_t norm_ws(int64_t, int64_t) { return 2 * kNormBlocks * sizeof(double); }

nk_status norm_sumsq(const float* C, int64_t ldc, const double* R, int64_t ldr, int64_t M,
                     int64_t N, double* out, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!ws || ws_bytes < norm_ws(M, N))
    return fail(NK_ERR_WORKSPACE, "norm needs %zu bytes of workspace", norm_ws(M, N));
  double* part = static_cast<double*>(ws);
  (void)nk::launch_k(norm_stage1, dim3(kNormBlocks), dim3(256), 0, st, 1, C, ldc, R, ldr, M, N, part);
  nk_status s = check_launch("norm_stage1");
  if (s != NK_OK) return s;
  (void)nk::launch_k(norm_stage2, dim3(1), dim3(1024), 0, st, 1, part, kNormBlocks, out);
  return check_launch("norm_stage2");
}

}  // namespace nk
