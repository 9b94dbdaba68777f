// ew.cuh -- fused elementwise programs (the nk_ew_program of nk.h) as the
// kernels see them, and the per-element interpreter they share.
//
// A program folds the linalg.generic loops that a lowering leaves around a
// contraction -- the bias-add loop of the lowered torch.nn.Linear (Sec. 2.1.2
// Listing "listing1") and the elementwise product of the GPUModule kernel
// (Sec. 3.1 Listing "gpumodules") -- into the kernel that produces (epilogue)
// or reads (prologue) the tensor.  Tensor operands share the layout of the
// tensor the program runs over, so an element's offset from that tensor's
// base also locates its operands.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nk.h"

namespace nk {

constexpr int kEwMax = NK_EW_MAX;

struct EwProg {
  int n;                    // 0 = no program
  int op[kEwMax];
  float a[kEwMax], b[kEwMax];
  const float* t[kEwMax];   // MUL / ADD operands (offset 0 = the tensor's base)
};

// The same program with every tensor operand moved by `off` elements (a
// kernel that sees a sub-range of the tensor, e.g. one filter tap).
inline EwProg ew_shift(EwProg e, int64_t off) {
  for (int i = 0; i < e.n; ++i)
    if (e.t[i]) e.t[i] += off;
  return e;
}

#ifdef __CUDACC__
// Runs program `e` on value x of the element at offset `off`.  Kept out of
// line: the unrolled epilogues call it per element only when a program is
// present, and the plain paths carry no extra code.  FP32 throughout; the
// transcendental steps call CUDA's erfcf / tanhf / expf, in forms without
// cancellation for negative x: Phi(x) = erfc(-x / sqrt 2) / 2, and
// (1 + tanh u) / 2 = 1 / (1 + e^(-2u)) for the tanh form of GELU.
static __device__ __noinline__ float ew_run(const EwProg& e, float x, int64_t off) {
  for (int i = 0; i < e.n; ++i) {
    const float a = e.a[i], b = e.b[i];
    switch (e.op[i]) {
      case NK_EW_MUL: x = __fmul_rn(x, e.t[i][off]); break;
      case NK_EW_ADD: x = __fadd_rn(x, e.t[i][off]); break;
      case NK_EW_AFFINE: x = __fmaf_rn(a, x, b); break;
      case NK_EW_RELU: x = (x > 0.f || x != x) ? x : 0.f; break;
      case NK_EW_GELU: x = 0.5f * x * erfcf(-x * 0.70710678118654752f); break;
      case NK_EW_GELU_TANH: {
        const float u = 0.79788456080286536f * fmaf(0.044715f * x, x * x, x);
        x = x / (1.f + expf(-2.f * u));
        break;
      }
      case NK_EW_SILU: x = x / (1.f + expf(-x)); break;
      case NK_EW_SIGMOID: x = 1.f / (1.f + expf(-x)); break;
      case NK_EW_TANH: x = tanhf(x); break;
      case NK_EW_CLAMP: x = x < a ? a : (x > b ? b : x); break;
      default: break;
    }
  }
  return x;
}

// Runs program `e` in place over the n consecutive floats at buf, the values
// of the elements whose offsets start at off0.  The tensor-core epilogues
// stage a 32-column segment in a local buffer, call this once, then store:
// the program reads its operands (which may alias the output) before the
// store, and the unrolled plain epilogue keeps no call in its body (a call
// there costs the plain path registers and speed even when no program is
// given).
static __device__ __noinline__ void ew_apply(const EwProg& e, float* buf, int n, int64_t off0) {
  for (int j = 0; j < n; ++j) buf[j] = ew_run(e, buf[j], off0 + j);
}

// 32-byte stores (one whole L2 sector per thread; the address must be
// 32-byte aligned).  The epilogues write one output row per lane, so a warp
// store touches 32 rows: with 16-byte stores each row's sector arrives in
// two halves, with these in one piece, and the L2 sees half the requests.
__device__ __forceinline__ void st_v8_f32(float* p, float a0, float a1, float a2, float a3, float a4, float a5,
                                          float a6, float a7) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a0), "f"(a1), "f"(a2),
               "f"(a3), "f"(a4), "f"(a5), "f"(a6), "f"(a7)
               : "memory");
}
__device__ __forceinline__ void st_v8_b32(void* p, const uint32_t* w) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]),
               "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
               : "memory");
}
// 32 consecutive FP32 values to a 32-byte aligned row segment.
__device__ __forceinline__ void store32_f32_v8(float* dst, const float* v) {
#pragma unroll
  for (int j = 0; j < 32; j += 8) st_v8_f32(dst + j, v[j], v[j + 1], v[j + 2], v[j + 3], v[j + 4], v[j + 5], v[j + 6], v[j + 7]);
}

// BF16 outputs (a convolution whose result feeds the next layer directly):
// the epilogue computes in FP32 as for an FP32 output, then rounds each
// value to BF16 with round-to-nearest-even (CUDA's conversion intrinsic).
// 32 consecutive values to a 16-byte aligned row segment: four 16-byte
// stores of eight BF16 each.
__device__ __forceinline__ void store32_bf16(__nv_bfloat16* dst, const float* v) {
#pragma unroll
  for (int j = 0; j < 32; j += 8) {
    __nv_bfloat162 h[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(v[j + 2 * e], v[j + 2 * e + 1]);
    *reinterpret_cast<uint4*>(dst + j) = *reinterpret_cast<const uint4*>(h);
  }
}
// The same to a 32-byte aligned segment in two 32-byte stores.
__device__ __forceinline__ void store32_bf16_v8(__nv_bfloat16* dst, const float* v) {
#pragma unroll
  for (int j = 0; j < 32; j += 16) {
    __nv_bfloat162 h[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) h[e] = __floats2bfloat162_rn(v[j + 2 * e], v[j + 2 * e + 1]);
    st_v8_b32(dst + j, reinterpret_cast<const uint32_t*>(h));
  }
}
#endif

}  // namespace nk
