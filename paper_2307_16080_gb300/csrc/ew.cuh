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
#endif

}  // namespace nk
