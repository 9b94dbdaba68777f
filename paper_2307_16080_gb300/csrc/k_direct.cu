// k_direct.cu -- the convolution of Sec. 4.1 Listing "2dnchwconv" as written:
// NCHW input, FCHW kernel, output-parallel,
//   out[n,co,ho,wo] += in[n, ci, ho*sh + ki*dh - pt, wo*sw + kj*dw - pl] * ker[co,ci,ki,kj]
// (stride 1, no padding in the listing; stride, dilation and zero padding
// here).  With a handful of channels -- the tuning experiment of Sec. 4.3
// uses (N, C, H, W) = (1, 1, 1280, 1280) and (Ci, Co, K) = (1, 3, 3) -- the
// contraction is far too short for tensor cores and the kernel is bound by
// HBM: each input element is read once through a shared-memory halo tile,
// each output element written once with 128-bit stores.
//
// Two kernels:
//   direct_rows_kernel (stride 1, dilation 1, 1x1 / 3x3 / 5x5 filters): each
//     thread owns 4 consecutive output columns of ROWS consecutive rows for
//     up to CO_G output channels and walks down the ROWS + KH - 1 input rows
//     it needs, one register segment of 4 + KW - 1 values per row (each input
//     row feeds every output row and tap that uses it), so the input is read
//     from DRAM once, with no shared memory and no index division; the
//     filter taps of an input channel sit in registers.  Outputs leave as
//     16-byte (or, on rows that are only 8-byte aligned, 8-byte) stores.
//   direct_stream_kernel (the same filters, one input channel -- the tuning
//     experiment's Ci = 1): as above, but a thread walks `rpt` output rows
//     keeping only KH rotating accumulator rows; an output row is stored as
//     soon as its last tap row has arrived, so the halo rows are amortised
//     over many rows and the stores spread through the loop.
//   direct_conv_kernel (any stride / dilation / filter up to 64 taps): a CTA
//     computes a 16 x 64 output tile of one image for up to 8 output
//     channels from a halo tile staged in shared memory, one input channel
//     at a time.
#include <cuda_runtime.h>

#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int TH = 16, TW = 64, CO_G = 8, THREADS = 256;
constexpr int MAX_IN_H = 64, MAX_IN_W = 176;   // halo tile limits (44 KB of shared memory)

struct Direct {
  const float* I;
  int64_t sIn, sIc, sIh;   // input strides (width stride 1)
  const float* Kr;         // FCHW, contiguous
  float* O;
  int64_t sOn, sOc, sOh;   // output strides (width stride 1)
  int N, CI, H, W, CO, KH, KW, OH, OW;
  int sh, sw, dh, dw, pt, pl;
  const float* bias;
  int relu;
  float beta;
  int in_h, in_w;          // halo tile extent
  EwProg ew;               // fused elementwise program (offsets from O)
};

// Shared memory is sized to the actual halo tile (18 x 66 floats for a 3 x 3
// stride-1 filter), so many CTAs share an SM and keep enough loads in flight
// to reach HBM bandwidth.
__global__ void __launch_bounds__(THREADS) direct_conv_kernel(const __grid_constant__ Direct p) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  extern __shared__ float smem_f[];
  float* ker = smem_f;                    // [CO_G][64] taps of one input channel
  float* tile = smem_f + CO_G * 64;       // [in_h][in_w] halo tile
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int wo0 = blockIdx.x * TW, ho0 = blockIdx.y * TH;
  const int n = blockIdx.z / ((p.CO + CO_G - 1) / CO_G);
  const int cg = blockIdx.z % ((p.CO + CO_G - 1) / CO_G);
  const int co0 = cg * CO_G;
  const int ncog = min(CO_G, p.CO - co0);
  const int ho = ho0 + ty;
  const int wo = wo0 + tx * 4;
  const int taps = p.KH * p.KW;
  const int ih0 = ho0 * p.sh - p.pt, iw0 = wo0 * p.sw - p.pl;
  float acc[CO_G][4];
#pragma unroll
  for (int c = 0; c < CO_G; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[c][j] = 0.f;

  for (int ci = 0; ci < p.CI; ++ci) {
    __syncthreads();
    const float* src = p.I + n * p.sIn + ci * p.sIc;
    // Eight loads in flight per thread before any lands in shared memory.
    const int total = p.in_h * p.in_w;
    for (int e0 = threadIdx.x; e0 < total; e0 += 8 * THREADS) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * THREADS;
        const int r = e / p.in_w, c = e - r * p.in_w;
        const int ih = ih0 + r, iw = iw0 + c;
        v[u] = (e < total && ih >= 0 && ih < p.H && iw >= 0 && iw < p.W) ? __ldg(src + ih * p.sIh + iw) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e0 + u * THREADS < total) tile[e0 + u * THREADS] = v[u];
    }
    for (int e = threadIdx.x; e < ncog * taps; e += THREADS) {
      const int c = e / taps, t = e % taps;
      ker[c * 64 + t] = __ldg(p.Kr + ((int64_t)(co0 + c) * p.CI + ci) * taps + t);
    }
    __syncthreads();
    for (int ki = 0; ki < p.KH; ++ki) {
      const int r = ty * p.sh + ki * p.dh;
      for (int kj = 0; kj < p.KW; ++kj) {
        float x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = tile[r * p.in_w + (tx * 4 + j) * p.sw + kj * p.dw];
        const int t = ki * p.KW + kj;
#pragma unroll
        for (int c = 0; c < CO_G; ++c) {
          if (c < ncog) {
            const float w = ker[c * 64 + t];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[c][j] = fmaf(x[j], w, acc[c][j]);
          }
        }
      }
    }
  }
  if (ho >= p.OH) return;
#pragma unroll
  for (int c = 0; c < CO_G; ++c) {
    if (c >= ncog) break;
    float* dst = p.O + n * p.sOn + (int64_t)(co0 + c) * p.sOc + (int64_t)ho * p.sOh + wo;
    const float b = p.bias ? p.bias[co0 + c] : 0.f;
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float o = acc[c][j];
      if (p.beta != 0.f && wo + j < p.OW) o = fmaf(p.beta, dst[j], o);
      o += b;
      if (p.relu) o = (o > 0.f || o != o) ? o : 0.f;
      if (p.ew.n && wo + j < p.OW) o = ew_run(p.ew, o, (dst - p.O) + j);
      v[j] = o;
    }
    if (wo + 3 < p.OW && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
      *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (wo + j < p.OW) dst[j] = v[j];
    }
  }
}

// Input segment x[0..SEG) = row ih, columns iw0 .. iw0+SEG-1, zero outside.
template <int SEG>
__device__ __forceinline__ void load_segment(const float* src, int64_t sIh, int H, int W, int ih, int iw0,
                                             float (&x)[SEG]) {
  if (ih < 0 || ih >= H) {
#pragma unroll
    for (int j = 0; j < SEG; ++j) x[j] = 0.f;
    return;
  }
  const float* row = src + (int64_t)ih * sIh;
  if (iw0 >= 0 && iw0 + SEG <= W) {
    const float* q = row + iw0;
    if (SEG >= 4 && (reinterpret_cast<uintptr_t>(q) & 15) == 0) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(q));
      x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
#pragma unroll
      for (int j = 4; j < SEG; ++j) x[j] = __ldg(q + j);
    } else {
#pragma unroll
      for (int j = 0; j < SEG; ++j) x[j] = __ldg(q + j);
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int iw = iw0 + j;
    x[j] = (iw >= 0 && iw < W) ? __ldg(row + iw) : 0.f;
  }
}

template <int KH, int KW, int CO_G, int ROWS>
__global__ void __launch_bounds__(128) direct_rows_kernel(const __grid_constant__ Direct p) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  constexpr int SEG = 4 + KW - 1;
  constexpr int TAPS = KH * KW;
  const int wo = blockIdx.x * 512 + threadIdx.x * 4;   // first of this thread's 4 output columns
  const int ho0 = blockIdx.y * ROWS;
  const int groups = (p.CO + CO_G - 1) / CO_G;
  const int n = blockIdx.z / groups;
  const int co0 = (blockIdx.z % groups) * CO_G;
  const int ncog = min(CO_G, p.CO - co0);
  if (wo >= p.OW) return;
  float acc[ROWS][CO_G][4];
#pragma unroll
  for (int r = 0; r < ROWS; ++r)
#pragma unroll
    for (int c = 0; c < CO_G; ++c)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[r][c][j] = 0.f;
  for (int ci = 0; ci < p.CI; ++ci) {
    float w[CO_G][TAPS];
#pragma unroll
    for (int c = 0; c < CO_G; ++c)
#pragma unroll
      for (int t = 0; t < TAPS; ++t)
        w[c][t] = c < ncog ? __ldg(p.Kr + ((int64_t)(co0 + c) * p.CI + ci) * TAPS + t) : 0.f;
    const float* src = p.I + n * p.sIn + ci * p.sIc;
#pragma unroll
    for (int r = 0; r < ROWS + KH - 1; ++r) {   // input row ho0 + r - pt
      float x[SEG];
      load_segment<SEG>(src, p.sIh, p.H, p.W, ho0 + r - p.pt, wo - p.pl, x);
#pragma unroll
      for (int kh = 0; kh < KH; ++kh) {
        const int orow = r - kh;   // the output row this input row meets through tap row kh
        if (orow < 0 || orow >= ROWS) continue;
#pragma unroll
        for (int c = 0; c < CO_G; ++c)
#pragma unroll
          for (int kw = 0; kw < KW; ++kw)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[orow][c][j] = fmaf(x[j + kw], w[c][kh * KW + kw], acc[orow][c][j]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int ho = ho0 + r;
    if (ho >= p.OH) break;
#pragma unroll
    for (int c = 0; c < CO_G; ++c) {
      if (c >= ncog) break;
      float* dst = p.O + n * p.sOn + (int64_t)(co0 + c) * p.sOc + (int64_t)ho * p.sOh + wo;
      const float b = p.bias ? __ldg(p.bias + co0 + c) : 0.f;
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float o = acc[r][c][j];
        if (p.beta != 0.f && wo + j < p.OW) o = fmaf(p.beta, dst[j], o);
        o += b;
        if (p.relu) o = (o > 0.f || o != o) ? o : 0.f;
        v[j] = o;
      }
      const uintptr_t a = reinterpret_cast<uintptr_t>(dst);
      if (wo + 3 < p.OW && (a & 15) == 0) {
        *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
      } else if (wo + 3 < p.OW && (a & 7) == 0) {
        *reinterpret_cast<float2*>(dst) = make_float2(v[0], v[1]);
        *reinterpret_cast<float2*>(dst + 2) = make_float2(v[2], v[3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (wo + j < p.OW) dst[j] = v[j];
      }
    }
  }
}

// Epilogue and store of 4 consecutive outputs of one row and channel.
__device__ __forceinline__ void store4(const Direct& p, float* dst, int wo, float b, const float (&a)[4]) {
  float v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float o = a[j];
    if (p.beta != 0.f && wo + j < p.OW) o = fmaf(p.beta, dst[j], o);
    o += b;
    if (p.relu) o = (o > 0.f || o != o) ? o : 0.f;
    v[j] = o;
  }
  const uintptr_t ad = reinterpret_cast<uintptr_t>(dst);
  if (wo + 3 < p.OW && (ad & 15) == 0) {
    *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
  } else if (wo + 3 < p.OW && (ad & 7) == 0) {
    *reinterpret_cast<float2*>(dst) = make_float2(v[0], v[1]);
    *reinterpret_cast<float2*>(dst + 2) = make_float2(v[2], v[3]);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (wo + j < p.OW) dst[j] = v[j];
  }
}

// One input channel: output row o lives in accumulator slot o % KH while
// input rows o .. o+KH-1 arrive; it is stored after the last of them.
template <int KH, int KW, int CO_G>
__global__ void __launch_bounds__(128) direct_stream_kernel(const __grid_constant__ Direct p, int rpt) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  constexpr int SEG = 4 + KW - 1;
  constexpr int TAPS = KH * KW;
  const int wo = blockIdx.x * 512 + threadIdx.x * 4;
  const int ho0 = blockIdx.y * rpt;
  const int groups = (p.CO + CO_G - 1) / CO_G;
  const int n = blockIdx.z / groups;
  const int co0 = (blockIdx.z % groups) * CO_G;
  const int ncog = min(CO_G, p.CO - co0);
  if (wo >= p.OW || ho0 >= p.OH) return;
  const int rows = min(rpt, p.OH - ho0);
  float w[CO_G][TAPS];
#pragma unroll
  for (int c = 0; c < CO_G; ++c)
#pragma unroll
    for (int t = 0; t < TAPS; ++t) w[c][t] = c < ncog ? __ldg(p.Kr + (int64_t)(co0 + c) * TAPS + t) : 0.f;
  float bias[CO_G];
#pragma unroll
  for (int c = 0; c < CO_G; ++c) bias[c] = (p.bias && c < ncog) ? __ldg(p.bias + co0 + c) : 0.f;
  float acc[KH][CO_G][4];
#pragma unroll
  for (int i = 0; i < KH; ++i)
#pragma unroll
    for (int c = 0; c < CO_G; ++c)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][c][j] = 0.f;
  const float* src = p.I + n * p.sIn;
  float* dst0 = p.O + n * p.sOn + (int64_t)co0 * p.sOc + wo;
  const int nin = rows + KH - 1;   // input rows ho0 - pt .. ho0 - pt + nin - 1
  for (int r0 = 0; r0 < nin; r0 += KH) {
#pragma unroll
    for (int u = 0; u < KH; ++u) {   // input row r = r0 + u, r0 a multiple of KH: slots are compile-time
      const int r = r0 + u;
      if (r >= nin) break;
      float x[SEG];
      load_segment<SEG>(src, p.sIh, p.H, p.W, ho0 + r - p.pt, wo - p.pl, x);
#pragma unroll
      for (int kh = 0; kh < KH; ++kh) {   // feeds output row r - kh through tap row kh
        const int o = r - kh;
        if (o < 0 || o >= rows) continue;
        const int slot = (u - kh + KH) % KH;
#pragma unroll
        for (int c = 0; c < CO_G; ++c)
#pragma unroll
          for (int kw = 0; kw < KW; ++kw)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[slot][c][j] = fmaf(x[j + kw], w[c][kh * KW + kw], acc[slot][c][j]);
      }
      const int o = r - (KH - 1);   // complete: its last tap row was this input row
      if (o >= 0 && o < rows) {
        const int slot = (u + 1) % KH;
#pragma unroll
        for (int c = 0; c < CO_G; ++c) {
          if (c >= ncog) break;
          store4(p, dst0 + (int64_t)c * p.sOc + (int64_t)(ho0 + o) * p.sOh, wo, bias[c], acc[slot][c]);
        }
#pragma unroll
        for (int c = 0; c < CO_G; ++c)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[slot][c][j] = 0.f;
      }
    }
  }
}

// Four output channels per thread keep the accumulators and taps in
// registers (eight with a 5 x 5 filter would spill).
template <int KH, int KW>
nk_status launch_rows(const Direct& p, cudaStream_t st) {
  constexpr int ROWS = 4, CO_R = 4;
  const int groups = (p.CO + CO_R - 1) / CO_R;
  if ((int64_t)p.N * groups > 65535) return fail(NK_ERR_UNSUPPORTED, "batch x channel groups too large");
  dim3 grid((unsigned)((p.OW + 511) / 512), (unsigned)((p.OH + ROWS - 1) / ROWS), (unsigned)(p.N * groups));
  if (grid.y > 65535) return fail(NK_ERR_UNSUPPORTED, "output too tall");
  (void)nk::launch_k(direct_rows_kernel<KH, KW, CO_R, ROWS>, dim3(grid), dim3(128), 0, st, 1, p);
  return check_launch("direct_rows_kernel");
}

// One input channel: rows per thread chosen so the grid makes about four
// waves of resident CTAs (6 per SM at this kernel's register count), which
// keeps the last wave's tail short; at least 4, at most 64 rows.
template <int KH, int KW>
nk_status launch_stream(const Direct& p, cudaStream_t st) {
  constexpr int CO_R = 4;
  int sms = 152;
  nk_status s = require_device(&sms);
  if (s != NK_OK) return s;
  const int groups = (p.CO + CO_R - 1) / CO_R;
  if ((int64_t)p.N * groups > 65535) return fail(NK_ERR_UNSUPPORTED, "batch x channel groups too large");
  const int64_t ctas_per_row = (int64_t)((p.OW + 511) / 512) * p.N * groups;
  const int64_t target = (int64_t)sms * 6 * 4;
  int64_t rpt = ((int64_t)p.OH * ctas_per_row + target - 1) / target;
  rpt = rpt < 4 ? 4 : rpt > 64 ? 64 : rpt;
  dim3 grid((unsigned)((p.OW + 511) / 512), (unsigned)((p.OH + rpt - 1) / rpt), (unsigned)(p.N * groups));
  if (grid.y > 65535) return fail(NK_ERR_UNSUPPORTED, "output too tall");
  (void)nk::launch_k(direct_stream_kernel<KH, KW, CO_R>, dim3(grid), dim3(128), 0, st, 1, p, (int)rpt);
  return check_launch("direct_stream_kernel");
}

}  // namespace
}  // namespace nk

using namespace nk;

extern "C" nk_status nk_conv2d_nchw_fchw(const nk_tensor* I, const nk_tensor* K, nk_tensor* O,
                                         const int64_t stride[2], const int64_t dilation[2],
                                         const int64_t pad[4], const nk_epilogue* epi, void* stream) {
  nk::NvtxRange nvtx_range_("nk_conv2d_nchw_fchw");
  nk_status s = NK_OK;
  if (!I || !K || !O || !stride || !dilation || !pad) return fail(NK_ERR_INVALID_ARG, "null argument");
  if (I->rank != 4 || K->rank != 4 || O->rank != 4) return fail(NK_ERR_INVALID_ARG, "I, K, O must have rank 4");
  if (I->dtype != NK_F32 || K->dtype != NK_F32 || O->dtype != NK_F32)
    return fail(NK_ERR_UNSUPPORTED, "the direct NCHW convolution is FP32");
  if (I->stride[3] != 1 || O->stride[3] != 1) return fail(NK_ERR_UNSUPPORTED, "width must have unit stride");
  const int64_t taps = K->shape[2] * K->shape[3];
  if (K->stride[3] != 1 || K->stride[2] != K->shape[3] || K->stride[1] != taps ||
      K->stride[0] != K->shape[1] * taps)
    return fail(NK_ERR_UNSUPPORTED, "the kernel must be contiguous FCHW");
  if (I->shape[1] != K->shape[1]) return fail(NK_ERR_INVALID_ARG, "input channels differ from the kernel's");
  for (int i = 0; i < 2; ++i)
    if (stride[i] < 1 || dilation[i] < 1) return fail(NK_ERR_INVALID_ARG, "stride and dilation must be >= 1");
  for (int i = 0; i < 4; ++i)
    if (pad[i] < 0) return fail(NK_ERR_INVALID_ARG, "padding must be >= 0");
  Direct p{};
  p.N = (int)I->shape[0]; p.CI = (int)I->shape[1]; p.H = (int)I->shape[2]; p.W = (int)I->shape[3];
  p.CO = (int)K->shape[0]; p.KH = (int)K->shape[2]; p.KW = (int)K->shape[3];
  p.sh = (int)stride[0]; p.sw = (int)stride[1]; p.dh = (int)dilation[0]; p.dw = (int)dilation[1];
  p.pt = (int)pad[0]; p.pl = (int)pad[2];
  const int64_t oh = (p.H + pad[0] + pad[1] - p.dh * (p.KH - 1) - 1) / p.sh + 1;
  const int64_t ow = (p.W + pad[2] + pad[3] - p.dw * (p.KW - 1) - 1) / p.sw + 1;
  if (oh < 1 || ow < 1) return fail(NK_ERR_INVALID_ARG, "empty output");
  if (O->shape[0] != p.N || O->shape[1] != p.CO || O->shape[2] != oh || O->shape[3] != ow)
    return fail(NK_ERR_INVALID_ARG, "O must be [%d,%d,%lld,%lld]", p.N, p.CO, (long long)oh, (long long)ow);
  p.OH = (int)oh; p.OW = (int)ow;
  if (taps > 64) return fail(NK_ERR_UNSUPPORTED, "more than 64 filter taps");
  p.in_h = (TH - 1) * p.sh + (p.KH - 1) * p.dh + 1;
  p.in_w = (TW - 1) * p.sw + (p.KW - 1) * p.dw + 1;
  if (p.in_h > MAX_IN_H || p.in_w > MAX_IN_W)
    return fail(NK_ERR_UNSUPPORTED, "stride/dilation/filter too large for the direct kernel's halo tile");
  p.I = static_cast<const float*>(I->ptr);
  p.sIn = I->stride[0]; p.sIc = I->stride[1]; p.sIh = I->stride[2];
  p.Kr = static_cast<const float*>(K->ptr);
  p.O = static_cast<float*>(O->ptr);
  p.sOn = O->stride[0]; p.sOc = O->stride[1]; p.sOh = O->stride[2];
  const nk_epilogue e0{nullptr, 0, 0, 1.f, 1.f, nullptr, nullptr, nullptr};
  const nk_epilogue& E = epi ? *epi : e0;
  p.bias = E.bias;
  p.relu = E.relu;
  p.beta = E.accumulate ? 1.f : 0.f;
  if (E.pro_a || E.pro_b)
    return fail(NK_ERR_UNSUPPORTED, "the direct NCHW convolution takes no operand prologue");
  if ((s = ew_program(E.ew, O, &p.ew, "ew")) != NK_OK) return s;
  if ((s = require_device()) != NK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The register-streaming kernels carry no epilogue program (a call in
  // their loops would slow the plain path); a program goes to the general
  // kernel below.
  const bool plain = p.ew.n == 0;
  if (plain && p.sh == 1 && p.sw == 1 && p.dh == 1 && p.dw == 1 && p.CI == 1) {
    if (p.KH == 3 && p.KW == 3) return launch_stream<3, 3>(p, st);
    if (p.KH == 5 && p.KW == 5) return launch_stream<5, 5>(p, st);
    if (p.KH == 1 && p.KW == 1) return launch_stream<1, 1>(p, st);
  }
  if (plain && p.sh == 1 && p.sw == 1 && p.dh == 1 && p.dw == 1) {
    if (p.KH == 3 && p.KW == 3) return launch_rows<3, 3>(p, st);
    if (p.KH == 5 && p.KW == 5) return launch_rows<5, 5>(p, st);
    if (p.KH == 1 && p.KW == 1) return launch_rows<1, 1>(p, st);
  }
  const int groups = (p.CO + CO_G - 1) / CO_G;
  if ((int64_t)p.N * groups > 65535) return fail(NK_ERR_UNSUPPORTED, "batch x channel groups too large");
  dim3 grid((unsigned)((p.OW + TW - 1) / TW), (unsigned)((p.OH + TH - 1) / TH), (unsigned)(p.N * groups));
  if (grid.y > 65535) return fail(NK_ERR_UNSUPPORTED, "output too tall");
  const size_t smem = (size_t)(CO_G * 64 + p.in_h * p.in_w) * sizeof(float);
  (void)nk::launch_k(direct_conv_kernel, dim3(grid), dim3(THREADS), smem, st, 1, p);
  return check_launch("direct_conv_kernel");
}
