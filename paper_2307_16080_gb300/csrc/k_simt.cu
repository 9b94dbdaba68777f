// k_simt.cu -- FP32 contraction on the CUDA cores (the plain FP32 path).
//
// linalg.matmul C[m,n] (+)= sum_k A[m,k] B[k,n] (Sec. 2.1.1 Listing
// "linalg-matmul") and, through an implicit im2col A-operand, the NHWC/HWCF
// convolution of Sec. 4.1 Listing "2dnchwconv".  The loop nest is tiled the
// way Sec. 4.3 tunes it -- output tiles per CTA, a reduction depth per step --
// but written for sm_103: 256 threads per CTA, BMxBN tiles of 64 or 128,
// BK = 16, a double-buffered shared-memory ring fed by 128-bit loads,
// register blocking of (BM/16)x(BN/16) outputs per thread, and FFMA in FP32.
//
// Split-K: the reduction range is cut into `splits` slices (grid z); each
// slice writes its partial tile to the workspace and a second kernel sums the
// slices in a fixed order with a warp-shuffle tree, then applies the epilogue.
#include <cuda_runtime.h>

#include <mutex>

#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int BK = 16;
constexpr int THREADS = 256;

// Operand loading modes.
enum AMode { A_SCALAR = 0, A_KVEC = 1, A_MVEC = 2, A_CONV_VEC = 3, A_CONV_SCALAR = 4 };
enum BMode { B_SCALAR = 0, B_NVEC = 1, B_KVEC = 2 };

struct KArgs {
  SimtGemm p;
  int k_chunk;      // reduction length handled by one grid-z slice
  float* partial;   // [splits][M][N] or null
};

// Implicit im2col element A[m,k] of the convolution (0 outside the input);
// *off = its offset in the input, or -1 for the zero padding.
__device__ __forceinline__ float conv_a(const SimtGemm& p, int m, int k, int64_t* off) {
  const ConvGeom& g = p.conv;
  int ow = m % g.ow;
  int t = m / g.ow;
  int oh = t % g.oh;
  int n = t / g.oh;
  int c = k % g.c;
  int tap = k / g.c;
  int kw = tap % g.kw;
  int kh = tap / g.kw;
  int ih = oh * g.sh + kh * g.dh - g.pt;
  int iw = ow * g.sw + kw * g.dw - g.pl;
  if (ih < 0 || ih >= g.h || iw < 0 || iw >= g.w) {
    *off = -1;
    return 0.f;
  }
  *off = n * g.sin_n + ih * g.sin_h + iw * g.sin_w + c;
  return p.A[*off];
}

// Four consecutive k (same tap, since C % 4 == 0) of conv row m; *off as
// for conv_a, for the first of the four.
__device__ __forceinline__ float4 conv_a4(const SimtGemm& p, int m, int k, int64_t* off) {
  const ConvGeom& g = p.conv;
  int ow = m % g.ow;
  int t = m / g.ow;
  int oh = t % g.oh;
  int n = t / g.oh;
  int c = k % g.c;
  int tap = k / g.c;
  int kw = tap % g.kw;
  int kh = tap / g.kw;
  int ih = oh * g.sh + kh * g.dh - g.pt;
  int iw = ow * g.sw + kw * g.dw - g.pl;
  if (ih < 0 || ih >= g.h || iw < 0 || iw >= g.w) {
    *off = -1;
    return make_float4(0.f, 0.f, 0.f, 0.f);
  }
  *off = n * g.sin_n + ih * g.sin_h + iw * g.sin_w + c;
  return __ldg(reinterpret_cast<const float4*>(p.A + *off));
}

// Prologue on four loaded values whose offsets are off, off+d, off+2d, off+3d.
__device__ __forceinline__ void pro4(const EwProg& e, float4& v, int64_t off, int64_t d) {
  v.x = ew_run(e, v.x, off);
  v.y = ew_run(e, v.y, off + d);
  v.z = ew_run(e, v.z, off + 2 * d);
  v.w = ew_run(e, v.w, off + 3 * d);
}

// FUSED: the variant that runs prologue / epilogue programs (instantiated
// with the scalar load modes only); the plain variants carry no call.
template <int RM, int RN, int AM, int BMD, bool FUSED>
__global__ void __launch_bounds__(THREADS, 2) simt_gemm_kernel(const __grid_constant__ KArgs args) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  constexpr int BM = 64 * RM;
  constexpr int BN = 64 * RN;
  constexpr int APAD = 4;
  constexpr int A_LD = BM + APAD;
  constexpr int NA = BM * BK / THREADS;   // scalars of A each thread loads per tile
  constexpr int NB = BN * BK / THREADS;
  __shared__ __align__(16) float As[2][BK][A_LD];
  __shared__ __align__(16) float Bs[2][BK][BN];

  const SimtGemm& p = args.p;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * args.k_chunk;
  const int kend = min(p.K, kbeg + args.k_chunk);
  const int ntiles = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;

  float ra[NA];
  float rb[NB];

  auto load_a = [&](int k0) {
    if constexpr (AM == A_KVEC || AM == A_CONV_VEC) {
#pragma unroll
      for (int j = 0; j < NA / 4; ++j) {
        int L = tid + j * THREADS;
        int row = L / 4, kq = (L % 4) * 4;
        int m = m0 + row, k = k0 + kq;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m < p.M && k < kend) {
          int64_t off = (int64_t)m * p.sam + k;
          if constexpr (AM == A_KVEC)
            v = __ldg(reinterpret_cast<const float4*>(p.A + off));
          else
            v = conv_a4(p, m, k, &off);
          if (FUSED && p.pro_a.n && off >= 0) pro4(p.pro_a, v, off, 1);
        }
        ra[4 * j + 0] = v.x; ra[4 * j + 1] = v.y; ra[4 * j + 2] = v.z; ra[4 * j + 3] = v.w;
      }
    } else if constexpr (AM == A_MVEC) {
#pragma unroll
      for (int j = 0; j < NA / 4; ++j) {
        int L = tid + j * THREADS;
        int kk = L / (BM / 4), mq = (L % (BM / 4)) * 4;
        int m = m0 + mq, k = k0 + kk;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m < p.M && k < kend) {
          v = __ldg(reinterpret_cast<const float4*>(p.A + (int64_t)k * p.sak + m));
          if (FUSED && p.pro_a.n) pro4(p.pro_a, v, (int64_t)k * p.sak + m, 1);
        }
        ra[4 * j + 0] = v.x; ra[4 * j + 1] = v.y; ra[4 * j + 2] = v.z; ra[4 * j + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        int L = tid + j * THREADS;
        int row = L % BM, kk = L / BM;
        int m = m0 + row, k = k0 + kk;
        float v = 0.f;
        if (m < p.M && k < kend) {
          int64_t off = (int64_t)m * p.sam + (int64_t)k * p.sak;
          if constexpr (AM == A_CONV_SCALAR) v = conv_a(p, m, k, &off);
          else v = p.A[off];
          if (FUSED && p.pro_a.n && off >= 0) v = ew_run(p.pro_a, v, off);
        }
        ra[j] = v;
      }
    }
  };
  auto store_a = [&](int buf) {
    if constexpr (AM == A_KVEC || AM == A_CONV_VEC) {
#pragma unroll
      for (int j = 0; j < NA / 4; ++j) {
        int L = tid + j * THREADS;
        int row = L / 4, kq = (L % 4) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) As[buf][kq + i][row] = ra[4 * j + i];
      }
    } else if constexpr (AM == A_MVEC) {
#pragma unroll
      for (int j = 0; j < NA / 4; ++j) {
        int L = tid + j * THREADS;
        int kk = L / (BM / 4), mq = (L % (BM / 4)) * 4;
        *reinterpret_cast<float4*>(&As[buf][kk][mq]) =
            make_float4(ra[4 * j], ra[4 * j + 1], ra[4 * j + 2], ra[4 * j + 3]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        int L = tid + j * THREADS;
        As[buf][L / BM][L % BM] = ra[j];
      }
    }
  };
  auto load_b = [&](int k0) {
    if constexpr (BMD == B_NVEC) {
#pragma unroll
      for (int j = 0; j < NB / 4; ++j) {
        int L = tid + j * THREADS;
        int kk = L / (BN / 4), nq = (L % (BN / 4)) * 4;
        int n = n0 + nq, k = k0 + kk;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < p.N && k < kend) {
          v = __ldg(reinterpret_cast<const float4*>(p.B + (int64_t)k * p.sbk + n));
          if (FUSED && p.pro_b.n) pro4(p.pro_b, v, (int64_t)k * p.sbk + n, 1);
        }
        rb[4 * j + 0] = v.x; rb[4 * j + 1] = v.y; rb[4 * j + 2] = v.z; rb[4 * j + 3] = v.w;
      }
    } else if constexpr (BMD == B_KVEC) {
#pragma unroll
      for (int j = 0; j < NB / 4; ++j) {
        int L = tid + j * THREADS;
        int col = L / 4, kq = (L % 4) * 4;
        int n = n0 + col, k = k0 + kq;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < p.N && k < kend) {
          v = __ldg(reinterpret_cast<const float4*>(p.B + (int64_t)n * p.sbn + k));
          if (FUSED && p.pro_b.n) pro4(p.pro_b, v, (int64_t)n * p.sbn + k, 1);
        }
        rb[4 * j + 0] = v.x; rb[4 * j + 1] = v.y; rb[4 * j + 2] = v.z; rb[4 * j + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        int L = tid + j * THREADS;
        int col = L % BN, kk = L / BN;
        int n = n0 + col, k = k0 + kk;
        float v = 0.f;
        if (n < p.N && k < kend) {
          const int64_t off = (int64_t)k * p.sbk + (int64_t)n * p.sbn;
          v = p.B[off];
          if (FUSED && p.pro_b.n) v = ew_run(p.pro_b, v, off);
        }
        rb[j] = v;
      }
    }
  };
  auto store_b = [&](int buf) {
    if constexpr (BMD == B_NVEC) {
#pragma unroll
      for (int j = 0; j < NB / 4; ++j) {
        int L = tid + j * THREADS;
        int kk = L / (BN / 4), nq = (L % (BN / 4)) * 4;
        *reinterpret_cast<float4*>(&Bs[buf][kk][nq]) =
            make_float4(rb[4 * j], rb[4 * j + 1], rb[4 * j + 2], rb[4 * j + 3]);
      }
    } else if constexpr (BMD == B_KVEC) {
#pragma unroll
      for (int j = 0; j < NB / 4; ++j) {
        int L = tid + j * THREADS;
        int col = L / 4, kq = (L % 4) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) Bs[buf][kq + i][col] = rb[4 * j + i];
      }
    } else {
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        int L = tid + j * THREADS;
        Bs[buf][L / BN][L % BN] = rb[j];
      }
    }
  };

  float acc[RM * 4][RN * 4];
#pragma unroll
  for (int i = 0; i < RM * 4; ++i)
#pragma unroll
    for (int j = 0; j < RN * 4; ++j) acc[i][j] = 0.f;

  if (ntiles > 0) {
    load_a(kbeg);
    load_b(kbeg);
    store_a(0);
    store_b(0);
    __syncthreads();
  }
  for (int t = 0; t < ntiles; ++t) {
    const int buf = t & 1;
    const bool more = t + 1 < ntiles;
    if (more) {
      load_a(kbeg + (t + 1) * BK);
      load_b(kbeg + (t + 1) * BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[RM * 4], b[RN * 4];
#pragma unroll
      for (int r = 0; r < RM; ++r) {
        float4 v = *reinterpret_cast<const float4*>(&As[buf][kk][r * 64 + ty * 4]);
        a[4 * r] = v.x; a[4 * r + 1] = v.y; a[4 * r + 2] = v.z; a[4 * r + 3] = v.w;
      }
#pragma unroll
      for (int r = 0; r < RN; ++r) {
        float4 v = *reinterpret_cast<const float4*>(&Bs[buf][kk][r * 64 + tx * 4]);
        b[4 * r] = v.x; b[4 * r + 1] = v.y; b[4 * r + 2] = v.z; b[4 * r + 3] = v.w;
      }
#pragma unroll
      for (int i = 0; i < RM * 4; ++i)
#pragma unroll
        for (int j = 0; j < RN * 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store_a(buf ^ 1);
      store_b(buf ^ 1);
    }
    __syncthreads();
  }

  // Epilogue: partial tile to the workspace, or the fused epilogue to C.
#pragma unroll
  for (int i = 0; i < RM * 4; ++i) {
    const int m = m0 + (i / 4) * 64 + ty * 4 + (i % 4);
    if (m >= p.M) continue;
#pragma unroll
    for (int r = 0; r < RN; ++r) {
      const int nb = n0 + r * 64 + tx * 4;
      if (args.partial) {
        float* dst = args.partial + ((int64_t)blockIdx.z * p.M + m) * p.N;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (nb + j < p.N) dst[nb + j] = acc[i][4 * r + j];
        continue;
      }
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = nb + j;
        float o = p.alpha * acc[i][4 * r + j];
        if (n < p.N) {
          if (p.beta != 0.f) o = fmaf(p.beta, p.C[(int64_t)m * p.scm + (int64_t)n * p.scn], o);
          if (p.bias) o += p.bias[p.bias_on_m ? m : n];
          if (p.relu) o = (o > 0.f || o != o) ? o : 0.f;
          if (FUSED && p.ew.n) o = ew_run(p.ew, o, (int64_t)m * p.scm + (int64_t)n * p.scn);
        }
        v[j] = o;
      }
      float* crow = p.C + (int64_t)m * p.scm;
      if (p.scn == 1 && nb + 3 < p.N && ((reinterpret_cast<uintptr_t>(crow + nb) & 15) == 0)) {
        *reinterpret_cast<float4*>(crow + nb) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (nb + j < p.N) crow[(int64_t)(nb + j) * p.scn] = v[j];
      }
    }
  }
}

// Split-K reduce: lanes of a warp form groups of S (a power of two); lane
// s of a group reads slice s of one output, the group sums with an xor
// shuffle tree (same order every run), lane 0 applies the epilogue.
template <bool EW>
__global__ void splitk_reduce_kernel(const __grid_constant__ SplitReduce r, int S) {
  nk::pdl_wait();      // earlier kernels on the stream have finished
  nk::pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int per_warp = 32 / S;
  const int s = lane % S;
  const int64_t total = (int64_t)r.M * r.N;
  const int64_t warp = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x / 32);
  const float alpha = r.scale_a ? __frcp_rn(__fmul_rn(*r.scale_a, *r.scale_b)) : r.alpha;
  for (int64_t base = warp * per_warp; base < total; base += nwarps * per_warp) {
    const int64_t idx = base + lane / S;
    float v = 0.f;
    if (idx < total && s < r.splits) v = r.partial[(int64_t)s * total + idx];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
      if (off < S) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (s == 0 && idx < total) {
      const int m = (int)(idx / r.N), n = (int)(idx % r.N);
      const int64_t off = (int64_t)m * r.scm + (int64_t)n * r.scn;
      float* c = r.C + off;
      __nv_bfloat16* ch = reinterpret_cast<__nv_bfloat16*>(r.C) + off;
      float o = alpha * v;
      if (r.beta != 0.f) o = fmaf(r.beta, r.out_bf16 ? __bfloat162float(*ch) : *c, o);
      if (r.bias) o += r.bias[r.bias_on_m ? m : n];
      if (r.relu) o = (o > 0.f || o != o) ? o : 0.f;
      if (EW && r.ew.n) o = ew_run(r.ew, o, off);
      if (r.out_bf16) *ch = __float2bfloat16_rn(o);
      else *c = o;
    }
  }
}

template <int RM, int RN, int AM>
nk_status launch_b(const KArgs& a, int bmode, dim3 grid, cudaStream_t st) {
  switch (bmode) {
    case B_NVEC: (void)nk::launch_k(simt_gemm_kernel<RM, RN, AM, B_NVEC, false>, dim3(grid), dim3(THREADS), 0, st, 1, a); break;
    case B_KVEC: (void)nk::launch_k(simt_gemm_kernel<RM, RN, AM, B_KVEC, false>, dim3(grid), dim3(THREADS), 0, st, 1, a); break;
    default: (void)nk::launch_k(simt_gemm_kernel<RM, RN, AM, B_SCALAR, false>, dim3(grid), dim3(THREADS), 0, st, 1, a); break;
  }
  return check_launch("simt_gemm_kernel");
}

// Programs present: scalar loads of any layout, FUSED kernel.
template <int RM, int RN>
nk_status launch_fused(const KArgs& a, dim3 grid, cudaStream_t st) {
  if (a.p.is_conv)
    (void)nk::launch_k(simt_gemm_kernel<RM, RN, A_CONV_SCALAR, B_SCALAR, true>, dim3(grid), dim3(THREADS), 0, st, 1, a);
  else
    (void)nk::launch_k(simt_gemm_kernel<RM, RN, A_SCALAR, B_SCALAR, true>, dim3(grid), dim3(THREADS), 0, st, 1, a);
  return check_launch("simt_gemm_kernel");
}

template <int RM, int RN>
nk_status launch_a(const KArgs& a, int amode, int bmode, dim3 grid, cudaStream_t st) {
  switch (amode) {
    case A_KVEC: return launch_b<RM, RN, A_KVEC>(a, bmode, grid, st);
    case A_MVEC: return launch_b<RM, RN, A_MVEC>(a, bmode, grid, st);
    case A_CONV_VEC: return launch_b<RM, RN, A_CONV_VEC>(a, bmode, grid, st);
    case A_CONV_SCALAR: return launch_b<RM, RN, A_CONV_SCALAR>(a, bmode, grid, st);
    default: return launch_b<RM, RN, A_SCALAR>(a, bmode, grid, st);
  }
}

inline bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

size_t simt_gemm_ws(int M, int N, int splits) {
  return splits > 1 ? (size_t)splits * M * N * sizeof(float) : 0;
}

nk_status simt_gemm(const SimtGemm& p, int tile, int splits, void* ws, size_t ws_bytes,
                    cudaStream_t st) {
  if (p.M <= 0 || p.N <= 0) return NK_OK;
  if (tile != 64 && tile != 128) return fail(NK_ERR_INVALID_ARG, "SIMT tile must be 64 or 128");
  if (splits < 1 || splits > 32) return fail(NK_ERR_INVALID_ARG, "split_k must be in [1, 32]");
  KArgs a;
  a.p = p;
  int kc = (p.K + splits - 1) / splits;
  kc = (kc + BK - 1) / BK * BK;
  if (kc == 0) kc = BK;
  splits = p.K > 0 ? (p.K + kc - 1) / kc : 1;
  a.k_chunk = kc;
  a.partial = nullptr;
  if (splits > 1) {
    if (!ws || ws_bytes < simt_gemm_ws(p.M, p.N, splits))
      return fail(NK_ERR_WORKSPACE, "split-K needs %zu bytes of workspace",
                  simt_gemm_ws(p.M, p.N, splits));
    a.partial = static_cast<float*>(ws);
  }
  // Pick the load modes from the layout and alignment.
  int amode, bmode;
  if (p.is_conv) {
    const ConvGeom& g = p.conv;
    bool vec = (g.c % 4 == 0) && g.sin_n % 4 == 0 && g.sin_h % 4 == 0 && g.sin_w % 4 == 0 &&
               al16(p.A);
    amode = vec ? A_CONV_VEC : A_CONV_SCALAR;
  } else if (p.sak == 1 && p.sam % 4 == 0 && p.K % 4 == 0 && al16(p.A)) {
    amode = A_KVEC;
  } else if (p.sam == 1 && p.sak % 4 == 0 && p.M % 4 == 0 && al16(p.A)) {
    amode = A_MVEC;
  } else {
    amode = A_SCALAR;
  }
  if (p.sbn == 1 && p.sbk % 4 == 0 && p.N % 4 == 0 && al16(p.B)) bmode = B_NVEC;
  else if (p.sbk == 1 && p.sbn % 4 == 0 && p.K % 4 == 0 && al16(p.B)) bmode = B_KVEC;
  else bmode = B_SCALAR;
  dim3 grid((p.N + tile - 1) / tile, (p.M + tile - 1) / tile, splits);
  if (grid.y > 65535) return fail(NK_ERR_UNSUPPORTED, "M too large for the SIMT grid");
  nk_status s;
  if (p.pro_a.n || p.pro_b.n || p.ew.n)
    s = tile == 128 ? launch_fused<2, 2>(a, grid, st) : launch_fused<1, 1>(a, grid, st);
  else
    s = tile == 128 ? launch_a<2, 2>(a, amode, bmode, grid, st) : launch_a<1, 1>(a, amode, bmode, grid, st);
  if (s != NK_OK || splits == 1) return s;
  SplitReduce r{};
  r.partial = a.partial;
  r.splits = splits;
  r.M = p.M;
  r.N = p.N;
  r.C = p.C;
  r.scm = p.scm;
  r.scn = p.scn;
  r.bias = p.bias;
  r.bias_on_m = p.bias_on_m;
  r.alpha = p.alpha;
  r.beta = p.beta;
  r.relu = p.relu;
  r.scale_a = nullptr;
  r.scale_b = nullptr;
  r.ew = p.ew;
  return splitk_reduce(r, st);
}

nk_status splitk_reduce(const SplitReduce& r, cudaStream_t st) {
  if (r.splits < 1 || r.splits > 32) return fail(NK_ERR_INVALID_ARG, "splits must be in [1, 32]");
  int S = 1;
  while (S < r.splits) S <<= 1;
  int sms = 0;
  nk_status s = require_device(&sms);
  if (s != NK_OK) return s;
  const int64_t total = (int64_t)r.M * r.N;
  const int64_t warps_needed = (total + (32 / S) - 1) / (32 / S);
  int64_t blocks = (warps_needed + 7) / 8;
  blocks = blocks < (int64_t)sms * 8 ? blocks : (int64_t)sms * 8;
  if (blocks < 1) blocks = 1;
  if (r.ew.n) (void)nk::launch_k(splitk_reduce_kernel<true>, dim3((unsigned)blocks), dim3(256), 0, st, 1, r, S);
  else (void)nk::launch_k(splitk_reduce_kernel<false>, dim3((unsigned)blocks), dim3(256), 0, st, 1, r, S);
  return check_launch("splitk_reduce_kernel");
}

}  // namespace nk

// ------------------------------------------------- split-K without allocation
// For callers that cannot allocate device memory at all: code running where
// cudaMalloc is unavailable or forbidden (inside a custom allocator's
// callbacks, while another runtime owns the memory pool, or in a process
// whose device memory budget is already spoken for).  The split-K partial
// sums go to this fixed, file-scope device array instead of a caller
// workspace; every GPU that loads the library keeps it until exit.
namespace nk {
namespace {

constexpr size_t kStaticScratchFloats = size_t(4) << 20;   // 16 MiB of FP32 partials
__device__ __align__(256) float g_splitk_scratch[kStaticScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
float* g_scratch_addr[kMaxDevices];   // device address of g_splitk_scratch, per device ordinal

}  // namespace
}  // namespace nk

extern "C" nk_status nk_matmul_f32_splitk_noalloc(const float* A, int64_t lda, const float* B,
                                                  int64_t ldb, float* C, int64_t ldc, int32_t M,
                                                  int32_t N, int32_t K, int32_t split_k,
                                                  void* stream) {
  nk::NvtxRange nvtx_range_("nk_matmul_f32_splitk_noalloc");
  using namespace nk;
  int sms = 0;
  nk_status s = require_device(&sms);
  if (s != NK_OK) return s;
  if (M < 0 || N < 0 || K < 0) return fail(NK_ERR_INVALID_ARG, "negative extent");
  if (split_k < 1 || split_k > 32) return fail(NK_ERR_INVALID_ARG, "split_k must be in [1, 32]");
  if (M == 0 || N == 0) return NK_OK;
  if (!A || !B || !C) return fail(NK_ERR_INVALID_ARG, "null pointer");
  if (lda < K || ldb < N || ldc < N) return fail(NK_ERR_INVALID_ARG, "leading dimension too small");
  if ((size_t)split_k * (size_t)M * (size_t)N > kStaticScratchFloats)
    return fail(NK_ERR_WORKSPACE,
                "split_k*M*N = %zu exceeds the static scratch of %zu floats (16 MiB)",
                (size_t)split_k * M * N, kStaticScratchFloats);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return fail(NK_ERR_UNSUPPORTED, "device ordinal %d: the static scratch table holds %d devices", dev,
                kMaxDevices);
  float* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      // Host code only sees a host-side stand-in for the array; the device
      // address comes from the runtime, once per device, with it current.
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_splitk_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_splitk_scratch)");
      g_scratch_addr[dev] = static_cast<float*>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  SimtGemm p{};
  p.A = A; p.sam = lda; p.sak = 1;
  p.B = B; p.sbk = ldb; p.sbn = 1;
  p.C = C; p.scm = ldc; p.scn = 1;
  p.M = M; p.N = N; p.K = K;
  p.alpha = 1.f; p.beta = 0.f;
  // The tile nk_matmul's FP32 rule picks: 64 x 64 while 128 x 128 tiles
  // would not give every SM one.
  const int tile = (int64_t)((M + 127) / 128) * ((N + 127) / 128) < sms ? 64 : 128;
  // Every slice overwrites its whole [M,N] partial tile, so the scratch needs
  // no clearing between calls.
  return simt_gemm(p, tile, split_k, scratch, kStaticScratchFloats * sizeof(float),
                   static_cast<cudaStream_t>(stream));
}
