// nk_internal.cuh -- declarations shared by the translation units of libnk.
//
// Host side: error reporting, device checks and the internal launch entry
// points of each kernel family.  Device side: the global failure word that
// bounded waits set when they give up.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <utility>

#include "../../include/nk.h"
#include "ew.cuh"

namespace nk {

// ------------------------------------------------------------------ NVTX
// A named range on the calling host thread for as long as the object lives:
// every public compute call and each phase of the schedule search opens one,
// so a profiler's timeline shows which library call issued which kernels.
// NVTX is header-only here; without an attached tool a range costs a branch.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ----------------------------------------------------------------- errors
nk_status fail(nk_status s, const char* fmt, ...);
nk_status cuda_fail(cudaError_t e, const char* what);
nk_status check_launch(const char* what);

// Verifies that the current device is an sm_103 part; caches the answer per
// device.  Fills the SM count when `sms` is non-null.
nk_status require_device(int* sms = nullptr);

// Device-side failure word.  Bit 0: a bounded wait expired.  Each
// translation unit that owns waiting kernels defines its own copy; the host
// reads and clears all of them in nk_sync_status.
enum : uint32_t { kErrTimeout = 1u, kErrLaunch = 2u };   // kErrLaunch: too little shared memory

// Spin budget shared by the waiting kernels (set through nk_set_wait_budget).
int64_t wait_budget();

// ------------------------------------------ programmatic dependent launch
// A kernel started by launch_k() may begin while the kernel before it on the
// stream is still running.  It does its set-up that touches no global data
// (mbarrier init, TMEM allocation, prefetch of parameter-space tensor maps),
// then pdl_wait(), which returns once every earlier kernel on the stream has
// completed and its writes are visible, and only then reads or writes global
// memory.  It calls pdl_trigger() after pdl_wait(), so the kernel after it
// may start its own set-up.  Because a grid triggers only after its own wait,
// at most two grids overlap; the earlier one is fully resident (a dependent
// launches only once every CTA of the earlier grid has triggered or exited)
// and needs nothing from the later one, so a later CTA blocked in pdl_wait()
// or in a TMEM allocation cannot hold it up.  Launched without the attribute
// (nk_set_pdl(0)) both instructions do nothing.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

bool pdl_enabled();   // nk_set_pdl; on by default

// cudaLaunchKernelEx with the programmatic-serialization attribute (when
// enabled) and an optional cluster of `cluster` CTAs along x.  The kernel
// must follow the pdl_wait() rule above.
template <typename... Kargs, typename... Args>
inline cudaError_t launch_k(void (*kern)(Kargs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            int cluster, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  unsigned n = 0;
  if (pdl_enabled()) {
    attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
  }
  if (cluster > 1) {
    attr[n].id = cudaLaunchAttributeClusterDimension;
    attr[n].val.clusterDim.x = (unsigned)cluster;
    attr[n].val.clusterDim.y = 1;
    attr[n].val.clusterDim.z = 1;
    ++n;
  }
  cfg.attrs = n ? attr : nullptr;
  cfg.numAttrs = n;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Reads and clears the failure words of every translation unit.
nk_status collect_device_errors(uint32_t* flags);

// Median device time (ms) of one call of `run` (which enqueues its kernels
// on the stream it is given): graph replays of back-to-back calls on a
// library stream, behind a hold kernel, so host call overhead is not timed
// (tune.cu).  Successive calls of `run` may cycle through `cycle` buffer
// sets; every timed sample then covers a whole number of cycles.
using RunFn = std::function<nk_status(cudaStream_t)>;
nk_status time_device(const RunFn& run, int reps, float* ms, int cycle = 1);
uint32_t tc_read_and_clear_errors();   // tcgen05 GEMM / conv units

// ----------------------------------------------------------- SIMT (FP32)
// A[m,k] at A + m*sam + k*sak; B[k,n] at B + k*sbk + n*sbn;
// C[m,n] at C + m*scm + n*scn (one of scm, scn is 1).
struct ConvGeom {
  int n, h, w, c;          // input NHWC extents
  int kh, kw;              // filter taps
  int oh, ow;              // output extents
  int sh, sw, dh, dw, pt, pl;
  int64_t sin_n, sin_h, sin_w;  // input strides (channel stride is 1)
};

struct SimtGemm {
  const float* A;
  int64_t sam, sak;
  const float* B;
  int64_t sbk, sbn;
  float* C;
  int64_t scm, scn;
  const float* bias;
  int bias_on_m;         // bias indexed by m (transposed problems)
  int M, N, K;
  float alpha, beta;
  int relu;
  int is_conv;           // A is the implicit im2col matrix of `conv`
  ConvGeom conv;
  EwProg ew;             // epilogue program (offsets from C)
  EwProg pro_a, pro_b;   // prologues on the loaded A / B (offsets from A, B; conv: from I)
};

// tile: 128 or 64 (square CTA tile); splits >= 1.  When splits > 1 the
// partial sums go to `ws` ([splits][M][N] FP32) and a reduce pass applies
// the epilogue.
nk_status simt_gemm(const SimtGemm& p, int tile, int splits, void* ws, size_t ws_bytes,
                    cudaStream_t st);
size_t simt_gemm_ws(int M, int N, int splits);

// Fixed-order split-K reduce with the fused epilogue (warp-shuffle tree).
struct SplitReduce {
  const float* partial;  // [splits][M][N] dense
  int splits;
  int M, N;
  float* C;
  int64_t scm, scn;
  const float* bias;
  int bias_on_m;
  float alpha, beta;
  int relu;
  const float* scale_a;  // when set, alpha = 1/(*scale_a * *scale_b) (device scalars)
  const float* scale_b;
  EwProg ew;             // epilogue program (offsets from C)
  int out_bf16;          // C holds BF16 (RNE of the FP32 result) instead of FP32
};
nk_status splitk_reduce(const SplitReduce& r, cudaStream_t st);

// Converts a fused elementwise program (nk.h rules) whose tensor operands must
// have the rank, shape and strides of `like`; NULL gives the empty program.
// `what` names the program in error messages.
nk_status ew_program(const nk_ew_program* prog, const nk_tensor* like, EwProg* out, const char* what);

// ------------------------------------------------------------- prep / norm
// `pro` (optional): a prologue program run on each element (offsets from x /
// in) before the amax or the cast sees it.
nk_status prep_amax(const float* x, int64_t rows, int64_t cols, int64_t ld, float* amax,
                    void* ws, size_t ws_bytes, cudaStream_t st, const EwProg* pro = nullptr);
size_t prep_amax_ws(int64_t n);
// kind: 0 = bf16, 1 = fp8 (scale from *amax), 2 = bf16 hi/lo pair
nk_status prep_cast(int kind, const float* in, int64_t rows, int64_t cols, int64_t ld_in,
                    const float* amax, void* out0, void* out1, int64_t ld_out, int transpose,
                    float* scale_out, cudaStream_t st, const EwProg* pro = nullptr);
// Y = prog(X) over a rank-r strided tensor (nk_elementwise).
nk_status ew_tensor(const float* x, const int64_t* sx, float* y, const int64_t* sy, const int64_t* shape,
                    int rank, const EwProg& prog, cudaStream_t st);
nk_status norm_sumsq(const float* C, int64_t ldc, const double* R, int64_t ldr, int64_t M,
                     int64_t N, double* out, void* ws, size_t ws_bytes, cudaStream_t st);
size_t norm_ws(int64_t M, int64_t N);

}  // namespace nk

namespace nk {

// -------------------------------------------------- tensor-core GEMM (tcgen05)
// Operands are K-major in device memory: A [M,K] with row stride lda, B given
// as Bt [N,K] with row stride ldb (elements; 16-byte multiples).  C is FP32
// row-major with row stride ldc.  kind: 0 = BF16, 1 = FP8 E4M3, 2 = BF16x3
// (A2/B2 hold the lo halves).  alpha = 1/(sa*sb) when scale pointers are set.
enum TcKind { TC_BF16 = 0, TC_FP8 = 1, TC_BF16X3 = 2 };

struct TcGemm {
  int kind;
  int M, N, K;
  const void* A;
  const void* B;
  const void* A2;
  const void* B2;
  int64_t lda, ldb;
  float* C;
  int64_t ldc;
  const float* bias;
  int bias_on_m;
  int relu;
  float beta;
  float alpha;
  const float* scale_a;   // device scalars (FP8 computed on device) or null
  const float* scale_b;
  EwProg ew;              // epilogue program (offsets from C)
};

nk_status tc_gemm(const TcGemm& g, const nk_schedule& s, void* ws, size_t ws_bytes,
                  cudaStream_t st);

// Implicit-GEMM convolution on the tensor cores, BF16 or E4M3 operands
// (kind TC_BF16 / TC_FP8).  I: NHWC with channel stride 1 and element
// strides sI_n, sI_h, sI_w (16-byte multiples); Wt: filter f / tap t /
// channel c at f*sW_f + t*ldw + c (K-major per filter tap; ldw, sW_f 16-byte
// multiples); O: FP32 [N*OH*OW, F] row-major.  E4M3: scale_i, scale_w are
// the device scalars s_i, s_w the operands were quantised with (the epilogue
// multiplies by 1/(s_i*s_w)); null for BF16.  out_bf16: O holds BF16, the
// epilogue's FP32 result rounded to nearest even (same [N*OH*OW, F] layout).
struct TcConv {
  int kind;
  const void* I;
  int64_t sI_n, sI_h, sI_w;
  const void* Wt;
  int64_t ldw;
  int64_t sW_f;
  ConvGeom g;
  int F;
  float* O;
  const float* bias;
  int relu;
  float beta;
  const float* scale_i;
  const float* scale_w;
  EwProg ew;              // epilogue program (offsets from O)
  int out_bf16;
  float alpha;            // E4M3 operands the caller quantised: 1/(s_i*s_w) (scale_i, scale_w null)
};
// tc_conv dispatches a window schedule (see below) to tc_halo_conv.
nk_status tc_conv(const TcConv& c, const nk_schedule& s, void* ws, size_t ws_bytes, cudaStream_t st);
size_t tc_conv_ws(const TcConv& c, const nk_schedule& s);
nk_schedule tc_conv_default_schedule(const ConvGeom& g, int F, int sms, int kind = TC_BF16);
bool tc_conv_schedule_valid(const ConvGeom& g, int F, const nk_schedule& s, int kind = TC_BF16);

// Stride-1 convolution from one shared input window per tile (k_tc_halo.cu).
// A conv schedule with tile_k = 64 * KH * KW (one pipeline stage = one
// 64-channel block of the window, read by every tap) selects it; tile_m =
// 128 * chains (1, 2, 4), tile_n 64 / 128 / 256 with chains * tile_n <= 256,
// stages = window slots (1..4), cluster 1, split_k 1.
// E4M3 operands (kind TC_FP8): stacked kernel rows only, tile_k = 128 * KH.
bool halo_schedule(const ConvGeom& g, const nk_schedule& s, int kind = TC_BF16);
bool halo_schedule_valid(const ConvGeom& g, int F, const nk_schedule& s, int kind = TC_BF16);
nk_status tc_halo_conv(const TcConv& c, const nk_schedule& s, cudaStream_t st);
nk_schedule tc_halo_default_schedule(const ConvGeom& g, int F, int sms, bool* ok, int kind = TC_BF16);
// Window tile of a window schedule: P, Q, R, NB, WR, rows, slot_rows, stk,
// tiles, chains (false when the schedule is not a legal window schedule).
bool halo_tile_info(const ConvGeom& g, int F, const nk_schedule& s, int32_t out[10], int kind = TC_BF16);
uint32_t halo_read_and_clear_errors();
size_t tc_gemm_ws(const TcGemm& g, const nk_schedule& s);
// Fills unset fields of `s` with the built-in choice for this problem.
nk_schedule tc_default_schedule(int kind, int M, int N, int K, int sms);
// The built-in matmul schedule: tc_default_schedule refitted to the tuner's
// corpus for BF16 and E4M3 (tune.cu).
nk_schedule matmul_default_schedule(int kind, int M, int N, int K, int sms);
bool tc_schedule_valid(int kind, const nk_schedule& s, int M, int N, int K);

}  // namespace nk
