/*
 * nk.h -- C ABI of the GB300 dense-contraction library (libnk.so).
 *
 * The library computes the dense contractions that nelli (arXiv 2307.16080)
 * writes as MLIR linalg ops and lowers through tiled loop nests:
 *
 *   linalg.matmul           C[m,n] (+)= sum_k A[m,k] * B[k,n]
 *                           (Sec. 1 Listing "for->affine"; Sec. 2.1.1 Listing
 *                           "linalg-matmul": maps (d0,d2),(d2,d1)->(d0,d1),
 *                           iterators parallel, parallel, reduction)
 *   linalg.batch_matmul     the same with a leading batch / group index
 *   linalg.conv_2d_nhwc_hwcf
 *                           O[n,oh,ow,f] (+)= sum_{kh,kw,c}
 *                              I[n, oh*sh + kh*dh - ph, ow*sw + kw*dw - pw, c]
 *                              * W[kh,kw,c,f]
 *                           (Sec. 4.1 Listing "2dnchwconv", output-parallel,
 *                           no kernel flip; NHWC/HWCF with stride, dilation
 *                           and zero padding)
 *
 * followed by the epilogue of the lowered torch.nn.Linear (Sec. 2.1.2 Listing
 * "listing1": zero-fill, contraction, bias add), extended with ReLU and a
 * dequantisation scale:   out = ReLU?(beta*C_in + alpha*acc + bias[n]),
 * then an optional fused elementwise program (nk_ew_program); operands may
 * pass through such a program before the contraction (prologues).
 *
 * Conventions for every entry point
 *  - The caller owns every buffer and the stream.  The library never frees or
 *    allocates caller-visible device memory; compute calls allocate nothing.
 *  - Device pointers are plain CUDA device addresses on the current device;
 *    `stream` is a cudaStream_t (NULL = legacy default stream).  Compute calls
 *    are asynchronous on that stream; host arguments are read before return.
 *  - Arguments are validated before anything is launched.  A non-OK status
 *    means nothing was launched; nk_last_error() gives a message.
 *  - Strides are in elements.  Every matrix needs one unit-stride dimension
 *    (its "major" dimension); FP32 operands and outputs may have any other
 *    stride.  BF16 / E4M3 operands are read by TMA directly and so need a
 *    16-byte aligned base and 16-byte multiples for the other strides
 *    (NK_ERR_MISALIGNED otherwise).
 *  - There is no CPU fallback: without a usable GB300 (sm_103) the calls
 *    return NK_ERR_CUDA.
 */
#ifndef NK_H
#define NK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NK_OK = 0,
  NK_ERR_INVALID_ARG = -1, /* null pointer, bad rank/shape/dtype combination  */
  NK_ERR_UNSUPPORTED = -2, /* legal request this build does not implement     */
  NK_ERR_MISALIGNED = -3,  /* pointer or stride breaks the 16-byte rule       */
  NK_ERR_WORKSPACE = -4,   /* workspace missing or smaller than required      */
  NK_ERR_CUDA = -5,        /* CUDA runtime/driver error (message has details) */
  NK_ERR_TIMEOUT = -6,     /* a bounded device-side wait expired              */
  NK_ERR_NO_SCHEDULE = -7  /* no legal schedule for this problem              */
} nk_status;

typedef enum { NK_F32 = 0, NK_BF16 = 1, NK_F8E4M3 = 2, NK_F64 = 3 } nk_dtype;

/* Arithmetic of the contraction; the accumulator is FP32 in every case.
 *  F32    : FP32 inputs, FP32 FFMA (CUDA cores).
 *  BF16   : operands rounded to bfloat16 (RNE), tcgen05 MMA.
 *  BF16X3 : x = hi + lo with hi = bf16(x), lo = bf16(x - hi); the MMA sums
 *           hi*hi + hi*lo + lo*hi (lo*lo dropped) to recover FP32 accuracy.
 *  FP8    : per-tensor scales s = 448/amax(|x|), q = e4m3_rn_sat(x*s),
 *           tcgen05 MMA on E4M3, result multiplied by 1/(s_a*s_b).        */
typedef enum {
  NK_PREC_F32 = 0,
  NK_PREC_BF16 = 1,
  NK_PREC_BF16X3 = 2,
  NK_PREC_FP8 = 3
} nk_precision;

/* A strided view of device memory: element (i0,..,i{r-1}) lives at
 * ptr + sum_d i_d * stride[d] elements.  rank <= 4; unused entries ignored. */
typedef struct {
  void* ptr;
  int32_t dtype; /* nk_dtype */
  int32_t rank;
  int64_t shape[4];
  int64_t stride[4];
} nk_tensor;

/* ------------------------------------------- fused elementwise programs */

/* A program of up to NK_EW_MAX elementwise operations, applied in order to
 * each element x of a tensor inside the kernel that produces or reads it.
 * These are the linalg.generic consumers and producers around a contraction
 * that a lowering otherwise leaves as separate loop nests -- the bias-add
 * loop after the matmul of the lowered torch.nn.Linear (Sec. 2.1.2 Listing
 * "listing1") and the elementwise product C[x,y] = A[x,y] * B[x,y] of the
 * GPUModule kernel (Sec. 3.1 Listing "gpumodules") -- folded into the
 * epilogue (or, for operands, into the conversion pass or the loads).
 * Every step computes in FP32 and rounds to FP32.
 *
 *   NK_EW_MUL        x = x * t[i]            (t: tensor operand, see below)
 *   NK_EW_ADD        x = x + t[i]
 *   NK_EW_AFFINE     x = fma(a, x, b)        (one rounding)
 *   NK_EW_RELU       x = max(x, 0)           (NaN stays NaN)
 *   NK_EW_GELU       x = x * Phi(x) = 0.5 x (1 + erf(x / sqrt 2))
 *   NK_EW_GELU_TANH  x = 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))
 *   NK_EW_SILU       x = x * sigmoid(x)
 *   NK_EW_SIGMOID    x = 1 / (1 + exp(-x))
 *   NK_EW_TANH       x = tanh(x)
 *   NK_EW_CLAMP      x = x < a ? a : (x > b ? b : x)   (a <= b; NaN stays NaN)
 *
 * A tensor operand `t` (MUL, ADD) is FP32 with the shape and the strides of
 * the tensor the program runs over (the output C / O for an epilogue, the
 * operand A, B, I or W for a prologue), so element (i0, i1, ..) of `t` pairs
 * with the same element of that tensor.  It may alias that tensor's output
 * only for an epilogue (each element is read before its own result is
 * written).  Checked before launch: 0 <= n <= NK_EW_MAX, known opcodes,
 * finite a <= b for CLAMP, and for MUL / ADD a non-NULL 4-byte aligned FP32
 * t of matching rank, shape and strides (NK_ERR_INVALID_ARG otherwise).   */
#define NK_EW_MAX 4
typedef enum {
  NK_EW_MUL = 1,
  NK_EW_ADD = 2,
  NK_EW_AFFINE = 3,
  NK_EW_RELU = 4,
  NK_EW_GELU = 5,
  NK_EW_GELU_TANH = 6,
  NK_EW_SILU = 7,
  NK_EW_SIGMOID = 8,
  NK_EW_TANH = 9,
  NK_EW_CLAMP = 10
} nk_ew_opcode;

typedef struct {
  int32_t op;   /* nk_ew_opcode */
  float a, b;   /* AFFINE: a*x + b; CLAMP: [a, b]; ignored otherwise */
  nk_tensor t;  /* MUL / ADD operand; ignored otherwise */
} nk_ew_op;

typedef struct {
  int32_t n;    /* number of operations, 0..NK_EW_MAX */
  nk_ew_op ops[NK_EW_MAX];
} nk_ew_program;

/* out = ew(ReLU?(beta*C_in + alpha*acc + bias[n])) with beta = accumulate ?
 * 1 : 0.
 * bias: FP32 device vector of length N (GEMM) / F (conv), or NULL.
 * scale_a, scale_b: only read for FP8 inputs that are already quantised
 * (dtype NK_F8E4M3): the quantisation scales s_a, s_b; alpha = 1/(s_a*s_b).
 * For FP32 inputs at NK_PREC_FP8 the library computes the scales itself.
 * ew: elementwise program run on every output element last, or NULL.
 * pro_a, pro_b: programs run on every element of the FP32 operand A and B
 * (conv: I and W) before the contraction, or NULL.  The transformed value is
 * what the precision rounds (BF16, BF16x3) or quantises (FP8: the amax and
 * the scale are taken over the transformed values); for the convolution the
 * zero padding stays zero.  An operand that is given already converted
 * (BF16 / E4M3 dtype, packed conv weights) takes no prologue
 * (NK_ERR_UNSUPPORTED).  A zero-initialised struct is the plain epilogue.  */
typedef struct {
  const float* bias;
  int32_t relu;
  int32_t accumulate;
  float scale_a;
  float scale_b;
  const nk_ew_program* ew;
  const nk_ew_program* pro_a;
  const nk_ew_program* pro_b;
} nk_epilogue;

/* Y = prog(X) elementwise: the GPUModule kernel of Sec. 3.1 (with prog = one
 * NK_EW_MUL by B it is C[x,y] = A[x,y] * B[x,y]) as a standalone pass.  X, Y:
 * FP32 tensors of the same rank (1..4) and shape; Y may be X (in place).
 * Tensor operands of `prog` have Y's shape and strides.  HBM-bound: one read
 * of X and of each operand, one write of Y.  Allocates nothing.            */
nk_status nk_elementwise(const nk_tensor* X, nk_tensor* Y, const nk_ew_program* prog,
                         void* stream);

/* Tile schedule.  tile_m x tile_n output tile per CTA; cluster 2 (only with
 * tile_m 256) makes two CTAs on two SMs a pair that computes one 256-row
 * tile with 2-SM MMAs, each CTA loading its own 128 rows of A and half of B
 * (no TMA load is multicast); tile_m 256 / 512 with cluster 1 is one CTA
 * holding 2 / 4 stacked 128-row tiles.  tile_k reduction depth per pipeline
 * stage, stages = shared-memory ring depth, split_k =
 * number of K slices reduced by a separate fixed-order pass.  Any field 0
 * means "choose".  For the shared-window convolution (tile_k = 64*KH*KW,
 * or 64*KH with the KW taps of a kernel row side by side along N; see
 * nk_conv2d_nhwc_hwcf) stages counts window slots and split_k is 1; with
 * stacked kernel rows tile_m 128 keeps one accumulator buffer (two CTAs per
 * SM, 1-4 slots) and tile_m 256 two (one CTA per SM, 2-8 slots), so the
 * epilogue of a tile overlaps the MMAs of the next.                       */
typedef struct {
  int32_t tile_m, tile_n, tile_k, cluster, stages, split_k;
} nk_schedule;

/* ---------------------------------------------------------------- matmul */

/* linalg.matmul: C = epilogue(A @ B).
 * A: [M,K], B: [K,N], C: [M,N] FP32 (C is also C_in when accumulate = 1).
 * dtype of A and B: F32 for any precision (BF16/BF16X3/FP8 convert them into
 * the workspace first), BF16 with NK_PREC_BF16, F8E4M3 with NK_PREC_FP8
 * (scales from `epi`).  Either dimension of A and B may be the unit-stride
 * one; (A B)^T = B^T A^T is used when C is column-major.
 * sched: NULL = built-in choice.  ws/ws_bytes: device scratch of at least
 * nk_matmul_workspace_size() bytes (may be NULL/0 when that size is 0).   */
nk_status nk_matmul(const nk_tensor* A, const nk_tensor* B, nk_tensor* C,
                    int32_t precision, const nk_epilogue* epi,
                    const nk_schedule* sched, void* ws, size_t ws_bytes,
                    void* stream);

/* Bytes of workspace nk_matmul needs for these operands and schedule.     */
nk_status nk_matmul_workspace_size(const nk_tensor* A, const nk_tensor* B,
                                   const nk_tensor* C, int32_t precision,
                                   const nk_schedule* sched, size_t* bytes);

/* ---------------------------------------------------------- grouped GEMM */

/* One independent GEMM of a group: C_g = A_g @ B_g (+ C_g if accumulate).
 * A_g: [M,K] row-major with leading dimension lda (elements), B_g: [K,N]
 * given as its transpose Bt [N,K] row-major with ldb, C_g: [M,N] FP32
 * row-major with ldc.  M, N, K >= 1; K a multiple of 8 and lda, ldb
 * multiples of 8 for BF16 (16-byte rows).                                  */
typedef struct {
  int32_t M, N, K;
  int32_t accumulate;
  const void* A;
  const void* Bt;
  float* C;
  int64_t lda, ldb, ldc;
} nk_gemm_group;

/* Opaque plan: group table, per-group TMA descriptors (A, B^T and, when
 * every group overwrites a 16-byte aligned C whose row stride and row
 * length N are multiples of 4 floats, C for TMA stores), tile table and the
 * group of every tile (4 bytes per
 * tile) in device memory, built once on the host side and replayed by one
 * persistent launch.  Creating a plan allocates; running it does not
 * (graph-safe).                                                           */
typedef struct nk_grouped_plan nk_grouped_plan;

/* Build a plan for G groups (host array `groups`, copied) at `precision`
 * NK_PREC_BF16 (BF16 operands; other precisions return NK_ERR_UNSUPPORTED).
 * sched (NULL = 128 x 128 tiles, deepest ring): tile_m 128 with cluster 1,
 * or tile_m 256 with cluster 2 (a CTA pair computes 256 x tile_n tiles with
 * cta_group::2 MMAs, each CTA loading half of B); tile_n 64 / 128 / 256;
 * split_k 1.  nk_grouped_tune (nk_tune.h) picks one by timing.            */
nk_status nk_grouped_plan_create(int32_t G, const nk_gemm_group* groups,
                                 int32_t precision, const nk_schedule* sched,
                                 nk_grouped_plan** plan);
nk_status nk_grouped_plan_run(const nk_grouped_plan* plan, void* stream);
nk_status nk_grouped_plan_destroy(nk_grouped_plan* plan);

/* linalg.batch_matmul generalised to uneven groups, as one call: builds the
 * plan in the caller's workspace (no allocation) and launches it.
 * ws must hold nk_grouped_workspace_size() bytes; the workspace must stay
 * untouched until the launch has completed.                               */
nk_status nk_batch_matmul_grouped(int32_t G, const nk_gemm_group* groups,
                                  int32_t precision, const nk_schedule* sched,
                                  void* ws, size_t ws_bytes, void* stream);
nk_status nk_grouped_workspace_size(int32_t G, const nk_gemm_group* groups,
                                    int32_t precision, const nk_schedule* sched,
                                    size_t* bytes);

/* ------------------------------------------------------------------ conv */

/* linalg.conv_2d_nhwc_hwcf with zero padding and the epilogue.
 * I: [N,H,W,C], W: [KH,KW,C,F], O: [N,OH,OW,F]; I and O with unit
 * stride in the last dimension.  O is FP32, or -- at NK_PREC_BF16 and
 * NK_PREC_FP8 -- BF16: the epilogue (bias, ReLU, accumulate, program)
 * computes in FP32 and each result is rounded to BF16 (RNE) as it is
 * stored, so the output can feed the next layer as its BF16 input (with
 * accumulate = 1 the BF16 O is read as C_in).  OH = (H + pt + pb - dh*(KH-1) - 1)/sh + 1
 * (same for OW).  stride = {sh, sw}, dilation = {dh, dw},
 * pad = {top, bottom, left, right}.
 * Precisions: NK_PREC_F32 (CUDA cores), NK_PREC_BF16, NK_PREC_FP8 (E4M3
 * with per-tensor scales s = 448/amax(|x|) of I and of W, computed on the
 * device and undone by 1/(s_i*s_w) in the epilogue; I and W FP32 -- or both
 * already E4M3: I NHWC with 16-byte multiples as strides and W packed by
 * nk_conv2d_pack_weights_fp8, with their scales s_i, s_w as epi->scale_a,
 * epi->scale_b, so that a call runs no amax and no quantisation).
 * I dtype: F32 (any precision; BF16 / E4M3 convert it into the workspace)
 * or BF16 with NK_PREC_BF16.  W dtype: F32 contiguous HWCF (converted per
 * call into the workspace), or -- NK_PREC_BF16 only -- BF16 already
 * packed by nk_conv2d_pack_weights, described as [KH,KW,C,F] with strides
 * {KW*ldw, ldw, 1, sF} (ldw >= C, sF >= KH*KW*ldw, multiples of 8; 16-byte
 * aligned base): no per-call conversion.
 * At NK_PREC_BF16 a stride-1 schedule with tile_k = 64*KH*KW selects the
 * shared-window kernel (each tile's input window is loaded once and read by
 * every tap), tile_k = 64*KH the same window with the KW taps of a kernel
 * row side by side along N; tile_k = 64 selects the per-tap implicit GEMM.
 * At NK_PREC_FP8 the K blocks hold 128 channels: tile_k = 128*KH selects
 * the stacked window kernel on E4M3 operands, tile_k = 128 the per-tap one. */
nk_status nk_conv2d_nhwc_hwcf(const nk_tensor* I, const nk_tensor* W,
                              nk_tensor* O, const int64_t stride[2],
                              const int64_t dilation[2], const int64_t pad[4],
                              int32_t precision, const nk_epilogue* epi,
                              const nk_schedule* sched, void* ws,
                              size_t ws_bytes, void* stream);
nk_status nk_conv2d_workspace_size(const nk_tensor* I, const nk_tensor* W,
                                   const nk_tensor* O, const int64_t stride[2],
                                   const int64_t dilation[2],
                                   const int64_t pad[4], int32_t precision,
                                   const nk_schedule* sched, size_t* bytes);

/* ---------------------------------------------------- grouped convolution */

/* One convolution of a grouped launch: linalg.conv_2d_nhwc_hwcf (Sec. 4.1,
 * in NHWC/HWCF) with its epilogue ReLU?(beta*O + acc + bias[f]).
 * I: BF16 NHWC [N,H,W,C], unit channel stride, 16-byte aligned base and
 * rows; W: BF16 packed by nk_conv2d_pack_weights (a [KH,KW,C,F] view with
 * strides {KW*ldw, ldw, 1, sF}); O: FP32 contiguous NHWC [N,OH,OW,F].
 * stride / dilation / pad as for nk_conv2d_nhwc_hwcf (stride <= 8).       */
typedef struct {
  nk_tensor I, W, O;
  int64_t stride[2], dilation[2], pad[4];
  const float* bias; /* FP32 [F] device vector or NULL */
  int32_t relu;
  int32_t accumulate;
} nk_conv_group;

/* Plan of G independent convolutions of uneven shapes computed by one
 * persistent launch (run with nk_grouped_plan_run, CUDA-graph replayable;
 * free with nk_grouped_plan_destroy).  Every group's tiles (its own output
 * tiling, input and weight tensor maps, bias, ReLU) share one grid; groups
 * are ordered by decreasing K so the longest tiles start first.
 * sched (NULL = 128 x 128 tiles, deepest ring): tile_m 128, tile_k 64,
 * cluster 1, split_k 1, tile_n 64 / 128 / 256.  Allocates the plan's
 * device table.                                                            */
nk_status nk_conv2d_grouped_plan_create(int32_t G, const nk_conv_group* groups,
                                        const nk_schedule* sched,
                                        nk_grouped_plan** plan);

/* Converts FP32 HWCF weights W [KH,KW,C,F] (contiguous) to the BF16 layout
 * the tensor-core convolution reads: element (kh,kw,c,f) at
 * Wp + f*(KH*KW*ldw) + (kh*KW + kw)*ldw + c, with ldw >= C a multiple of 8
 * (channels c >= C of a row are never read).  Wp: device memory of
 * F*KH*KW*ldw*2 bytes, 16-byte aligned, owned by the caller.  Asynchronous
 * on `stream`; pass the result to nk_conv2d_nhwc_hwcf as a BF16 W with
 * strides {KW*ldw, ldw, 1, KH*KW*ldw} so repeated calls skip the cast.   */
nk_status nk_conv2d_pack_weights(const nk_tensor* W, void* Wp, int64_t ldw,
                                 void* stream);

/* E4M3 weights for NK_PREC_FP8 convolutions, quantised once: the
 * per-tensor scale s_w = 448/amax(|W|) (s_w = 1 when amax is 0) is computed
 * on the device and written to *scale (device float), and each weight is
 * stored as e4m3_rn_sat(W * s_w) in the packed layout of
 * nk_conv2d_pack_weights: (kh,kw,c,f) at Wp + f*(KH*KW*ldw) + (kh*KW+kw)*ldw
 * + c, ldw >= C a multiple of 16.  W: FP32 HWCF [KH,KW,C,F], contiguous.
 * Wp: F*KH*KW*ldw bytes of device memory, 16-byte aligned.  ws/ws_bytes:
 * device scratch of nk_conv2d_pack_weights_fp8_workspace_size() bytes.
 * Asynchronous on `stream`.  Pass the result as an E4M3 W with strides
 * {KW*ldw, ldw, 1, KH*KW*ldw} and s_w as epi->scale_b, together with an
 * E4M3 I (quantised by the caller, e.g. with nk_amax and nk_cast_fp8 on the
 * [N*H*W, C] view; s_i as epi->scale_a): the convolution then runs with no
 * per-call quantisation and multiplies its result by 1/(s_i s_w).          */
nk_status nk_conv2d_pack_weights_fp8(const nk_tensor* W, void* Wp, int64_t ldw,
                                     float* scale, void* ws, size_t ws_bytes,
                                     void* stream);
size_t nk_conv2d_pack_weights_fp8_workspace_size(void);

/* The convolution exactly as Sec. 4.1 Listing "2dnchwconv" lays it out:
 * I: [N,CI,H,W] (NCHW), K: [CO,CI,KH,KW] (FCHW, contiguous), O: [N,CO,OH,OW],
 * all FP32 with unit stride along W;
 *   O[n,co,ho,wo] = ReLU?(beta*O + bias[co] + sum_{ci,ki,kj}
 *        I[n,ci,ho*sh+ki*dh-pt, wo*sw+kj*dw-pl] * K[co,ci,ki,kj])
 * (zero padding).  A direct, output-parallel kernel for few channels (the
 * tuning experiment of Sec. 4.3 uses CI=1, CO=3, 3x3 on 1280x1280), bound by
 * HBM rather than by the tensor cores.  Limits: at most 64 filter taps and a
 * halo tile of 64 x 176 input elements per 16 x 64 output tile
 * (NK_ERR_UNSUPPORTED beyond).  Allocates nothing.                          */
nk_status nk_conv2d_nchw_fchw(const nk_tensor* I, const nk_tensor* K,
                              nk_tensor* O, const int64_t stride[2],
                              const int64_t dilation[2], const int64_t pad[4],
                              const nk_epilogue* epi, void* stream);

/* --------------------------------------------------------- operand prep */

/* amax = max |x| over n FP32 values, written as one float to `amax` (device).
 * Needs nk_prep_workspace_size(n) bytes of scratch.                         */
nk_status nk_amax(const float* x, int64_t n, float* amax, void* ws,
                  size_t ws_bytes, void* stream);
size_t nk_prep_workspace_size(int64_t n);

/* Cast a [rows, cols] FP32 matrix (row stride ld_in) to BF16 (RNE), FP8 E4M3
 * (q = e4m3_rn_sat(x * s) with s = 448/(*amax), s = 1 if amax = 0; the scale
 * is also stored to *scale_out when non-NULL) or the BF16 hi/lo pair.
 * transpose = 1 writes out[c, r] (row stride ld_out) so a [K,N] operand
 * becomes the K-major [N,K] layout the tensor cores read.                  */
nk_status nk_cast_bf16(const float* in, int64_t rows, int64_t cols, int64_t ld_in,
                       void* out, int64_t ld_out, int32_t transpose, void* stream);
nk_status nk_cast_fp8(const float* in, int64_t rows, int64_t cols, int64_t ld_in,
                      const float* amax, void* out, int64_t ld_out,
                      int32_t transpose, float* scale_out, void* stream);
nk_status nk_split_bf16x3(const float* in, int64_t rows, int64_t cols,
                          int64_t ld_in, void* hi, void* lo, int64_t ld_out,
                          int32_t transpose, void* stream);

/* ------------------------------------------------------------ validation */

/* sumsq[0] = sum (C - R)^2, sumsq[1] = sum R^2 over an [M,N] FP32 matrix C
 * (row stride ldc) and FP64 reference R (row stride ldr), accumulated in FP64
 * on the device in a fixed order (run-to-run identical).  The relative
 * Frobenius error is sqrt(sumsq[0] / sumsq[1]).  sumsq: 2 doubles (device).
 * Needs nk_norm_workspace_size(M, N) bytes.                                  */
nk_status nk_rel_frobenius(const float* C, int64_t ldc, const double* R,
                           int64_t ldr, int64_t M, int64_t N, double* sumsq,
                           void* ws, size_t ws_bytes, void* stream);
size_t nk_norm_workspace_size(int64_t M, int64_t N);

/* ------------------------------------------------ split-K, no allocation */

/* C = A @ B in FP32 on the CUDA cores with split-K, for callers that cannot
 * allocate device memory (code running inside an allocator callback, under a
 * runtime that owns the whole memory pool, or with no device memory budget
 * left): the split_k partial sums live in a fixed 16 MiB array inside the
 * library instead of a caller workspace.  The paper has no counterpart; this
 * is a deployment convenience around the split-K path of nk_matmul.
 * A: [M,K] row-major (row stride lda), B: [K,N] row-major (ldb), C: [M,N]
 * row-major FP32 (ldc), all device pointers; split_k in [1, 32].
 * Limit: split_k * M * N <= 4194304 floats, else NK_ERR_WORKSPACE (nothing is
 * launched).  Allocates nothing: no cudaMalloc, no cudaFree.
 * The array is shared by every call on a device and keeps the last call's
 * partials; each call overwrites all it reads, so no clearing is needed, but
 * calls whose kernels overlap on the same GPU (for example on two streams)
 * race on it -- serialise them.
 * The first call on each device looks up the array's device address with
 * that device current; make that first call before any stream capture.   */
nk_status nk_matmul_f32_splitk_noalloc(const float* A, int64_t lda,
                                       const float* B, int64_t ldb, float* C,
                                       int64_t ldc, int32_t M, int32_t N,
                                       int32_t K, int32_t split_k, void* stream);

/* ---------------------------------------------------------- diagnostics */

/* Thread-local message describing the last non-OK status of this thread.  */
const char* nk_last_error(void);

/* Synchronise `stream`, then report device-side failures: NK_ERR_TIMEOUT if
 * a bounded wait inside a kernel expired since the last call (the flag is
 * cleared), NK_ERR_CUDA for a runtime error.                                */
nk_status nk_sync_status(void* stream);

/* Test hook: the spin budget (iterations) of every bounded device wait;
 * 0 restores the default.  Lets a test drive the timeout path on purpose. */
nk_status nk_set_wait_budget(int64_t iterations);

/* Programmatic dependent launch (on by default).  When on, every compute
 * kernel of this library (not the tuner's own timing kernels) is launched
 * so that it may start while the kernel before it on the same stream is
 * finishing: it prepares its shared memory, mbarriers
 * and tensor memory, then waits, on the device, until all earlier work on
 * the stream has completed and is visible before it reads or writes any
 * global memory.  Results are identical either way; only the gap between
 * back-to-back kernels (a stream, or a CUDA graph captured from one)
 * changes.  The setting is process-wide and is read at each launch, so a
 * graph keeps the setting it was captured with.  The paper has no
 * counterpart: it is a launch-latency measure of this GPU.                  */
nk_status nk_set_pdl(int32_t enabled);
int32_t nk_get_pdl(void);

/* Number of SMs and the compute capability of the current device.          */
nk_status nk_device_info(int32_t* sm_count, int32_t* cc_major, int32_t* cc_minor);

#ifdef __cplusplus
}
#endif

#endif /* NK_H */
