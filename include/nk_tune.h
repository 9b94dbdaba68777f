/*
 * nk_tune.h -- schedule search and the learned tile-cost model of libnk.
 *
 * The paper tunes its tiled loop nest by black-box search over tile sizes and
 * unroll factors (Sec. 4.3, Figure "nevergrad": the tiling pass and an unroll
 * op, parameterised, timed on the device, fed back to the optimiser).  Here
 * the search space is the tensor-core schedule (tile_n, cluster, stages,
 * split_k); candidates are timed on the GPU with CUDA events, and a small MLP
 * (16 -> 128 -> 128 -> 1, GELU) trained on those timings ranks the candidates
 * so only the top few need timing.
 */
#ifndef NK_TUNE_H
#define NK_TUNE_H

#include "nk.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { NK_OP_MATMUL = 0, NK_OP_CONV2D = 1 } nk_op;
/* EXHAUSTIVE: time every legal schedule.  MODEL_TOPK: rank all with the cost
 * model, time the top `topk`.  EVOLUTION: a derivative-free (1+1) evolution
 * strategy over the schedule grid -- the black-box search of Sec. 4.3 --
 * started from the built-in default, `topk` timings in all (mlp_params are
 * not used).                                                               */
typedef enum { NK_TUNE_EXHAUSTIVE = 0, NK_TUNE_MODEL_TOPK = 1, NK_TUNE_EVOLUTION = 2 } nk_tune_mode;

/* A tensor-core problem: matmul (M, N, K) or conv (n, h, w, c -> f with a
 * kh x kw filter, equal stride and padding on both axes, dilation 1).
 * precision: NK_PREC_BF16 / NK_PREC_FP8 / NK_PREC_BF16X3 (matmul),
 * NK_PREC_BF16 / NK_PREC_FP8 (conv).                                       */
typedef struct {
  int32_t op;
  int32_t precision;
  int32_t M, N, K;
  int32_t n, h, w, c, f, kh, kw, stride, pad;
} nk_problem;

typedef struct {
  int32_t candidates; /* legal schedules enumerated                        */
  int32_t timed;      /* schedules timed on the GPU                        */
  float best_ms;      /* median time of the returned schedule              */
  float default_ms;   /* median time of the built-in default schedule      */
} nk_tune_report;

/* Number of model features per (problem, schedule) pair.                   */
#define NK_TUNE_FEATURES 16

/* Legal schedules of a problem in a fixed order (the tie-break order of the
 * search).  Writes at most `cap` to `out` (host) and the total to *count.  */
nk_status nk_enumerate_schedules(const nk_problem* p, nk_schedule* out, int32_t cap,
                                 int32_t* count);

/* The built-in schedule (used when nk_matmul / nk_conv2d get sched = NULL). */
nk_status nk_default_schedule(const nk_problem* p, nk_schedule* out);

/* Workspace bytes the call for this problem needs at its precision and
 * schedule (NULL = built-in choice), with FP32 operands as the plain case
 * takes them: nk_matmul with A [M,K], B [K,N], C [M,N] row-major, or
 * nk_conv2d_nhwc_hwcf with contiguous NHWC I, HWCF W and NHWC O (pad on
 * all four sides, dilation 1).  The same number the operand-based
 * nk_matmul_workspace_size / nk_conv2d_workspace_size return.             */
nk_status nk_workspace_size(const nk_problem* p, const nk_schedule* sched, size_t* bytes);

/* Diagnostics, host only (no GPU): the tile a window schedule (tile_k =
 * 64*KH*KW, or 64*KH with stacked kernel rows) launches for a stride-1 NHWC
 * convolution of N x H x W x C -> F with a KH x KW filter, dilations dh, dw
 * and pad {top, bottom, left, right}.  out[10] (host) receives: the window
 * row pitch P (pixels), the output columns Q, rows R and images NB of a
 * tile, the window rows per image WR, the pixels one window box loads, the
 * rows reserved per window slot, the taps side by side along N (KW when
 * stacked, else 1), the number of tiles, and the accumulator chains.  Lets
 * a test check, without a GPU, that every row a valid output reads stays in
 * its tile, its warp, the window box and the slot.  NK_ERR_NO_SCHEDULE when
 * `s` is not a legal window schedule there.  The paper has no counterpart. */
nk_status nk_conv_window_tile(int32_t n, int32_t h, int32_t w, int32_t c, int32_t f, int32_t kh, int32_t kw,
                              int32_t dh, int32_t dw, const int32_t pad[4], const nk_schedule* s,
                              int32_t out[10]);

/* Model features of `count` schedules for one problem, host array
 * [count][NK_TUNE_FEATURES]: log2 M, N, K; is_conv; taps; stride; precision
 * one-hot (BF16, FP8, BF16x3); log2 tile_m, tile_n, tile_k; cluster; stages;
 * log2 split_k; log2(work units / SMs) -- each scaled to about [0, 1].     */
nk_status nk_schedule_features(const nk_problem* p, const nk_schedule* s, int32_t count,
                               float* features);

/* Median device time, in milliseconds, of one run of a schedule on synthetic
 * operands of the problem's shape.  After warm-up runs, `inner` back-to-back
 * runs (so that one sample lasts about 400 us: the GPU event clock ticks in
 * steps of about 2 us) are captured into a CUDA graph; `reps` replays, each
 * between two CUDA events on a library-owned stream and all queued behind a
 * short hold kernel so that host-side call overhead is not timed, give
 * `reps` samples of time / inner.  Synchronises `stream` first; allocates
 * and keeps library-owned scratch operands (grown on demand, released by
 * nk_tune_release).                                                        */
nk_status nk_time_schedule(const nk_problem* p, const nk_schedule* s, int32_t reps,
                           float* median_ms, void* stream);
nk_status nk_tune_release(void);

/* Pick a schedule.  EXHAUSTIVE times every legal candidate; MODEL_TOPK runs
 * the cost model (`mlp_params`: device FP32 parameters, see nk_mlp_*) over
 * all candidates on the GPU and times only the `topk` best-predicted ones.
 * Ties in median time go to the earlier candidate.  `rep` may be NULL.      */
nk_status nk_tune(const nk_problem* p, int32_t mode, int32_t topk, const float* mlp_params,
                  int32_t reps, nk_schedule* best, nk_tune_report* rep, void* stream);

/* Grouped GEMM: the tile of a grouped plan (nk_grouped_plan_create) for this
 * set of groups.  Times every legal grouped schedule (tile_m 128 on one CTA
 * or 256 on a CTA pair with cluster 2; tile_n 64 / 128 / 256; split_k 1;
 * stages 2..8 within shared memory) as a
 * persistent launch on the caller's operands and returns the fastest in
 * *best (ties to the earlier candidate).  While timing, every group's C is
 * overwritten (accumulate flags are ignored); its contents afterwards are
 * unspecified.  Synchronises `stream`; allocates plan tables while it runs.
 * `rep` may be NULL (default_ms: the schedule nk_grouped_plan_create picks
 * for sched = NULL).                                                       */
nk_status nk_grouped_tune(int32_t G, const nk_gemm_group* groups, int32_t precision, int32_t reps,
                          nk_schedule* best, nk_tune_report* rep, void* stream);

/* Grouped convolutions (nk_conv2d_grouped_plan_create): times every legal
 * grouped conv schedule (tile_m 128, tile_k 64, cluster 1, split_k 1;
 * tile_n 64 / 128 / 256; stages 2..8) on the caller's groups and returns the
 * fastest; every group's O is overwritten while timing (accumulate flags
 * are ignored).  Same conventions as nk_grouped_tune.                      */
nk_status nk_conv2d_grouped_tune(int32_t G, const nk_conv_group* groups, int32_t reps,
                                 nk_schedule* best, nk_tune_report* rep, void* stream);

/* ------------------------------------------------------- the cost model */
/* Parameters: one FP32 device buffer of nk_mlp_param_count() values laid out
 * W1 [128][16], b1 [128], W2 [128][128], b2 [128], W3 [128], b3 [1].
 * y = W3 g(W2 g(W1 x + b1) + b2) + b3, g(z) = z Phi(z) (exact GELU).       */
size_t nk_mlp_param_count(void);

/* y[i] for the B rows of X [B][16] (device).                                 */
nk_status nk_mlp_forward(const float* params, const float* X, int64_t B, float* y,
                         void* stream);

/* Gradient of L = mean_i (y_i - t_i)^2 with respect to every parameter into
 * grad (device, nk_mlp_param_count() floats) and L into *loss (device, may be
 * NULL).  Per-block partial sums are added in a fixed order, so the result is
 * identical run to run.  Needs nk_mlp_workspace_size(B) bytes.             */
size_t nk_mlp_workspace_size(int64_t B);
nk_status nk_mlp_grad(const float* params, const float* X, const float* t, int64_t B,
                      float* grad, float* loss, void* ws, size_t ws_bytes, void* stream);

/* One Adam step (Kingma & Ba 2015, Algorithm 1) at step t >= 1 on all
 * parameters: m, v are device moment buffers of the same length.            */
nk_status nk_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t t,
                      float lr, float beta1, float beta2, float eps, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NK_TUNE_H */
