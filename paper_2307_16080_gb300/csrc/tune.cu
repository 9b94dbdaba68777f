// tune.cu -- schedule search for the tensor-core kernels.
//
// The paper searches tile sizes and unroll factors of its loop nest with a
// black-box optimiser that compiles, runs and times each point (Sec. 4.3).
// Here the points are tensor-core schedules (tile_n, cluster, stages,
// split_k): they are enumerated in a fixed order, timed on the GPU with
// CUDA events on synthetic operands of the problem's shape, and -- in model
// mode -- first ranked by the learned cost model (k_mlp.cu) so only the top
// few are timed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/nk_tune.h"
#include "nk_internal.cuh"

namespace nk {
namespace {

std::mutex g_mu;
void* g_scratch = nullptr;
size_t g_scratch_bytes = 0;
size_t g_filled = 0;

// Deterministic operand bits: BF16 values in [-1, 1); E4M3 codes without NaN.
__global__ void fill_kernel(uint16_t* p, size_t n16) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)(i * 2654435761u) ^ (uint32_t)(i >> 29);
    h ^= h >> 15;
    h *= 0x2c1b3c6du;
    h ^= h >> 12;
    const float f = (float)(h & 0xFFFF) / 32768.f - 1.f;
    __nv_bfloat16 b = __float2bfloat16_rn(f);
    p[i] = *reinterpret_cast<uint16_t*>(&b) & 0xF7F7u;  // as E4M3 pairs: exponent <= 14, no NaN
  }
}

nk_status scratch(size_t bytes, void** out) {
  if (bytes > g_scratch_bytes) {
    if (g_scratch) cudaFree(g_scratch);
    g_scratch = nullptr;
    g_scratch_bytes = 0;
    g_filled = 0;
    cudaError_t e = cudaMalloc(&g_scratch, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(tune scratch)");
    g_scratch_bytes = bytes;
  }
  *out = g_scratch;
  return NK_OK;
}

nk_status fill(size_t bytes) {
  if (bytes <= g_filled) return NK_OK;
  fill_kernel<<<1024, 256>>>(static_cast<uint16_t*>(g_scratch), bytes / 2);
  nk_status s = check_launch("fill_kernel");
  if (s == NK_OK) g_filled = bytes;
  return s;
}

int kind_of(int prec) {
  return prec == NK_PREC_FP8 ? TC_FP8 : prec == NK_PREC_BF16X3 ? TC_BF16X3 : TC_BF16;
}

nk_status check_problem(const nk_problem* p) {
  if (!p) return fail(NK_ERR_INVALID_ARG, "problem is NULL");
  if (p->op == NK_OP_MATMUL) {
    if (p->M < 1 || p->N < 1 || p->K < 1) return fail(NK_ERR_INVALID_ARG, "matmul extents must be positive");
    if (p->precision != NK_PREC_BF16 && p->precision != NK_PREC_FP8 && p->precision != NK_PREC_BF16X3)
      return fail(NK_ERR_UNSUPPORTED, "tuning covers the tensor-core precisions");
    return NK_OK;
  }
  if (p->op == NK_OP_CONV2D) {
    if (p->n < 1 || p->h < 1 || p->w < 1 || p->c < 1 || p->f < 1 || p->kh < 1 || p->kw < 1 || p->stride < 1 ||
        p->pad < 0)
      return fail(NK_ERR_INVALID_ARG, "conv extents must be positive");
    if (p->precision != NK_PREC_BF16 && p->precision != NK_PREC_FP8)
      return fail(NK_ERR_UNSUPPORTED, "conv tuning covers BF16 and FP8");
    if ((p->h + 2 * p->pad - p->kh) / p->stride + 1 < 1 || (p->w + 2 * p->pad - p->kw) / p->stride + 1 < 1)
      return fail(NK_ERR_INVALID_ARG, "empty conv output");
    return NK_OK;
  }
  return fail(NK_ERR_INVALID_ARG, "unknown op %d", p->op);
}

ConvGeom geom_of(const nk_problem* p) {
  ConvGeom g{};
  g.n = p->n; g.h = p->h; g.w = p->w; g.c = p->c;
  g.kh = p->kh; g.kw = p->kw;
  g.sh = g.sw = p->stride;
  g.dh = g.dw = 1;
  g.pt = g.pl = p->pad;
  g.oh = (p->h + 2 * p->pad - p->kh) / p->stride + 1;
  g.ow = (p->w + 2 * p->pad - p->kw) / p->stride + 1;
  const int cp = (p->c + 7) / 8 * 8;
  g.sin_w = cp; g.sin_h = (int64_t)p->w * cp; g.sin_n = (int64_t)p->h * p->w * cp;
  return g;
}

// GEMM view (M, N, K) of a problem.
void gemm_view(const nk_problem* p, int64_t& M, int64_t& N, int64_t& K) {
  if (p->op == NK_OP_MATMUL) { M = p->M; N = p->N; K = p->K; return; }
  const ConvGeom g = geom_of(p);
  M = (int64_t)g.n * g.oh * g.ow; N = p->f; K = (int64_t)g.kh * g.kw * g.c;
}

std::vector<nk_schedule> enumerate(const nk_problem* p) {
  std::vector<nk_schedule> out;
  const int kind = kind_of(p->precision);
  int64_t M, N, K;
  gemm_view(p, M, N, K);
  const int tk = kind == TC_FP8 ? 128 : 64;
  const int64_t nkb = p->op == NK_OP_CONV2D ? (int64_t)p->kh * p->kw * ((p->c + tk - 1) / tk) : (K + tk - 1) / tk;
  for (int tm : {128, 256, 512})
  for (int tn : {64, 128, 256, 512})
    for (int cl : {1, 2})
      for (int split : {1, 2, 4, 8, 16})
        for (int st = 2; st <= 8; ++st) {
          nk_schedule s{tm, tn, tk, cl, st, split};
          if (split > nkb) continue;
          if (p->op == NK_OP_CONV2D ? !tc_conv_schedule_valid(geom_of(p), p->f, s, kind)
                                    : !tc_schedule_valid(kind, s, (int)M, (int)N, (int)K))
            continue;
          out.push_back(s);
        }
  // stride-1 convolutions: the shared-window kernel (tile_k = 64 * taps)
  if (p->op == NK_OP_CONV2D && p->kh * p->kw > 1 && p->stride == 1 && kind == TC_BF16) {
    const ConvGeom g = geom_of(p);
    for (int tm : {128, 256, 512})
      for (int tn : {64, 128, 256})
        for (int st = 1; st <= 4; ++st) {
          nk_schedule s{tm, tn, 64 * p->kh * p->kw, 1, st, 1};
          if (halo_schedule_valid(g, p->f, s)) out.push_back(s);
        }
    // kernel rows stacked along N (tile_k = 64 * KH): one accumulator buffer
    // (tile_m 128, two CTAs per SM) or two (tile_m 256, one CTA per SM)
    for (int st = 1; st <= 4; ++st) {
      nk_schedule s{128, 64, 64 * p->kh, 1, st, 1};
      if (p->kh >= 2 && p->kw >= 2 && halo_schedule_valid(g, p->f, s)) out.push_back(s);
    }
    for (int st = 2; st <= 8; ++st) {
      nk_schedule s{256, 64, 64 * p->kh, 1, st, 1};
      if (p->kh >= 2 && p->kw >= 2 && halo_schedule_valid(g, p->f, s)) out.push_back(s);
    }
  }
  // E4M3 stride-1 convolutions: the stacked window kernel (tile_k = 128 * KH)
  if (p->op == NK_OP_CONV2D && p->kh >= 2 && p->kw >= 2 && p->stride == 1 && kind == TC_FP8) {
    const ConvGeom g = geom_of(p);
    for (int tm : {128, 256})
      for (int st = 1; st <= 8; ++st) {
        nk_schedule s{tm, 64, 128 * p->kh, 1, st, 1};
        if (halo_schedule_valid(g, p->f, s, TC_FP8)) out.push_back(s);
      }
  }
  return out;
}

nk_schedule default_of(const nk_problem* p, int sms) {
  if (p->op == NK_OP_CONV2D) return tc_conv_default_schedule(geom_of(p), p->f, sms, kind_of(p->precision));
  return matmul_default_schedule(kind_of(p->precision), p->M, p->N, p->K, sms);
}

void features(const nk_problem* p, const nk_schedule& s, int sms, float* f) {
  int64_t M, N, K;
  gemm_view(p, M, N, K);
  const int kind = kind_of(p->precision);
  const int64_t tiles = ((M + 127) / 128) * ((N + s.tile_n - 1) / s.tile_n);
  f[0] = (float)(std::log2((double)M) / 16.0);
  f[1] = (float)(std::log2((double)N) / 16.0);
  f[2] = (float)(std::log2((double)K) / 16.0);
  f[3] = p->op == NK_OP_CONV2D ? 1.f : 0.f;
  f[4] = p->op == NK_OP_CONV2D ? (float)(p->kh * p->kw) / 9.f : 0.f;
  f[5] = p->op == NK_OP_CONV2D ? (float)p->stride / 2.f : 0.f;
  f[6] = kind == TC_BF16 ? 1.f : 0.f;
  f[7] = kind == TC_FP8 ? 1.f : 0.f;
  f[8] = kind == TC_BF16X3 ? 1.f : 0.f;
  f[9] = (float)(std::log2((double)s.tile_m) / 8.0);
  f[10] = (float)(std::log2((double)s.tile_n) / 8.0);
  f[11] = (float)(std::log2((double)s.tile_k) / 8.0);
  f[12] = (float)s.cluster / 2.f;
  f[13] = (float)s.stages / 8.f;
  f[14] = (float)(std::log2((double)s.split_k) / 4.0);
  f[15] = (float)(std::log2((double)(tiles * s.split_k) / (double)sms) / 4.0);
}

int sm_count() {
  int sms = 152, dev = 0, v = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      v > 0)
    sms = v;
  return sms;
}

// Launches one schedule on the scratch operands.
struct Runner {
  const nk_problem* p;
  char* base = nullptr;
  size_t op_bytes = 0, total = 0;
  TcGemm g{};
  TcConv c{};

  explicit Runner(const nk_problem* pp, const nk_schedule& s) : p(pp) {
    int64_t M, N, K;
    gemm_view(p, M, N, K);
    const size_t split_bytes = s.split_k > 1 ? (size_t)s.split_k * M * N * 4 : 0;
    if (p->op == NK_OP_MATMUL) {
      const int kind = kind_of(p->precision);
      const int esz = kind == TC_FP8 ? 1 : 2;
      const int64_t ld = (K + 15) / 16 * 16;
      const size_t a = (size_t)M * ld * esz, b = (size_t)N * ld * esz;
      const size_t parts = kind == TC_BF16X3 ? 2 : 1;
      op_bytes = parts * (a + b);
      total = op_bytes + (size_t)M * N * 4 + split_bytes + 4096;
      g.kind = kind; g.M = (int)M; g.N = (int)N; g.K = (int)K;
      g.lda = ld; g.ldb = ld; g.ldc = N; g.alpha = 1.f;
    } else {
      const int kind = kind_of(p->precision);
      const int esz = kind == TC_FP8 ? 1 : 2;
      const ConvGeom geo = geom_of(p);
      const int64_t cp = (p->c + 16 / esz - 1) / (16 / esz) * (16 / esz);
      const size_t ib = (size_t)p->n * p->h * p->w * cp * esz;
      const size_t wb = (size_t)p->f * p->kh * p->kw * cp * esz;
      op_bytes = ib + wb;
      total = op_bytes + (size_t)M * N * 4 + split_bytes + 4096;
      c.kind = kind; c.g = geo; c.F = p->f; c.ldw = cp; c.sW_f = (int64_t)p->kh * p->kw * cp;
      c.alpha = 1.f;
      c.sI_w = cp; c.sI_h = (int64_t)p->w * cp; c.sI_n = (int64_t)p->h * p->w * cp;
    }
  }
  void bind(char* b) {
    base = b;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    if (p->op == NK_OP_MATMUL) {
      const int esz = g.kind == TC_FP8 ? 1 : 2;
      const size_t a = al((size_t)g.M * g.lda * esz), bb = al((size_t)g.N * g.ldb * esz);
      g.A = b; g.B = b + a;
      if (g.kind == TC_BF16X3) { g.A2 = b + a + bb; g.B2 = b + 2 * a + bb; }
      g.C = reinterpret_cast<float*>(b + (g.kind == TC_BF16X3 ? 2 : 1) * (a + bb));
    } else {
      const int esz = c.kind == TC_FP8 ? 1 : 2;
      const size_t ib = al((size_t)p->n * p->h * p->w * c.ldw * esz);
      c.I = b;
      c.Wt = b + ib;
      c.O = reinterpret_cast<float*>(b + ib + al((size_t)p->f * p->kh * p->kw * c.ldw * esz));
    }
  }
  size_t padded_total() const { return total + 4 * 256; }
  char* ws(int64_t M, int64_t N) const {
    (void)M; (void)N;
    const float* o = p->op == NK_OP_MATMUL ? g.C : c.O;
    int64_t MM, NN, KK;
    gemm_view(p, MM, NN, KK);
    return reinterpret_cast<char*>(const_cast<float*>(o)) + (((size_t)MM * NN * 4 + 255) / 256 * 256);
  }
  nk_status run(const nk_schedule& s, cudaStream_t st) {
    int64_t M, N, K;
    gemm_view(p, M, N, K);
    const size_t wsb = s.split_k > 1 ? (size_t)s.split_k * M * N * 4 : 0;
    if (p->op == NK_OP_MATMUL) return tc_gemm(g, s, ws(M, N), wsb, st);
    return tc_conv(c, s, ws(M, N), wsb, st);
  }
};

// Holds the GPU for `ns` nanoseconds of the global timer (at most 2^24
// polls), so that the timed launches behind it are all queued before the
// GPU reaches them and host-side launch work stays outside the timings.
__global__ void hold_kernel(uint64_t ns) {
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int i = 0; i < (1 << 24); ++i) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 >= ns) break;
  }
}

nk_status device_flag_fail(uint32_t flags) {
  if (flags & kErrTimeout) return fail(NK_ERR_TIMEOUT, "a bounded device wait expired while timing");
  return fail(NK_ERR_CUDA, "a kernel reported a launch-configuration error (flags %u) while timing", flags);
}

cudaStream_t timing_stream() {
  static cudaStream_t st[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!st[dev]) cudaStreamCreateWithFlags(&st[dev], cudaStreamNonBlocking);
  return st[dev];
}

// Captures `runs` back-to-back calls of `run` into a graph.
nk_status capture_runs(const RunFn& run, int runs, cudaStream_t st, cudaGraphExec_t* exec) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture(tune)");
  nk_status status = NK_OK;
  for (int i = 0; i < runs && status == NK_OK; ++i) status = run(st);
  e = cudaStreamEndCapture(st, &graph);
  if (status != NK_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return status != NK_OK ? status : cuda_fail(e, "cudaStreamEndCapture(tune)");
  }
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  return e == cudaSuccess ? NK_OK : cuda_fail(e, "cudaGraphInstantiate(tune)");
}

}  // namespace

// Built-in matmul schedule, fitted to the tuner's corpus (150 matmul
// problems, M, N up to ~8000, every legal schedule timed on a GB300).  For
// BF16 and E4M3: the wide pair tile (256 x 512, two MMA chains) once the
// problem has 10 GFLOP of work and at least a tenth of the SMs' worth of
// pair tiles; below that one 128 x 64 tile per CTA with three stages, more
// and narrower tiles than before keeping more independent MMA chains busy,
// and split-K while the tiles would leave half the SMs idle.  Over the
// corpus this took the mean regret of the default from 56 % to 9 % (BF16)
// and from 70 % to 6 % (E4M3).  BF16x3 keeps tc_default_schedule, which the
// corpus has ahead (15.5 % against 16.2 %).
nk_schedule matmul_default_schedule(int kind, int M, int N, int K, int sms) {
  if (kind == TC_BF16X3) return tc_default_schedule(kind, M, N, K, sms);
  nk_schedule s{};
  s.tile_k = kind == TC_FP8 ? 128 : 64;
  const int64_t pair_tiles = (int64_t)((M + 255) / 256) * ((N + 511) / 512);
  if (2.0 * M * N * K >= 1e10 && pair_tiles * 10 >= sms) {
    s.tile_m = 256; s.tile_n = 512; s.cluster = 2; s.stages = 4; s.split_k = 1;
    return s;
  }
  s.tile_m = 128;
  s.tile_n = 64;
  s.cluster = 1;
  s.stages = 3;
  const int64_t tiles = (int64_t)((M + 127) / 128) * ((N + 63) / 64);
  const int nkb = (K + s.tile_k - 1) / s.tile_k;
  s.split_k = 1;
  while (tiles * s.split_k * 2 <= sms && nkb / (s.split_k * 2) >= 4 && s.split_k < 16) s.split_k *= 2;
  return s;
}

// Median device time of one call of `run`.  Two eager calls first (errors
// surface, caches and kernel attributes warm).  The GPU's event clock ticks
// in steps of about 2 us, so each timed sample is a graph of `inner`
// back-to-back calls (inner chosen so a sample lasts about 400 us) between
// two events, and the samples are queued behind hold_kernel: what is timed is
// the kernels alone, not the host work of a call.  `cycle`: consecutive calls
// of `run` work on `cycle` different buffer sets in turn, so `inner` is a
// multiple of it (every sample visits every set).
nk_status time_device(const RunFn& run, int reps, float* ms, int cycle) {
  cudaStream_t st = timing_stream();
  if (!st) return fail(NK_ERR_CUDA, "no timing stream");
  nk_status status = NK_OK;
  for (int i = 0; i < 2; ++i)
    if ((status = run(st)) != NK_OK) return status;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize(tune)");
  {
    uint32_t flags = 0;
    collect_device_errors(&flags);
    if (flags) return device_flag_fail(flags);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // rough duration of one call: 8 eager calls between two events
  cudaEventRecord(e0, st);
  for (int i = 0; i < 8 && status == NK_OK; ++i) status = run(st);
  cudaEventRecord(e1, st);
  e = cudaStreamSynchronize(st);
  float rough = 0.f;
  cudaEventElapsedTime(&rough, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != NK_OK) return status;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize(tune)");
  rough = std::max(rough / 8.f, 0.002f);
  cycle = std::max(1, cycle);
  int inner = std::max(1, std::min(64, (int)std::ceil(0.4f / rough)));
  inner = (std::max(inner, cycle) + cycle - 1) / cycle * cycle;
  cudaGraphExec_t exec = nullptr;
  if ((status = capture_runs(run, inner, st, &exec)) != NK_OK) return status;

  reps = reps < 1 ? 1 : reps;
  std::vector<cudaEvent_t> ev(2 * reps);
  for (auto& x : ev) cudaEventCreate(&x);
  e = cudaGraphLaunch(exec, st);   // warm the graph
  // about 20 us of host work per sample, so hold the GPU that long per sample
  const uint64_t hold = std::min<uint64_t>(50000ull + 20000ull * (uint64_t)reps, 20000000ull);
  hold_kernel<<<1, 1, 0, st>>>(hold);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) {
    cudaEventRecord(ev[2 * i], st);
    e = cudaGraphLaunch(exec, st);
    cudaEventRecord(ev[2 * i + 1], st);
  }
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  std::vector<float> t(reps, 0.f);
  for (int i = 0; i < reps; ++i) {
    cudaEventElapsedTime(&t[i], ev[2 * i], ev[2 * i + 1]);
    t[i] /= (float)inner;
  }
  for (auto& x : ev) cudaEventDestroy(x);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return cuda_fail(e, "timed replays (tune)");
  uint32_t flags = 0;
  collect_device_errors(&flags);
  if (flags) return device_flag_fail(flags);
  std::sort(t.begin(), t.end());
  *ms = t[reps / 2];
  return NK_OK;
}

namespace {

// Buffer sets a timing cycles through: enough that together they hold twice
// the L2, so that every timed call finds its operands evicted by the calls
// since its set was last used (at most 128 sets; problems larger than the
// L2 use one).
int rotation_sets(size_t set_bytes) {
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
      l2 <= 0)
    l2 = 126 << 20;
  const size_t sets = (2 * (size_t)l2 + set_bytes - 1) / set_bytes;
  return (int)std::min<size_t>(std::max<size_t>(sets, 1), 128);
}

// Device time of one schedule on synthetic operands of the problem's shape,
// cold in L2: back-to-back calls rotate over rotation_sets() copies of the
// operands, outputs and workspace.
nk_status time_one(const nk_problem* p, const nk_schedule& s, int reps, float* ms, cudaStream_t user) {
  Runner r(p, s);
  const size_t per = (r.padded_total() + 255) / 256 * 256;
  const int sets = rotation_sets(per);
  void* buf = nullptr;
  nk_status status = scratch(per * sets, &buf);
  if (status != NK_OK) return status;
  std::vector<Runner> rs(sets, r);
  for (int i = 0; i < sets; ++i) rs[i].bind(static_cast<char*>(buf) + per * i);
  if ((status = fill(per * sets)) != NK_OK) return status;
  cudaError_t e = user ? cudaStreamSynchronize(user) : cudaSuccess;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  int next = 0;
  return time_device([&](cudaStream_t st) { return rs[next++ % sets].run(s, st); }, reps, ms, sets);
}

// (1+1) evolution strategy on the schedule grid.  Coordinates: tile_m,
// tile_n, cluster, stages, split_k and the conv path (tile_k: per-tap K
// blocks or the shared window), each an ordered list of levels.  A child
// moves one coordinate one level (or, with probability 1/4, to a random
// level); illegal or already-timed children are redrawn; the child replaces
// the parent when it is faster.  SplitMix64 seeded from the problem, so the
// search is repeatable.  `budget` timings in all, the start included.
struct Rng {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  int below(int n) { return (int)(next() % (uint64_t)n); }
};

nk_status evolve(const nk_problem* p, const std::vector<nk_schedule>& cand, int budget, int reps,
                 cudaStream_t cs, int* best_i, float* best_ms) {
  const int tk0 = p->precision == NK_PREC_FP8 ? 128 : 64;
  const int tk1 = p->op == NK_OP_CONV2D ? 64 * p->kh * p->kw : tk0;
  const int L_TM[] = {128, 256, 512}, L_TN[] = {64, 128, 256, 512}, L_CL[] = {1, 2},
            L_ST[] = {1, 2, 3, 4, 5, 6, 7, 8}, L_SK[] = {1, 2, 4, 8, 16}, L_TK[] = {tk0, tk1};
  const int* LV[6] = {L_TM, L_TN, L_CL, L_ST, L_SK, L_TK};
  const int NL[6] = {3, 4, 2, 8, 5, tk1 != tk0 ? 2 : 1};
  auto level_of = [&](int c, int v) {
    for (int i = 0; i < NL[c]; ++i)
      if (LV[c][i] == v) return i;
    return 0;
  };
  auto find = [&](const int* lv) -> int {
    for (size_t i = 0; i < cand.size(); ++i) {
      const nk_schedule& s = cand[i];
      if (s.tile_m == LV[0][lv[0]] && s.tile_n == LV[1][lv[1]] && s.cluster == LV[2][lv[2]] &&
          s.stages == LV[3][lv[3]] && s.split_k == LV[4][lv[4]] && s.tile_k == LV[5][lv[5]])
        return (int)i;
    }
    return -1;
  };
  Rng rng{(uint64_t)p->op * 1000003ull ^ (uint64_t)p->M * 7919ull ^ (uint64_t)p->N * 104729ull ^
          (uint64_t)p->K * 1299709ull ^ (uint64_t)p->n * 15485863ull ^ (uint64_t)p->h * 32452843ull ^
          (uint64_t)p->c * 49979687ull ^ (uint64_t)p->f * 67867967ull ^ (uint64_t)p->kh * 86028121ull ^
          (uint64_t)p->stride * 104395301ull ^ (uint64_t)p->precision};
  std::vector<char> seen(cand.size(), 0);
  const nk_schedule d = default_of(p, sm_count());
  int cur = -1;
  for (size_t i = 0; i < cand.size(); ++i)
    if (cand[i].tile_m == d.tile_m && cand[i].tile_n == d.tile_n && cand[i].cluster == d.cluster &&
        cand[i].stages == d.stages && cand[i].split_k == d.split_k && cand[i].tile_k == d.tile_k)
      cur = (int)i;
  if (cur < 0) cur = 0;
  float cur_ms = 0.f;
  nk_status st = time_one(p, cand[cur], reps, &cur_ms, cs);
  if (st != NK_OK) return st;
  seen[cur] = 1;
  int timed = 1;
  const int limit = budget < (int)cand.size() ? budget : (int)cand.size();
  while (timed < limit) {
    int lv[6];
    const nk_schedule& s = cand[cur];
    const int base[6] = {level_of(0, s.tile_m), level_of(1, s.tile_n), level_of(2, s.cluster),
                         level_of(3, s.stages), level_of(4, s.split_k), level_of(5, s.tile_k)};
    int child = -1;
    for (int tries = 0; tries < 64 && child < 0; ++tries) {
      for (int c = 0; c < 6; ++c) lv[c] = base[c];
      const int c = rng.below(6);
      if (rng.below(4) == 0) lv[c] = rng.below(NL[c]);
      else lv[c] = lv[c] + (rng.below(2) ? 1 : -1);
      if (lv[c] < 0 || lv[c] >= NL[c]) continue;
      const int i = find(lv);
      if (i >= 0 && !seen[i]) child = i;
    }
    if (child < 0) {   // the neighbourhood is exhausted: any untimed candidate
      int k = rng.below((int)cand.size());
      for (size_t j = 0; j < cand.size() && seen[k]; ++j) k = (k + 1) % (int)cand.size();
      if (seen[k]) break;
      child = k;
    }
    float ms = 0.f;
    if ((st = time_one(p, cand[child], reps, &ms, cs)) != NK_OK) return st;
    seen[child] = 1;
    ++timed;
    if (ms < cur_ms) { cur = child; cur_ms = ms; }
  }
  *best_i = cur;
  *best_ms = cur_ms;
  return NK_OK;
}

}  // namespace
}  // namespace nk

using namespace nk;

extern "C" {

nk_status nk_enumerate_schedules(const nk_problem* p, nk_schedule* out, int32_t cap, int32_t* count) {
  nk_status s = check_problem(p);
  if (s != NK_OK) return s;
  if (!count) return fail(NK_ERR_INVALID_ARG, "count is NULL");
  const auto v = enumerate(p);
  *count = (int32_t)v.size();
  for (int i = 0; i < (int)v.size() && i < cap && out; ++i) out[i] = v[i];
  return NK_OK;
}

nk_status nk_default_schedule(const nk_problem* p, nk_schedule* out) {
  nk_status s = check_problem(p);
  if (s != NK_OK) return s;
  if (!out) return fail(NK_ERR_INVALID_ARG, "out is NULL");
  *out = default_of(p, sm_count());
  return NK_OK;
}

nk_status nk_conv_window_tile(int32_t n, int32_t h, int32_t w, int32_t c, int32_t f, int32_t kh, int32_t kw,
                              int32_t dh, int32_t dw, const int32_t pad[4], const nk_schedule* s, int32_t out[10]) {
  if (!pad || !s || !out) return fail(NK_ERR_INVALID_ARG, "pad, schedule and out must be non-NULL");
  if (n < 1 || h < 1 || w < 1 || c < 1 || f < 1 || kh < 1 || kw < 1 || dh < 1 || dw < 1 || pad[0] < 0 ||
      pad[1] < 0 || pad[2] < 0 || pad[3] < 0)
    return fail(NK_ERR_INVALID_ARG, "extents, dilations must be positive and pads non-negative");
  ConvGeom g{};
  g.n = n; g.h = h; g.w = w; g.c = c;
  g.kh = kh; g.kw = kw;
  g.sh = g.sw = 1;
  g.dh = dh; g.dw = dw;
  g.pt = pad[0]; g.pl = pad[2];
  g.oh = h + pad[0] + pad[1] - (kh - 1) * dh;
  g.ow = w + pad[2] + pad[3] - (kw - 1) * dw;
  if (g.oh < 1 || g.ow < 1) return fail(NK_ERR_INVALID_ARG, "empty output");
  const int cp = (c + 7) / 8 * 8;
  g.sin_w = cp; g.sin_h = (int64_t)w * cp; g.sin_n = (int64_t)h * w * cp;
  if (!halo_tile_info(g, f, *s, out)) return fail(NK_ERR_NO_SCHEDULE, "not a legal window schedule for this convolution");
  return NK_OK;
}

nk_status nk_schedule_features(const nk_problem* p, const nk_schedule* s, int32_t count, float* f) {
  nk_status st = check_problem(p);
  if (st != NK_OK) return st;
  if (count < 0 || (count > 0 && (!s || !f))) return fail(NK_ERR_INVALID_ARG, "bad feature arguments");
  const int sms = sm_count();
  for (int i = 0; i < count; ++i) features(p, s[i], sms, f + (size_t)i * NK_TUNE_FEATURES);
  return NK_OK;
}

nk_status nk_workspace_size(const nk_problem* p, const nk_schedule* sched, size_t* bytes) {
  if (!bytes) return fail(NK_ERR_INVALID_ARG, "bytes is NULL");
  if (!p) return fail(NK_ERR_INVALID_ARG, "problem is NULL");
  // Descriptors only: planning reads shapes and strides, never the memory.
  void* const dummy = reinterpret_cast<void*>(static_cast<uintptr_t>(4096));
  auto dense = [&](nk_tensor& t, int rank, const int64_t* shape) {
    t = nk_tensor{};
    t.ptr = dummy;
    t.dtype = NK_F32;
    t.rank = rank;
    int64_t st = 1;
    for (int d = rank - 1; d >= 0; --d) {
      t.shape[d] = shape[d];
      t.stride[d] = st;
      st *= shape[d];
    }
  };
  if (p->op == NK_OP_MATMUL) {
    if (p->M < 1 || p->N < 1 || p->K < 1) return fail(NK_ERR_INVALID_ARG, "matmul extents must be positive");
    nk_tensor A, B, C;
    const int64_t sa[2] = {p->M, p->K}, sb[2] = {p->K, p->N}, sc[2] = {p->M, p->N};
    dense(A, 2, sa); dense(B, 2, sb); dense(C, 2, sc);
    return nk_matmul_workspace_size(&A, &B, &C, p->precision, sched, bytes);
  }
  if (p->op == NK_OP_CONV2D) {
    if (p->n < 1 || p->h < 1 || p->w < 1 || p->c < 1 || p->f < 1 || p->kh < 1 || p->kw < 1 || p->stride < 1 ||
        p->pad < 0)
      return fail(NK_ERR_INVALID_ARG, "conv extents must be positive");
    const int64_t oh = (p->h + 2 * p->pad - p->kh) / p->stride + 1, ow = (p->w + 2 * p->pad - p->kw) / p->stride + 1;
    if (oh < 1 || ow < 1) return fail(NK_ERR_INVALID_ARG, "empty conv output");
    nk_tensor I, W, O;
    const int64_t si[4] = {p->n, p->h, p->w, p->c}, sw[4] = {p->kh, p->kw, p->c, p->f}, so[4] = {p->n, oh, ow, p->f};
    dense(I, 4, si); dense(W, 4, sw); dense(O, 4, so);
    const int64_t stride[2] = {p->stride, p->stride}, dil[2] = {1, 1}, pad[4] = {p->pad, p->pad, p->pad, p->pad};
    return nk_conv2d_workspace_size(&I, &W, &O, stride, dil, pad, p->precision, sched, bytes);
  }
  return fail(NK_ERR_INVALID_ARG, "unknown op %d", p->op);
}

nk_status nk_grouped_tune(int32_t G, const nk_gemm_group* groups, int32_t precision, int32_t reps,
                          nk_schedule* best, nk_tune_report* rep, void* stream) {
  nk::NvtxRange nvtx_range_("nk_grouped_tune");
  if (!best) return fail(NK_ERR_INVALID_ARG, "best is NULL");
  if (G < 1 || !groups) return fail(NK_ERR_INVALID_ARG, "need at least one group");
  nk_status st = require_device();
  if (st != NK_OK) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  cudaError_t e = user ? cudaStreamSynchronize(user) : cudaSuccess;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  std::vector<nk_gemm_group> gs(groups, groups + G);
  for (auto& q : gs) q.accumulate = 0;   // repeated runs must not pile up into C
  auto time_plan = [&](const nk_schedule* s, float* ms) -> nk_status {
    nk_grouped_plan* plan = nullptr;
    nk_status r = nk_grouped_plan_create(G, gs.data(), precision, s, &plan);
    if (r != NK_OK) return r;
    r = time_device([&](cudaStream_t cs) { return nk_grouped_plan_run(plan, cs); }, reps, ms, 1);
    nk_grouped_plan_destroy(plan);
    return r;
  };
  float dms = 0.f;
  if ((st = time_plan(nullptr, &dms)) != NK_OK) return st;
  int cands = 0, timed = 0;
  float best_ms = 0.f;
  for (int tm : {128, 256})   // 256: CTA pairs
  for (int tn : {64, 128, 256})
    for (int stages = 2; stages <= 8; ++stages) {
      const nk_schedule s{tm, tn, 64, tm == 256 ? 2 : 1, stages, 1};
      nk_grouped_plan* probe = nullptr;
      nk_status r = nk_grouped_plan_create(G, gs.data(), precision, &s, &probe);
      if (r == NK_ERR_NO_SCHEDULE) continue;   // does not fit shared memory
      if (r != NK_OK) return r;
      nk_grouped_plan_destroy(probe);
      ++cands;
      float ms = 0.f;
      if ((st = time_plan(&s, &ms)) != NK_OK) return st;
      ++timed;
      if (timed == 1 || ms < best_ms) {
        best_ms = ms;
        *best = s;
      }
    }
  if (rep) {
    rep->candidates = cands;
    rep->timed = timed;
    rep->best_ms = best_ms;
    rep->default_ms = dms;
  }
  return NK_OK;
}

nk_status nk_conv2d_grouped_tune(int32_t G, const nk_conv_group* groups, int32_t reps, nk_schedule* best,
                                 nk_tune_report* rep, void* stream) {
  nk::NvtxRange nvtx_range_("nk_conv2d_grouped_tune");
  if (!best) return fail(NK_ERR_INVALID_ARG, "best is NULL");
  if (G < 1 || !groups) return fail(NK_ERR_INVALID_ARG, "need at least one group");
  nk_status st = require_device();
  if (st != NK_OK) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  cudaError_t e = user ? cudaStreamSynchronize(user) : cudaSuccess;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  std::vector<nk_conv_group> gs(groups, groups + G);
  for (auto& q : gs) q.accumulate = 0;   // repeated runs must not pile up into O
  auto time_plan = [&](const nk_schedule* s, float* ms) -> nk_status {
    nk_grouped_plan* plan = nullptr;
    nk_status r = nk_conv2d_grouped_plan_create(G, gs.data(), s, &plan);
    if (r != NK_OK) return r;
    r = time_device([&](cudaStream_t cs) { return nk_grouped_plan_run(plan, cs); }, reps, ms, 1);
    nk_grouped_plan_destroy(plan);
    return r;
  };
  float dms = 0.f;
  if ((st = time_plan(nullptr, &dms)) != NK_OK) return st;
  int cands = 0, timed = 0;
  float best_ms = 0.f;
  for (int tn : {64, 128, 256})
    for (int stages = 2; stages <= 8; ++stages) {
      const nk_schedule s{128, tn, 64, 1, stages, 1};
      nk_grouped_plan* probe = nullptr;
      nk_status r = nk_conv2d_grouped_plan_create(G, gs.data(), &s, &probe);
      if (r == NK_ERR_NO_SCHEDULE) continue;   // does not fit shared memory
      if (r != NK_OK) return r;
      nk_grouped_plan_destroy(probe);
      ++cands;
      float ms = 0.f;
      if ((st = time_plan(&s, &ms)) != NK_OK) return st;
      ++timed;
      if (timed == 1 || ms < best_ms) {
        best_ms = ms;
        *best = s;
      }
    }
  if (rep) {
    rep->candidates = cands;
    rep->timed = timed;
    rep->best_ms = best_ms;
    rep->default_ms = dms;
  }
  return NK_OK;
}

nk_status nk_time_schedule(const nk_problem* p, const nk_schedule* s, int32_t reps, float* median_ms,
                           void* stream) {
  nk::NvtxRange nvtx_range_("nk_time_schedule");
  nk_status st = check_problem(p);
  if (st != NK_OK) return st;
  if ((st = require_device()) != NK_OK) return st;
  if (!s || !median_ms) return fail(NK_ERR_INVALID_ARG, "null pointer");
  std::lock_guard<std::mutex> lk(g_mu);
  return time_one(p, *s, reps, median_ms, static_cast<cudaStream_t>(stream));
}

nk_status nk_tune_release(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch) cudaFree(g_scratch);
  g_scratch = nullptr;
  g_scratch_bytes = 0;
  g_filled = 0;
  return NK_OK;
}

nk_status nk_tune(const nk_problem* p, int32_t mode, int32_t topk, const float* mlp_params, int32_t reps,
                  nk_schedule* best, nk_tune_report* rep, void* stream) {
  nk::NvtxRange nvtx_range_("nk_tune");
  nk_status st = check_problem(p);
  if (st != NK_OK) return st;
  if ((st = require_device()) != NK_OK) return st;
  if (!best) return fail(NK_ERR_INVALID_ARG, "best is NULL");
  if (mode != NK_TUNE_EXHAUSTIVE && mode != NK_TUNE_MODEL_TOPK && mode != NK_TUNE_EVOLUTION)
    return fail(NK_ERR_INVALID_ARG, "unknown mode");
  if (mode == NK_TUNE_MODEL_TOPK && (!mlp_params || topk < 1))
    return fail(NK_ERR_INVALID_ARG, "model mode needs parameters and topk >= 1");
  if (mode == NK_TUNE_EVOLUTION && topk < 1) return fail(NK_ERR_INVALID_ARG, "evolution needs a budget >= 1");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const auto cand = enumerate(p);
  if (cand.empty()) return fail(NK_ERR_NO_SCHEDULE, "no legal schedule");
  if (mode == NK_TUNE_EVOLUTION) {
    std::lock_guard<std::mutex> lk(g_mu);
    nk::NvtxRange phase("nk_tune: evolution search");
    int bi = 0;
    float bms = 0.f;
    st = evolve(p, cand, topk, reps, cs, &bi, &bms);
    if (st != NK_OK) return st;
    *best = cand[bi];
    if (rep) {
      rep->candidates = (int32_t)cand.size();
      rep->timed = topk < (int)cand.size() ? topk : (int32_t)cand.size();
      rep->best_ms = bms;
      float dms = 0.f;
      st = time_one(p, default_of(p, sm_count()), reps, &dms, cs);
      if (st != NK_OK) return st;
      rep->default_ms = dms;
    }
    return NK_OK;
  }
  std::vector<int> order(cand.size());
  for (size_t i = 0; i < cand.size(); ++i) order[i] = (int)i;
  if (mode == NK_TUNE_MODEL_TOPK) {
    nk::NvtxRange phase("nk_tune: cost-model ranking");
    const int sms = sm_count();
    std::vector<float> feat(cand.size() * NK_TUNE_FEATURES);
    for (size_t i = 0; i < cand.size(); ++i) features(p, cand[i], sms, feat.data() + i * NK_TUNE_FEATURES);
    float* dX = nullptr;
    cudaError_t e = cudaMalloc(&dX, feat.size() * 4 + cand.size() * 4);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(tune features)");
    float* dy = dX + feat.size();
    std::vector<float> pred(cand.size());
    e = cudaMemcpyAsync(dX, feat.data(), feat.size() * 4, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) st = nk_mlp_forward(mlp_params, dX, (int64_t)cand.size(), dy, stream);
    if (e == cudaSuccess && st == NK_OK) e = cudaMemcpyAsync(pred.data(), dy, pred.size() * 4, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    cudaFree(dX);
    if (st != NK_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "cost-model inference");
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pred[a] < pred[b]; });
    if ((int)order.size() > topk) order.resize(topk);
    std::sort(order.begin(), order.end());   // time in enumeration order: same tie-break as exhaustive
  }
  std::lock_guard<std::mutex> lk(g_mu);
  float best_ms = INFINITY;
  int best_i = -1;
  {
    nk::NvtxRange phase(mode == NK_TUNE_MODEL_TOPK ? "nk_tune: timing the top-k" : "nk_tune: timing every candidate");
    for (int i : order) {
      float ms = 0.f;
      st = time_one(p, cand[i], reps, &ms, cs);
      if (st != NK_OK) return st;
      if (ms < best_ms) { best_ms = ms; best_i = i; }
    }
  }
  *best = cand[best_i];
  if (rep) {
    nk::NvtxRange phase("nk_tune: timing the built-in default");
    rep->candidates = (int32_t)cand.size();
    rep->timed = (int32_t)order.size();
    rep->best_ms = best_ms;
    float dms = 0.f;
    const nk_schedule d = default_of(p, sm_count());
    st = time_one(p, d, reps, &dms, cs);
    if (st != NK_OK) return st;
    rep->default_ms = dms;
  }
  return NK_OK;
}

}  // extern "C"
