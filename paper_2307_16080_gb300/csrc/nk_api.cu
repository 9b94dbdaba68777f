// nk_api.cu -- the C ABI: argument checks, problem normalisation, workspace
// layout and dispatch to the kernel families.
//
// linalg.matmul (Sec. 2.1.1 Listing "linalg-matmul") is normalised so that the
// output is row-major: a column-major C is computed as C^T = B^T A^T (the
// operands swap roles and the bias moves to the row index).  FP32 requests
// run on the CUDA cores; BF16 / BF16x3 / FP8 requests first cast the FP32
// operands into K-major buffers in the caller's workspace, then run the
// tcgen05 kernel.  Nothing here allocates device memory.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <cmath>
#include <mutex>
#include <string>
#include <utility>

#include "nk_internal.cuh"

namespace nk {

static thread_local std::string t_last_error;

nk_status fail(nk_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return s;
}

nk_status cuda_fail(cudaError_t e, const char* what) {
  return fail(NK_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

nk_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NK_OK : cuda_fail(e, what);
}

static std::mutex g_dev_mu;
static int g_dev_state[64];   // 0 unknown, 1 ok, 2 unsupported
static int g_dev_sms[64];

nk_status require_device(int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(NK_ERR_CUDA, "device ordinal %d out of range", dev);
  {
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (g_dev_state[dev] == 0) {
      cudaDeviceProp prop;
      e = cudaGetDeviceProperties(&prop, dev);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
      g_dev_state[dev] = (prop.major == 10 && prop.minor == 3) ? 1 : 2;
      g_dev_sms[dev] = prop.multiProcessorCount;
    }
  }
  if (g_dev_state[dev] != 1)
    return fail(NK_ERR_CUDA, "device %d is not an sm_103 (GB300) GPU; this library has no other path",
                dev);
  if (sms) *sms = g_dev_sms[dev];
  return NK_OK;
}

static std::atomic<int64_t> g_wait_budget{0};
static constexpr int64_t kDefaultWaitBudget = int64_t(1) << 31;   // ~seconds of spinning
int64_t wait_budget() {
  int64_t b = g_wait_budget.load();
  return b > 0 ? b : kDefaultWaitBudget;
}

static std::atomic<int> g_pdl{1};
bool pdl_enabled() { return g_pdl.load(std::memory_order_relaxed) != 0; }

nk_status collect_device_errors(uint32_t* flags) {
  *flags = tc_read_and_clear_errors() | halo_read_and_clear_errors();
  return NK_OK;
}

}  // namespace nk

using namespace nk;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int dtype_size(int dt) {
  switch (dt) {
    case NK_F32: return 4;
    case NK_BF16: return 2;
    case NK_F8E4M3: return 1;
    case NK_F64: return 8;
    default: return 0;
  }
}

}  // namespace

nk_status nk::ew_program(const nk_ew_program* prog, const nk_tensor* like, EwProg* out, const char* what) {
  *out = EwProg{};
  if (!prog) return NK_OK;
  if (prog->n < 0 || prog->n > NK_EW_MAX)
    return fail(NK_ERR_INVALID_ARG, "%s: %d operations (0..%d allowed)", what, prog->n, NK_EW_MAX);
  int64_t elems = 1;
  for (int d = 0; d < like->rank; ++d) elems *= like->shape[d];
  for (int i = 0; i < prog->n; ++i) {
    const nk_ew_op& o = prog->ops[i];
    out->op[i] = o.op;
    out->a[i] = o.a;
    out->b[i] = o.b;
    out->t[i] = nullptr;
    switch (o.op) {
      case NK_EW_MUL:
      case NK_EW_ADD: {
        const nk_tensor& t = o.t;
        if (t.dtype != NK_F32) return fail(NK_ERR_INVALID_ARG, "%s op %d: the tensor operand must be FP32", what, i);
        if (t.rank != like->rank)
          return fail(NK_ERR_INVALID_ARG, "%s op %d: the tensor operand has rank %d, not %d", what, i, t.rank,
                      like->rank);
        for (int d = 0; d < like->rank; ++d)
          if (t.shape[d] != like->shape[d])
            return fail(NK_ERR_INVALID_ARG, "%s op %d: the tensor operand's dim %d is %lld, not %lld", what, i, d,
                        (long long)t.shape[d], (long long)like->shape[d]);
        for (int d = 0; d < like->rank; ++d) {
          if (like->shape[d] > 1 && t.stride[d] != like->stride[d])
            return fail(NK_ERR_INVALID_ARG, "%s op %d: the tensor operand's stride %d is %lld, not %lld", what, i,
                        d, (long long)t.stride[d], (long long)like->stride[d]);
        }
        if (elems > 0 && !t.ptr) return fail(NK_ERR_INVALID_ARG, "%s op %d: NULL tensor operand", what, i);
        if (reinterpret_cast<uintptr_t>(t.ptr) & 3)
          return fail(NK_ERR_INVALID_ARG, "%s op %d: the tensor operand is not 4-byte aligned", what, i);
        out->t[i] = static_cast<const float*>(t.ptr);
        break;
      }
      case NK_EW_AFFINE:
        if (o.a != o.a || o.b != o.b) return fail(NK_ERR_INVALID_ARG, "%s op %d: NaN coefficient", what, i);
        break;
      case NK_EW_CLAMP:
        if (o.a != o.a || o.b != o.b || !(o.a <= o.b))
          return fail(NK_ERR_INVALID_ARG, "%s op %d: CLAMP needs a <= b (no NaN)", what, i);
        break;
      case NK_EW_RELU:
      case NK_EW_GELU:
      case NK_EW_GELU_TANH:
      case NK_EW_SILU:
      case NK_EW_SIGMOID:
      case NK_EW_TANH:
        break;
      default:
        return fail(NK_ERR_INVALID_ARG, "%s op %d: unknown opcode %d", what, i, o.op);
    }
  }
  out->n = prog->n;
  return NK_OK;
}

namespace {

// A rank-2 view after normalisation.
struct View {
  const void* p;
  int64_t s0, s1;   // strides of dim 0 and dim 1 (elements)
};

struct MatmulPlan {
  int M = 0, N = 0, K = 0;
  View A{}, B{}, C{};
  int bias_on_m = 0;
  int in_dtype = NK_F32;
  int prec = NK_PREC_F32;
  nk_schedule sched{};
  int64_t ldk = 0;       // leading dimension of the cast operands
  size_t off_a = 0, off_b = 0, off_a2 = 0, off_b2 = 0, off_scal = 0, off_amax = 0, off_kern = 0;
  size_t kern_bytes = 0;
  size_t total = 0;
  bool direct = false;   // operands already in tensor-core form (no cast)
};

nk_status check_matrix(const nk_tensor* t, const char* name) {
  if (!t) return fail(NK_ERR_INVALID_ARG, "%s is NULL", name);
  if (t->rank != 2) return fail(NK_ERR_INVALID_ARG, "%s must have rank 2 (got %d)", name, t->rank);
  if (t->shape[0] < 0 || t->shape[1] < 0)
    return fail(NK_ERR_INVALID_ARG, "%s has a negative extent", name);
  if (dtype_size(t->dtype) == 0) return fail(NK_ERR_INVALID_ARG, "%s has unknown dtype %d", name, t->dtype);
  if (t->shape[0] * t->shape[1] > 0) {
    if (!t->ptr) return fail(NK_ERR_INVALID_ARG, "%s has a NULL pointer", name);
    bool unit = t->stride[1] == 1 || t->stride[0] == 1 || t->shape[1] == 1 || t->shape[0] == 1;
    if (!unit) return fail(NK_ERR_UNSUPPORTED, "%s needs a unit stride in one dimension", name);
  }
  return NK_OK;
}

// True when the view is row-major (unit stride on dim 1), false for column-major.
bool row_major(const nk_tensor* t) {
  if (t->stride[1] == 1) return true;
  if (t->stride[0] == 1) return false;
  return t->shape[1] <= 1;
}

nk_status plan_matmul(const nk_tensor* A, const nk_tensor* B, const nk_tensor* C, int prec,
                      const nk_schedule* user, MatmulPlan& P) {
  nk_status s;
  if ((s = check_matrix(A, "A")) != NK_OK) return s;
  if ((s = check_matrix(B, "B")) != NK_OK) return s;
  if ((s = check_matrix(C, "C")) != NK_OK) return s;
  const int64_t M = A->shape[0], K = A->shape[1], N = B->shape[1];
  if (B->shape[0] != K) return fail(NK_ERR_INVALID_ARG, "A is [%lld,%lld] but B is [%lld,%lld]",
                                    (long long)M, (long long)K, (long long)B->shape[0], (long long)N);
  if (C->shape[0] != M || C->shape[1] != N)
    return fail(NK_ERR_INVALID_ARG, "C must be [%lld,%lld]", (long long)M, (long long)N);
  if (C->dtype != NK_F32) return fail(NK_ERR_UNSUPPORTED, "C must be FP32");
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX)
    return fail(NK_ERR_UNSUPPORTED, "extents above 2^31-1");
  if (A->dtype != B->dtype) return fail(NK_ERR_INVALID_ARG, "A and B must share a dtype");
  if (prec < NK_PREC_F32 || prec > NK_PREC_FP8) return fail(NK_ERR_INVALID_ARG, "unknown precision %d", prec);
  P.in_dtype = A->dtype;
  P.prec = prec;
  if (prec == NK_PREC_F32 && A->dtype != NK_F32)
    return fail(NK_ERR_INVALID_ARG, "NK_PREC_F32 needs FP32 operands");
  if (A->dtype == NK_BF16 && prec != NK_PREC_BF16)
    return fail(NK_ERR_INVALID_ARG, "BF16 operands go with NK_PREC_BF16");
  if (A->dtype == NK_F8E4M3 && prec != NK_PREC_FP8)
    return fail(NK_ERR_INVALID_ARG, "E4M3 operands go with NK_PREC_FP8");
  if (A->dtype == NK_F64) return fail(NK_ERR_UNSUPPORTED, "FP64 operands are not supported");

  // Transpose identity when C is column-major: C^T = B^T A^T.
  const bool c_row = row_major(C);
  if (c_row) {
    P.M = (int)M; P.N = (int)N; P.K = (int)K;
    P.A = {A->ptr, A->stride[0], A->stride[1]};
    P.B = {B->ptr, B->stride[0], B->stride[1]};
    P.C = {C->ptr, C->stride[0], C->stride[1]};
    P.bias_on_m = 0;
  } else {
    P.M = (int)N; P.N = (int)M; P.K = (int)K;
    P.A = {B->ptr, B->stride[1], B->stride[0]};
    P.B = {A->ptr, A->stride[1], A->stride[0]};
    P.C = {C->ptr, C->stride[1], C->stride[0]};
    P.bias_on_m = 1;
  }
  P.sched = user ? *user : nk_schedule{0, 0, 0, 0, 0, 0};
  P.total = 0;
  if (prec == NK_PREC_F32) {
    int split = P.sched.split_k > 0 ? P.sched.split_k : 1;
    int tile = P.sched.tile_m > 0 ? P.sched.tile_m : 128;
    if (P.sched.tile_m == 0 && (int64_t)((P.M + 127) / 128) * ((P.N + 127) / 128) < 152) tile = 64;
    P.sched.tile_m = P.sched.tile_n = tile;
    P.sched.tile_k = 16;
    P.sched.cluster = 1;
    P.sched.stages = 2;
    P.sched.split_k = split;
    P.total = simt_gemm_ws(P.M, P.N, split);
    return NK_OK;
  }
  // Tensor-core precisions.
  int kind = prec == NK_PREC_BF16 ? TC_BF16 : prec == NK_PREC_FP8 ? TC_FP8 : TC_BF16X3;
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) sms = v;
  }
  nk_schedule d = matmul_default_schedule(kind, P.M, P.N, P.K, sms);
  nk_schedule& S = P.sched;
  if (S.tile_m == 0) S.tile_m = d.tile_m;
  if (S.tile_n == 0) S.tile_n = d.tile_n;
  if (S.tile_k == 0) S.tile_k = d.tile_k;
  if (S.cluster == 0) S.cluster = d.cluster;
  if (S.stages == 0) S.stages = d.stages;
  if (S.split_k == 0) S.split_k = d.split_k;
  if (!tc_schedule_valid(kind, S, P.M, P.N, P.K))
    return fail(NK_ERR_NO_SCHEDULE, "schedule %dx%dx%d cluster %d stages %d split %d is not legal here",
                S.tile_m, S.tile_n, S.tile_k, S.cluster, S.stages, S.split_k);
  const int esz = kind == TC_FP8 ? 1 : 2;
  if (A->dtype != NK_F32) {
    // Direct path: A must be K-major ([M,K] row-major) and B K-major ([K,N] column-major).
    P.direct = true;
    if (!c_row) return fail(NK_ERR_UNSUPPORTED, "pre-cast operands need a row-major C");
    if (!(P.A.s1 == 1 || P.K == 1) || !(P.B.s0 == 1 || P.K == 1))
      return fail(NK_ERR_UNSUPPORTED,
                  "pre-cast operands must be K-major: A [M,K] row-major, B [K,N] column-major");
    if (!aligned16(P.A.p) || !aligned16(P.B.p) || (P.A.s0 * esz) % 16 || (P.B.s1 * esz) % 16)
      return fail(NK_ERR_MISALIGNED, "pre-cast operands need 16-byte aligned bases and row strides");
    P.ldk = 0;
    TcGemm g{};
    g.kind = kind; g.M = P.M; g.N = P.N; g.K = P.K;
    P.kern_bytes = tc_gemm_ws(g, S);
    P.off_kern = 0;
    P.total = align_up(P.kern_bytes);
    return NK_OK;
  }
  P.ldk = round_up(P.K, 16);
  size_t off = 0;
  const size_t a_bytes = align_up((size_t)P.M * P.ldk * esz);
  const size_t b_bytes = align_up((size_t)P.N * P.ldk * esz);
  P.off_a = off; off += a_bytes;
  P.off_b = off; off += b_bytes;
  if (kind == TC_BF16X3) {
    P.off_a2 = off; off += a_bytes;
    P.off_b2 = off; off += b_bytes;
  }
  P.off_scal = off; off += kAlign;                         // amax_a, amax_b, s_a, s_b
  if (kind == TC_FP8) { P.off_amax = off; off += align_up(prep_amax_ws(0)); }
  TcGemm g{};
  g.kind = kind; g.M = P.M; g.N = P.N; g.K = P.K;
  P.kern_bytes = tc_gemm_ws(g, S);
  P.off_kern = off; off += align_up(P.kern_bytes);
  P.total = off;
  return NK_OK;
}

}  // namespace

extern "C" {

const char* nk_last_error(void) { return t_last_error.c_str(); }

nk_status nk_device_info(int32_t* sm_count, int32_t* cc_major, int32_t* cc_minor) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  if (sm_count) *sm_count = prop.multiProcessorCount;
  if (cc_major) *cc_major = prop.major;
  if (cc_minor) *cc_minor = prop.minor;
  return NK_OK;
}

nk_status nk_set_wait_budget(int64_t iterations) {
  if (iterations < 0) return fail(NK_ERR_INVALID_ARG, "negative wait budget");
  g_wait_budget.store(iterations);
  return NK_OK;
}

nk_status nk_set_pdl(int32_t enabled) {
  nk::g_pdl.store(enabled ? 1 : 0);
  return NK_OK;
}

int32_t nk_get_pdl(void) { return nk::pdl_enabled() ? 1 : 0; }

nk_status nk_sync_status(void* stream) {
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  uint32_t flags = 0;
  collect_device_errors(&flags);
  if (flags & kErrLaunch) return fail(NK_ERR_CUDA, "a kernel was launched with less shared memory than its layout");
  if (flags & kErrTimeout) return fail(NK_ERR_TIMEOUT, "a bounded device wait expired");
  return NK_OK;
}

nk_status nk_matmul_workspace_size(const nk_tensor* A, const nk_tensor* B, const nk_tensor* C,
                                   int32_t precision, const nk_schedule* sched, size_t* bytes) {
  if (!bytes) return fail(NK_ERR_INVALID_ARG, "bytes is NULL");
  MatmulPlan P;
  nk_status s = plan_matmul(A, B, C, precision, sched, P);
  if (s != NK_OK) return s;
  *bytes = P.total;
  return NK_OK;
}

nk_status nk_matmul(const nk_tensor* A, const nk_tensor* B, nk_tensor* C, int32_t precision,
                    const nk_epilogue* epi, const nk_schedule* sched, void* ws, size_t ws_bytes,
                    void* stream) {
  nk::NvtxRange nvtx_range_("nk_matmul");
  MatmulPlan P;
  nk_status s = plan_matmul(A, B, C, precision, sched, P);
  if (s != NK_OK) return s;
  const nk_epilogue e0{nullptr, 0, 0, 1.f, 1.f, nullptr, nullptr, nullptr};
  const nk_epilogue& E = epi ? *epi : e0;
  // Fused programs; operands swap roles with C column-major (C^T = B^T A^T),
  // and so do their prologues.  Offsets stay memory offsets of each tensor.
  EwProg ew, pro_a, pro_b;
  if ((s = ew_program(E.ew, C, &ew, "ew")) != NK_OK) return s;
  if ((s = ew_program(E.pro_a, A, &pro_a, "pro_a")) != NK_OK) return s;
  if ((s = ew_program(E.pro_b, B, &pro_b, "pro_b")) != NK_OK) return s;
  if (P.bias_on_m) std::swap(pro_a, pro_b);
  if (P.direct && (pro_a.n || pro_b.n))
    return fail(NK_ERR_UNSUPPORTED, "operands given as BF16 / E4M3 take no prologue (it runs before the cast)");
  if ((s = require_device()) != NK_OK) return s;
  if (P.total > 0 && (!ws || ws_bytes < P.total))
    return fail(NK_ERR_WORKSPACE, "nk_matmul needs %zu bytes of workspace (got %zu)", P.total, ws_bytes);
  if (ws && !aligned16(ws)) return fail(NK_ERR_MISALIGNED, "workspace must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P.M == 0 || P.N == 0) return NK_OK;
  char* w = static_cast<char*>(ws);

  if (P.prec == NK_PREC_F32) {
    SimtGemm g{};
    g.A = static_cast<const float*>(P.A.p); g.sam = P.A.s0; g.sak = P.A.s1;
    g.B = static_cast<const float*>(P.B.p); g.sbk = P.B.s0; g.sbn = P.B.s1;
    g.C = static_cast<float*>(const_cast<void*>(P.C.p)); g.scm = P.C.s0; g.scn = P.C.s1;
    g.bias = E.bias; g.bias_on_m = P.bias_on_m;
    g.M = P.M; g.N = P.N; g.K = P.K;
    g.alpha = 1.f; g.beta = E.accumulate ? 1.f : 0.f; g.relu = E.relu;
    g.is_conv = 0;
    g.ew = ew; g.pro_a = pro_a; g.pro_b = pro_b;
    return simt_gemm(g, P.sched.tile_m, P.sched.split_k, ws, ws_bytes, st);
  }

  const int kind = P.prec == NK_PREC_BF16 ? TC_BF16 : P.prec == NK_PREC_FP8 ? TC_FP8 : TC_BF16X3;
  TcGemm g{};
  g.kind = kind; g.M = P.M; g.N = P.N; g.K = P.K;
  g.C = static_cast<float*>(const_cast<void*>(P.C.p));
  g.ldc = P.C.s0;
  if (P.C.s1 != 1 && P.N > 1) return fail(NK_ERR_UNSUPPORTED, "C needs a unit stride");
  g.bias = E.bias; g.bias_on_m = P.bias_on_m; g.relu = E.relu;
  g.beta = E.accumulate ? 1.f : 0.f;
  g.alpha = 1.f;
  g.ew = ew;
  if (P.direct) {
    g.A = P.A.p; g.lda = P.A.s0;
    g.B = P.B.p; g.ldb = P.B.s1;
    if (kind == TC_FP8) {
      if (!(E.scale_a > 0.f) || !(E.scale_b > 0.f))
        return fail(NK_ERR_INVALID_ARG, "pre-quantised FP8 needs positive scale_a and scale_b");
      g.alpha = 1.f / (E.scale_a * E.scale_b);
    }
    return tc_gemm(g, P.sched, w + P.off_kern, P.kern_bytes, st);
  }
  // Cast the FP32 operands into K-major buffers.
  const float* Af = static_cast<const float*>(P.A.p);
  const float* Bf = static_cast<const float*>(P.B.p);
  // A [M,K]: row-major -> plain cast; column-major -> transposing cast of A^T [K,M].
  const bool a_kmajor = P.A.s1 == 1 || P.K == 1;
  const bool b_kmajor = P.B.s0 == 1 || P.K == 1;   // B [K,N] column-major = Bt row-major
  float* scal = reinterpret_cast<float*>(w + P.off_scal);   // amax_a, amax_b, s_a, s_b
  void* a0 = w + P.off_a;
  void* b0 = w + P.off_b;
  void* a1 = kind == TC_BF16X3 ? w + P.off_a2 : nullptr;
  void* b1 = kind == TC_BF16X3 ? w + P.off_b2 : nullptr;
  const int ck = kind == TC_BF16 ? 0 : kind == TC_FP8 ? 1 : 2;
  if (kind == TC_FP8) {
    void* aw = w + P.off_amax;
    const size_t awb = prep_amax_ws(0);
    if (a_kmajor) s = prep_amax(Af, P.M, P.K, P.A.s0, scal + 0, aw, awb, st, &pro_a);
    else s = prep_amax(Af, P.K, P.M, P.A.s1, scal + 0, aw, awb, st, &pro_a);
    if (s != NK_OK) return s;
    if (b_kmajor) s = prep_amax(Bf, P.N, P.K, P.B.s1, scal + 1, aw, awb, st, &pro_b);
    else s = prep_amax(Bf, P.K, P.N, P.B.s0, scal + 1, aw, awb, st, &pro_b);
    if (s != NK_OK) return s;
  }
  if (a_kmajor) s = prep_cast(ck, Af, P.M, P.K, P.A.s0, scal + 0, a0, a1, P.ldk, 0, scal + 2, st, &pro_a);
  else s = prep_cast(ck, Af, P.K, P.M, P.A.s1, scal + 0, a0, a1, P.ldk, 1, scal + 2, st, &pro_a);
  if (s != NK_OK) return s;
  if (b_kmajor) s = prep_cast(ck, Bf, P.N, P.K, P.B.s1, scal + 1, b0, b1, P.ldk, 0, scal + 3, st, &pro_b);
  else s = prep_cast(ck, Bf, P.K, P.N, P.B.s0, scal + 1, b0, b1, P.ldk, 1, scal + 3, st, &pro_b);
  if (s != NK_OK) return s;
  g.A = a0; g.B = b0; g.A2 = a1; g.B2 = b1;
  g.lda = P.ldk; g.ldb = P.ldk;
  if (kind == TC_FP8) { g.scale_a = scal + 2; g.scale_b = scal + 3; }
  return tc_gemm(g, P.sched, w + P.off_kern, P.kern_bytes, st);
}

// ------------------------------------------------------------------ conv
// BF16 or E4M3 weights in the tensor-core layout: W[kh,kw,c,f] at
// f*sF + (kh*KW + kw)*ldw + c, ldw >= C, sF >= KH*KW*ldw, both multiples of
// 16 bytes (8 BF16, 16 E4M3: 16-byte rows for TMA).
static bool packed_weights(const nk_tensor* W) {
  const int64_t ldw = W->stride[1], sF = W->stride[3];
  const int per16 = W->dtype == NK_F8E4M3 ? 16 : 8;
  return W->stride[2] == 1 && ldw >= W->shape[2] && ldw % per16 == 0 && W->stride[0] == W->shape[1] * ldw &&
         sF % per16 == 0 && sF >= W->shape[0] * W->shape[1] * ldw;
}

static nk_status plan_conv(const nk_tensor* I, const nk_tensor* W, const nk_tensor* O,
                           const int64_t stride[2], const int64_t dilation[2], const int64_t pad[4],
                           ConvGeom& g) {
  if (!I || !W || !O) return fail(NK_ERR_INVALID_ARG, "I, W and O must be non-NULL");
  if (!stride || !dilation || !pad) return fail(NK_ERR_INVALID_ARG, "stride, dilation, pad must be non-NULL");
  if (I->rank != 4 || W->rank != 4 || O->rank != 4) return fail(NK_ERR_INVALID_ARG, "I, W, O must have rank 4");
  if (I->stride[3] != 1 || O->stride[3] != 1)
    return fail(NK_ERR_UNSUPPORTED, "the last dimension of I and O must have unit stride");
  if (O->dtype != NK_F32 && O->dtype != NK_BF16) return fail(NK_ERR_UNSUPPORTED, "O must be FP32 or BF16");
  if ((I->dtype != NK_F32 && I->dtype != NK_BF16 && I->dtype != NK_F8E4M3) ||
      (W->dtype != NK_F32 && W->dtype != NK_BF16 && W->dtype != NK_F8E4M3))
    return fail(NK_ERR_INVALID_ARG, "I and W must be FP32, BF16 or E4M3");
  for (int i = 0; i < 2; ++i)
    if (stride[i] < 1 || dilation[i] < 1) return fail(NK_ERR_INVALID_ARG, "stride and dilation must be >= 1");
  for (int i = 0; i < 4; ++i)
    if (pad[i] < 0) return fail(NK_ERR_INVALID_ARG, "padding must be >= 0");
  if (I->shape[3] != W->shape[2]) return fail(NK_ERR_INVALID_ARG, "I channels != W input channels");
  g.n = (int)I->shape[0]; g.h = (int)I->shape[1]; g.w = (int)I->shape[2]; g.c = (int)I->shape[3];
  g.kh = (int)W->shape[0]; g.kw = (int)W->shape[1];
  g.sh = (int)stride[0]; g.sw = (int)stride[1]; g.dh = (int)dilation[0]; g.dw = (int)dilation[1];
  g.pt = (int)pad[0]; g.pl = (int)pad[2];
  const int64_t oh = (I->shape[1] + pad[0] + pad[1] - dilation[0] * (W->shape[0] - 1) - 1) / stride[0] + 1;
  const int64_t ow = (I->shape[2] + pad[2] + pad[3] - dilation[1] * (W->shape[1] - 1) - 1) / stride[1] + 1;
  if (oh < 1 || ow < 1) return fail(NK_ERR_INVALID_ARG, "empty output window");
  if (O->shape[0] != I->shape[0] || O->shape[1] != oh || O->shape[2] != ow || O->shape[3] != W->shape[3])
    return fail(NK_ERR_INVALID_ARG, "O must be [%lld,%lld,%lld,%lld]", (long long)I->shape[0],
                (long long)oh, (long long)ow, (long long)W->shape[3]);
  g.oh = (int)oh; g.ow = (int)ow;
  g.sin_n = I->stride[0]; g.sin_h = I->stride[1]; g.sin_w = I->stride[2];
  if (W->dtype == NK_BF16 || W->dtype == NK_F8E4M3) {
    // packed for the tensor cores (nk_conv2d_pack_weights / _fp8): channels
    // contiguous per filter tap, taps at a uniform stride
    if (!packed_weights(W))
      return fail(NK_ERR_UNSUPPORTED,
                  "a BF16 / E4M3 W must be packed: strides {KW*ldw, ldw, 1, sF} with ldw >= C and "
                  "sF >= KH*KW*ldw, both 16-byte multiples (see nk_conv2d_pack_weights)");
  } else if (W->stride[3] != 1 || W->stride[2] != W->shape[3] || W->stride[1] != W->shape[2] * W->shape[3] ||
             W->stride[0] != W->shape[1] * W->shape[2] * W->shape[3]) {
    return fail(NK_ERR_UNSUPPORTED, "an FP32 W must be contiguous HWCF");
  }
  if ((int64_t)g.n * g.oh * g.ow > INT32_MAX) return fail(NK_ERR_UNSUPPORTED, "output too large");
  return NK_OK;
}

// Workspace layout of a tensor-core convolution: BF16 copies of I (when given
// in FP32, channels padded to a multiple of 8) and of W transposed to
// [F][taps][Cp], then the split-K partials.
struct ConvPlan {
  nk_schedule sched{};
  int kind = TC_BF16;     // TC_BF16 or TC_FP8 operands
  int Cp = 0;             // channels per row of a converted operand (16-byte rows)
  bool cast_i = false, cast_w = false;
  size_t off_i = 0, off_w = 0, off_scal = 0, off_amax = 0, off_k = 0, kern = 0, total = 0;
};

static nk_status plan_tc_conv(const nk_tensor* I, const nk_tensor* W, const nk_tensor* O, const ConvGeom& g,
                              int precision, const nk_schedule* user, ConvPlan& P) {
  P.kind = precision == NK_PREC_FP8 ? TC_FP8 : TC_BF16;
  const bool f8_in = I->dtype == NK_F8E4M3, f8_w = W->dtype == NK_F8E4M3;
  if (P.kind == TC_FP8 && !((I->dtype == NK_F32 && W->dtype == NK_F32) || (f8_in && f8_w)))
    return fail(NK_ERR_UNSUPPORTED,
                "an E4M3 convolution takes FP32 I and W (quantised per call with per-tensor scales) or both "
                "already in E4M3 (I NHWC, W packed by nk_conv2d_pack_weights_fp8; scales in the epilogue)");
  if (P.kind == TC_BF16 && (f8_in || f8_w))
    return fail(NK_ERR_UNSUPPORTED, "E4M3 operands need NK_PREC_FP8");
  if ((W->dtype == NK_BF16 || f8_w) && (reinterpret_cast<uintptr_t>(W->ptr) & 15))
    return fail(NK_ERR_MISALIGNED, "packed weights must be 16-byte aligned");
  if (f8_in && ((reinterpret_cast<uintptr_t>(I->ptr) & 15) || g.sin_w % 16 || g.sin_h % 16 || g.sin_n % 16))
    return fail(NK_ERR_MISALIGNED, "an E4M3 I needs a 16-byte aligned base and 16-byte multiples for its strides");
  int sms = 152, dev = 0, v = 0;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
    sms = v;
  const int F = (int)W->shape[3];
  nk_schedule S = user ? *user : nk_schedule{0, 0, 0, 0, 0, 0};
  if (!S.tile_m || !S.tile_n || !S.tile_k || !S.cluster || !S.stages || !S.split_k) {
    const nk_schedule d = tc_conv_default_schedule(g, F, sms, P.kind);
    if (S.tile_m == 0) S.tile_m = d.tile_m;
    if (S.tile_n == 0) S.tile_n = d.tile_n;
    if (S.tile_k == 0) S.tile_k = d.tile_k;
    if (S.cluster == 0) S.cluster = d.cluster;
    if (S.stages == 0) S.stages = d.stages;
    if (S.split_k == 0) S.split_k = d.split_k;
  }
  if (!tc_conv_schedule_valid(g, F, S, P.kind)) return fail(NK_ERR_NO_SCHEDULE, "illegal conv schedule");
  P.sched = S;
  const int esz = P.kind == TC_FP8 ? 1 : 2;
  const int per16 = 16 / esz;   // elements per 16-byte step
  P.Cp = (g.c + per16 - 1) / per16 * per16;
  P.cast_i = I->dtype == NK_F32;
  if (P.cast_i && !(g.sin_w == g.c && g.sin_h == (int64_t)g.w * g.c && g.sin_n == (int64_t)g.h * g.w * g.c))
    return fail(NK_ERR_UNSUPPORTED, "an FP32 conv input must be contiguous NHWC for the tensor-core path");
  size_t off = 0;
  if (P.cast_i) { P.off_i = off; off += align_up((size_t)g.n * g.h * g.w * P.Cp * esz); }
  P.cast_w = W->dtype == NK_F32;
  if (P.cast_w) { P.off_w = off; off += align_up((size_t)F * g.kh * g.kw * P.Cp * esz); }
  if (P.kind == TC_FP8 && P.cast_i) {   // per-call quantisation
    P.off_scal = off; off += kAlign;                      // amax_i, amax_w, s_i, s_w
    P.off_amax = off; off += align_up(prep_amax_ws(0));
  }
  TcConv c{};
  c.kind = P.kind; c.g = g; c.F = F;
  P.kern = tc_conv_ws(c, S);
  P.off_k = off; off += align_up(P.kern);
  P.total = off;
  return NK_OK;
}

// FP32 HWCF weights [taps*C, F] -> [F][taps][ldw] (ldw >= C with 16-byte
// rows): one transposing cast when ldw == C, else one per tap.  ck: 0 BF16,
// 1 E4M3 scaled by 448 / *amax (the scale written to *scale_out).
static nk_status pack_weights(int ck, const float* Wf, int taps, int C, int F, int64_t ldw, void* out,
                              const float* amax, float* scale_out, cudaStream_t st, const EwProg* pro = nullptr) {
  char* wt = static_cast<char*>(out);
  const int esz = ck == 1 ? 1 : 2;
  if (ldw == C)
    return prep_cast(ck, Wf, (int64_t)taps * C, F, F, amax, wt, nullptr, (int64_t)taps * C, 1, scale_out, st, pro);
  for (int tap = 0; tap < taps; ++tap) {
    const EwProg sp = pro ? ew_shift(*pro, (int64_t)tap * C * F) : EwProg{};
    nk_status s = prep_cast(ck, Wf + (int64_t)tap * C * F, C, F, F, amax, wt + (size_t)tap * ldw * esz, nullptr,
                            (int64_t)taps * ldw, 1, scale_out, st, &sp);
    if (s != NK_OK) return s;
  }
  return NK_OK;
}

static bool o_dense(const nk_tensor* O) {
  return O->stride[2] == O->shape[3] && O->stride[1] == O->shape[2] * O->stride[2] &&
         O->stride[0] == O->shape[1] * O->stride[1];
}

nk_status nk_conv2d_workspace_size(const nk_tensor* I, const nk_tensor* W, const nk_tensor* O,
                                   const int64_t stride[2], const int64_t dilation[2],
                                   const int64_t pad[4], int32_t precision,
                                   const nk_schedule* sched, size_t* bytes) {
  if (!bytes) return fail(NK_ERR_INVALID_ARG, "bytes is NULL");
  ConvGeom g;
  nk_status s = plan_conv(I, W, O, stride, dilation, pad, g);
  if (s != NK_OK) return s;
  const int M = g.n * g.oh * g.ow, N = (int)W->shape[3];
  if (precision == NK_PREC_BF16 || precision == NK_PREC_FP8) {
    ConvPlan P;
    if ((s = plan_tc_conv(I, W, O, g, precision, sched, P)) != NK_OK) return s;
    *bytes = P.total;
    return NK_OK;
  }
  if (precision != NK_PREC_F32) return fail(NK_ERR_UNSUPPORTED, "conv precision %d not available", precision);
  const int split = sched && sched->split_k > 0 ? sched->split_k : 1;
  *bytes = simt_gemm_ws(M, N, split);
  return NK_OK;
}

nk_status nk_conv2d_nhwc_hwcf(const nk_tensor* I, const nk_tensor* W, nk_tensor* O,
                              const int64_t stride[2], const int64_t dilation[2],
                              const int64_t pad[4], int32_t precision, const nk_epilogue* epi,
                              const nk_schedule* sched, void* ws, size_t ws_bytes, void* stream) {
  nk::NvtxRange nvtx_range_("nk_conv2d_nhwc_hwcf");
  ConvGeom g;
  nk_status s = plan_conv(I, W, O, stride, dilation, pad, g);
  if (s != NK_OK) return s;
  const nk_epilogue e0{nullptr, 0, 0, 1.f, 1.f, nullptr, nullptr, nullptr};
  const nk_epilogue& E = epi ? *epi : e0;
  if (!o_dense(O)) return fail(NK_ERR_UNSUPPORTED, "O must be contiguous NHWC");
  EwProg ew, pro_i, pro_w;
  if ((s = ew_program(E.ew, O, &ew, "ew")) != NK_OK) return s;
  if ((s = ew_program(E.pro_a, I, &pro_i, "pro_a (I)")) != NK_OK) return s;
  if ((s = ew_program(E.pro_b, W, &pro_w, "pro_b (W)")) != NK_OK) return s;
  if ((pro_i.n && I->dtype != NK_F32) || (pro_w.n && W->dtype != NK_F32))
    return fail(NK_ERR_UNSUPPORTED,
                "a prologue needs an FP32 operand (BF16 / E4M3 / packed operands are already converted)");
  if ((s = require_device()) != NK_OK) return s;
  if (precision == NK_PREC_BF16 || precision == NK_PREC_FP8) {
    ConvPlan P;
    if ((s = plan_tc_conv(I, W, O, g, precision, sched, P)) != NK_OK) return s;
    if (P.total > 0 && (!ws || ws_bytes < P.total))
      return fail(NK_ERR_WORKSPACE, "conv needs %zu bytes of workspace (got %zu)", P.total, ws_bytes);
    if (ws && !aligned16(ws)) return fail(NK_ERR_MISALIGNED, "workspace must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    const int F = (int)W->shape[3], taps = g.kh * g.kw;
    const int ck = P.kind == TC_FP8 ? 1 : 0;
    TcConv c{};
    c.kind = P.kind; c.g = g; c.F = F;
    // E4M3: per-tensor amax of I and W, then s = 448 / amax in the casts
    const bool prequant = P.kind == TC_FP8 && I->dtype == NK_F8E4M3;
    c.alpha = 1.f;
    if (prequant) {
      // the caller's scales: the result is multiplied by 1/(s_i s_w)
      if (!(E.scale_a > 0.f) || !(E.scale_b > 0.f) || !std::isfinite(E.scale_a) || !std::isfinite(E.scale_b))
        return fail(NK_ERR_INVALID_ARG, "pre-quantised E4M3 operands need positive finite scale_a (I), scale_b (W)");
      c.alpha = 1.f / (E.scale_a * E.scale_b);
    }
    float* scal = (P.kind == TC_FP8 && !prequant) ? reinterpret_cast<float*>(w + P.off_scal) : nullptr;
    if (P.kind == TC_FP8 && !prequant) {
      void* aw = w + P.off_amax;
      const size_t awb = prep_amax_ws(0);
      if ((s = prep_amax(static_cast<const float*>(I->ptr), (int64_t)g.n * g.h * g.w, g.c, g.c, scal + 0, aw, awb,
                         st, &pro_i)) != NK_OK)
        return s;
      if ((s = prep_amax(static_cast<const float*>(W->ptr), (int64_t)taps * g.c, F, F, scal + 1, aw, awb, st,
                         &pro_w)) != NK_OK)
        return s;
      c.scale_i = scal + 2;
      c.scale_w = scal + 3;
    }
    if (P.cast_i) {
      s = prep_cast(ck, static_cast<const float*>(I->ptr), (int64_t)g.n * g.h * g.w, g.c, g.c,
                    scal ? scal + 0 : nullptr, w + P.off_i, nullptr, P.Cp, 0, scal ? scal + 2 : nullptr, st, &pro_i);
      if (s != NK_OK) return s;
      c.I = w + P.off_i;
      c.sI_w = P.Cp; c.sI_h = (int64_t)g.w * P.Cp; c.sI_n = (int64_t)g.h * g.w * P.Cp;
    } else {
      c.I = I->ptr;
      c.sI_w = g.sin_w; c.sI_h = g.sin_h; c.sI_n = g.sin_n;
    }
    if (P.cast_w) {
      char* wt = w + P.off_w;
      if ((s = pack_weights(ck, static_cast<const float*>(W->ptr), g.kh * g.kw, g.c, F, P.Cp, wt,
                            scal ? scal + 1 : nullptr, scal ? scal + 3 : nullptr, st, &pro_w)) != NK_OK)
        return s;
      c.Wt = wt;
      c.ldw = P.Cp;
      c.sW_f = (int64_t)taps * P.Cp;
    } else {
      c.Wt = W->ptr;
      c.ldw = W->stride[1];
      c.sW_f = W->stride[3];
    }
    c.O = static_cast<float*>(O->ptr);
    c.out_bf16 = O->dtype == NK_BF16 ? 1 : 0;
    if (c.out_bf16 && (reinterpret_cast<uintptr_t>(O->ptr) & 1))
      return fail(NK_ERR_MISALIGNED, "a BF16 O must be 2-byte aligned");
    c.bias = E.bias;
    c.relu = E.relu;
    c.beta = E.accumulate ? 1.f : 0.f;
    c.ew = ew;
    return tc_conv(c, P.sched, w + P.off_k, P.kern, st);
  }
  if (precision != NK_PREC_F32 || I->dtype != NK_F32 || W->dtype != NK_F32)
    return fail(NK_ERR_UNSUPPORTED, "conv precision %d with I dtype %d / W dtype %d not available", precision,
                I->dtype, W->dtype);
  if (O->dtype != NK_F32) return fail(NK_ERR_UNSUPPORTED, "the FP32 convolution writes an FP32 O");
  SimtGemm p{};
  p.A = static_cast<const float*>(I->ptr);
  p.B = static_cast<const float*>(W->ptr);
  p.sbk = W->shape[3]; p.sbn = 1;
  p.C = static_cast<float*>(O->ptr); p.scm = O->shape[3]; p.scn = 1;
  p.bias = E.bias; p.bias_on_m = 0;
  p.M = g.n * g.oh * g.ow; p.N = (int)W->shape[3]; p.K = g.kh * g.kw * g.c;
  p.alpha = 1.f; p.beta = E.accumulate ? 1.f : 0.f; p.relu = E.relu;
  p.is_conv = 1; p.conv = g;
  p.ew = ew; p.pro_a = pro_i; p.pro_b = pro_w;
  int tile = sched && sched->tile_m > 0 ? sched->tile_m : 64;
  int split = sched && sched->split_k > 0 ? sched->split_k : 1;
  return simt_gemm(p, tile, split, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

nk_status nk_conv2d_pack_weights(const nk_tensor* W, void* Wp, int64_t ldw, void* stream) {
  nk::NvtxRange nvtx_range_("nk_conv2d_pack_weights");
  if (!W || !Wp) return fail(NK_ERR_INVALID_ARG, "W and Wp must be non-NULL");
  if (W->rank != 4 || W->dtype != NK_F32) return fail(NK_ERR_INVALID_ARG, "W must be a rank-4 FP32 tensor");
  if (W->stride[3] != 1 || W->stride[2] != W->shape[3] || W->stride[1] != W->shape[2] * W->shape[3] ||
      W->stride[0] != W->shape[1] * W->shape[2] * W->shape[3])
    return fail(NK_ERR_UNSUPPORTED, "W must be contiguous HWCF");
  for (int i = 0; i < 4; ++i)
    if (W->shape[i] < 1) return fail(NK_ERR_INVALID_ARG, "W extents must be positive");
  if (ldw < W->shape[2] || ldw % 8) return fail(NK_ERR_INVALID_ARG, "ldw must be >= C and a multiple of 8");
  if (!aligned16(Wp)) return fail(NK_ERR_MISALIGNED, "Wp must be 16-byte aligned");
  nk_status s = require_device();
  if (s != NK_OK) return s;
  return pack_weights(0, static_cast<const float*>(W->ptr), (int)(W->shape[0] * W->shape[1]), (int)W->shape[2],
                      (int)W->shape[3], ldw, Wp, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

nk_status nk_conv2d_pack_weights_fp8(const nk_tensor* W, void* Wp, int64_t ldw, float* scale, void* ws,
                                     size_t ws_bytes, void* stream) {
  nk::NvtxRange nvtx_range_("nk_conv2d_pack_weights_fp8");
  if (!W || !Wp || !scale) return fail(NK_ERR_INVALID_ARG, "W, Wp and scale must be non-NULL");
  if (W->rank != 4 || W->dtype != NK_F32) return fail(NK_ERR_INVALID_ARG, "W must be a rank-4 FP32 tensor");
  if (W->stride[3] != 1 || W->stride[2] != W->shape[3] || W->stride[1] != W->shape[2] * W->shape[3] ||
      W->stride[0] != W->shape[1] * W->shape[2] * W->shape[3])
    return fail(NK_ERR_UNSUPPORTED, "W must be contiguous HWCF");
  for (int i = 0; i < 4; ++i)
    if (W->shape[i] < 1) return fail(NK_ERR_INVALID_ARG, "W extents must be positive");
  if (ldw < W->shape[2] || ldw % 16) return fail(NK_ERR_INVALID_ARG, "ldw must be >= C and a multiple of 16");
  if (!aligned16(Wp)) return fail(NK_ERR_MISALIGNED, "Wp must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(scale) & 3) return fail(NK_ERR_MISALIGNED, "scale must be 4-byte aligned");
  const int taps = (int)(W->shape[0] * W->shape[1]), C = (int)W->shape[2], F = (int)W->shape[3];
  const size_t need = align_up(prep_amax_ws((int64_t)taps * C * F)) + kAlign;
  if (!ws || ws_bytes < need) return fail(NK_ERR_WORKSPACE, "packing needs %zu bytes of workspace", need);
  if (!aligned16(ws)) return fail(NK_ERR_MISALIGNED, "workspace must be 16-byte aligned");
  nk_status s = require_device();
  if (s != NK_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* amax = reinterpret_cast<float*>(static_cast<char*>(ws) + align_up(prep_amax_ws(0)));
  const float* Wf = static_cast<const float*>(W->ptr);
  if ((s = prep_amax(Wf, (int64_t)taps * C, F, F, amax, ws, prep_amax_ws(0), st)) != NK_OK) return s;
  return pack_weights(1, Wf, taps, C, F, ldw, Wp, amax, scale, st);
}

size_t nk_conv2d_pack_weights_fp8_workspace_size(void) { return align_up(prep_amax_ws(0)) + kAlign; }

// ------------------------------------------------------------- elementwise
nk_status nk_elementwise(const nk_tensor* X, nk_tensor* Y, const nk_ew_program* prog, void* stream) {
  nk::NvtxRange nvtx_range_("nk_elementwise");
  if (!X || !Y) return fail(NK_ERR_INVALID_ARG, "X and Y must be non-NULL");
  if (X->rank < 1 || X->rank > 4 || Y->rank != X->rank)
    return fail(NK_ERR_INVALID_ARG, "X and Y need the same rank, 1..4");
  if (X->dtype != NK_F32 || Y->dtype != NK_F32) return fail(NK_ERR_UNSUPPORTED, "X and Y must be FP32");
  int64_t n = 1;
  for (int d = 0; d < X->rank; ++d) {
    if (X->shape[d] < 0 || X->shape[d] != Y->shape[d])
      return fail(NK_ERR_INVALID_ARG, "X and Y shapes differ (dim %d)", d);
    n *= X->shape[d];
  }
  if (n > 0 && (!X->ptr || !Y->ptr)) return fail(NK_ERR_INVALID_ARG, "NULL data pointer");
  if (((reinterpret_cast<uintptr_t>(X->ptr) | reinterpret_cast<uintptr_t>(Y->ptr)) & 3))
    return fail(NK_ERR_INVALID_ARG, "X and Y must be 4-byte aligned");
  EwProg e;
  nk_status s = ew_program(prog, Y, &e, "prog");
  if (s != NK_OK) return s;
  if ((s = require_device()) != NK_OK) return s;
  return ew_tensor(static_cast<const float*>(X->ptr), X->stride, static_cast<float*>(Y->ptr), Y->stride, Y->shape,
                   Y->rank, e, static_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------- operand prep
size_t nk_prep_workspace_size(int64_t n) { return prep_amax_ws(n); }

nk_status nk_amax(const float* x, int64_t n, float* amax, void* ws, size_t ws_bytes, void* stream) {
  nk::NvtxRange nvtx_range_("nk_amax");
  nk_status s = require_device();
  if (s != NK_OK) return s;
  if (n < 0) return fail(NK_ERR_INVALID_ARG, "negative length");
  return prep_amax(x, 1, n, n, amax, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

static nk_status check_cast(const float* in, int64_t rows, int64_t cols, int64_t ld_in, const void* out,
                            int64_t ld_out, int transpose) {
  if (rows < 0 || cols < 0) return fail(NK_ERR_INVALID_ARG, "negative extent");
  if (rows * cols == 0) return NK_OK;
  if (!in || !out) return fail(NK_ERR_INVALID_ARG, "null pointer");
  if (ld_in < cols) return fail(NK_ERR_INVALID_ARG, "ld_in < cols");
  if (ld_out < (transpose ? rows : cols)) return fail(NK_ERR_INVALID_ARG, "ld_out too small");
  return NK_OK;
}

nk_status nk_cast_bf16(const float* in, int64_t rows, int64_t cols, int64_t ld_in, void* out,
                       int64_t ld_out, int32_t transpose, void* stream) {
  nk::NvtxRange nvtx_range_("nk_cast_bf16");
  nk_status s = check_cast(in, rows, cols, ld_in, out, ld_out, transpose);
  if (s != NK_OK) return s;
  return prep_cast(0, in, rows, cols, ld_in, nullptr, out, nullptr, ld_out, transpose, nullptr,
                   static_cast<cudaStream_t>(stream));
}

nk_status nk_cast_fp8(const float* in, int64_t rows, int64_t cols, int64_t ld_in, const float* amax,
                      void* out, int64_t ld_out, int32_t transpose, float* scale_out, void* stream) {
  nk::NvtxRange nvtx_range_("nk_cast_fp8");
  nk_status s = check_cast(in, rows, cols, ld_in, out, ld_out, transpose);
  if (s != NK_OK) return s;
  if (!amax) return fail(NK_ERR_INVALID_ARG, "amax is NULL");
  return prep_cast(1, in, rows, cols, ld_in, amax, out, nullptr, ld_out, transpose, scale_out,
                   static_cast<cudaStream_t>(stream));
}

nk_status nk_split_bf16x3(const float* in, int64_t rows, int64_t cols, int64_t ld_in, void* hi,
                          void* lo, int64_t ld_out, int32_t transpose, void* stream) {
  nk::NvtxRange nvtx_range_("nk_split_bf16x3");
  nk_status s = check_cast(in, rows, cols, ld_in, hi, ld_out, transpose);
  if (s != NK_OK) return s;
  if (!lo && rows * cols) return fail(NK_ERR_INVALID_ARG, "lo is NULL");
  return prep_cast(2, in, rows, cols, ld_in, nullptr, hi, lo, ld_out, transpose, nullptr,
                   static_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------ validation
size_t nk_norm_workspace_size(int64_t M, int64_t N) { return norm_ws(M, N); }

nk_status nk_rel_frobenius(const float* C, int64_t ldc, const double* R, int64_t ldr, int64_t M,
                           int64_t N, double* sumsq, void* ws, size_t ws_bytes, void* stream) {
  nk::NvtxRange nvtx_range_("nk_rel_frobenius");
  nk_status s = require_device();
  if (s != NK_OK) return s;
  if (M < 0 || N < 0) return fail(NK_ERR_INVALID_ARG, "negative extent");
  if (!sumsq || (M * N > 0 && (!C || !R))) return fail(NK_ERR_INVALID_ARG, "null pointer");
  if (ldc < N || ldr < N) return fail(NK_ERR_INVALID_ARG, "leading dimension smaller than N");
  return norm_sumsq(C, ldc, R, ldr, M, N, sumsq, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

