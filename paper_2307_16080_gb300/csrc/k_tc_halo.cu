// k_tc_halo.cu -- stride-1 linalg.conv_2d_nhwc_hwcf on the tensor cores from
// one shared input window per tile.
//
// O[n,oh,ow,f] = sum_{kh,kw,c} I[n, oh+kh*dh-pt, ow+kw*dw-pl, c] W[kh,kw,c,f]
// (Sec. 4.1, the conv loop nest, here in NHWC/HWCF with dilation and zero
// padding).  As an implicit GEMM, filter tap (kh, kw) reads the input pixels
// under the output tile shifted by (kh*dh, kw*dw).  With stride 1 those
// shifted views nearly coincide: an output tile of R rows x Q columns only
// ever reads a window of WR = R + (KH-1)*dh input rows by P = Q + (KW-1)*dw
// input columns.  That window is brought into shared memory once per
// 64-channel block by one 4-D TMA box -- one 128-byte swizzled row per input
// pixel, P pixels per window row -- and all KH*KW taps read it in place.
//
// Row m of the tile's GEMM is window pixel m, i.e. output (y, x) of image b
// is m = (b*WR + y)*P + x; the P - Q columns x >= Q of each row (and the
// KH-1 halo rows after each image) are computed and discarded.  Tap (kh, kw)
// is then the same window starting kh*dh*P + kw*dw rows later, which is just
// a later start address in the MMA's shared-memory descriptor: the 128B
// swizzle is a function of the address bits (each row keeps its phase), so a
// start on any 128-byte row is valid.  The tap-by-tap path reloads a shifted
// box per tap, KH*KW loads of nearly the same pixels.
//
// MCH stacked 128-row accumulator chains cover one window of up to
// MCH*128 GEMM rows and share every weight tile.  The filter tiles
// ([F][taps][C], K-major) stream through their own ring, or stay resident
// for the whole launch when one N tile holds all filters and they fit.
//
// Stacked kernel rows (schedule tile_k = 64*KH): the KW taps of one kernel
// row go side by side along N.  Each weight tile holds KW boxes of 64
// filters, so one MMA of N = 64*KW reads the window once at kernel row kh's
// offset kh*dh*P and yields every tap of that row.  Accumulator column
// kw*64 + f of GEMM row m is then tap kw's partial sum for output row
// m - kw*dw.  The epilogue adds them with warp shuffles: lane l takes lane
// l + kw*dw.  Window rows have a pitch P of 8, 16 or 32, so they sit inside
// one warp and a valid output never reads across a warp.  That makes KH MMAs
// per 16 channels instead of KH*KW narrow ones.
//
// When one column tile spans the output width and P >= W + pad_left, a
// stacked tile may hold Q = OW columns: a shift past the window row then
// stands for right padding and the epilogue leaves it out (whole-width
// tiles; a 7-wide image fits a pitch of 8).
//
// Variants (template parameters): DB, two accumulators and eight epilogue
// warps on one CTA per SM, so a tile's epilogue overlaps the next tile;
// F8, E4M3 operands in 128-channel blocks (kind::f8f6f4, K = 32 per MMA);
// RES, the residual ADD + ReLU inline in the store path.  Outputs are FP32
// or BF16 (rounded once after the whole epilogue).
//
//   warp 0      TMA producer: window slots (one per channel block: 64 BF16
//               or 128 E4M3 channels) and weight tiles (one per tap, or per
//               kernel row when stacked, and channel block).
//   warp 1      TMEM allocation; one thread issues tcgen05.mma, M = 128,
//               N = BN (stacked: 64*KW), K = 16 (E4M3: 32), MCH chains x 4 K
//               steps per tap.
//   warps 2..   epilogue (4 warps, 8 for DB): tcgen05.ld, the tap shuffles
//               when stacked, bias, beta*O, ReLU, the residual, FP32 or BF16
//               stores of the valid rows; with two accumulator buffers
//               overlapped with the next tile's MMAs.
//
// Every wait is bounded (tc_ptx.cuh); on expiry the CTA drains its copies and
// MMAs, frees TMEM and exits, and the host reports NK_ERR_TIMEOUT.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <vector>

#include "nk_internal.cuh"
#include "tc_ptx.cuh"

namespace nk {

__device__ unsigned int g_halo_err;

uint32_t halo_read_and_clear_errors() {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_halo_err, sizeof v) != cudaSuccess) return 0;
  const unsigned int z = 0;
  cudaMemcpyToSymbol(g_halo_err, &z, sizeof z);
  return v;
}

namespace {

constexpr int kThreads = 192;       // producer, MMA issuer, 4 epilogue warps
constexpr int kThreadsDB = 320;     // double-buffered stacked kernel: 8 epilogue warps
constexpr int kRow = 128;            // bytes per pixel row (64 BF16 channels) / per filter row
constexpr int kMaxSmem = 232448;     // 227 KB opt-in limit
constexpr int kBarBytes = 1024;      // barriers (at most 127), TMEM slot and abort flag

struct HaloTile {
  int Q, R, NB;          // output columns, rows and images of a tile
  int P, WR;             // window row pitch (pixels) and window rows per image
  int rows;              // pixels one window box writes: NB * WR * P
  int slot_rows;         // rows reserved per window slot (>= rows and >= the last row any tap reads)
  int tiles_w, tiles_h, tiles_b;
  int N, OH, OW, KH, KW, dh, dw, pt, pl;
  int cblocks;           // channel blocks of one 128-byte row
  int cblk;              // channels per block: 64 BF16 or 128 E4M3
  int stk;               // taps side by side along N: KW when kernel rows are stacked, else 1
};

struct HaloParams {
  CUtensorMap tmI;       // 4-D input {C, W, H, N}, box {64, P, WR, NB}
  CUtensorMap tmW;       // 3-D filters {C, taps, F}, box {64, 1, BN}
  HaloTile t;
  int F, bn;
  int wslots, bslots;    // window ring depth, weight ring depth
  int resident;          // weights loaded once (bslots == taps * cblocks, one N tile)
  int tiles_m, tiles_n, units;
  uint32_t slot_bytes;   // bytes per window slot (1024-aligned)
  float* O;              // [N*OH*OW][F]
  const float* bias;
  int relu;
  float beta;
  int c_vec;             // 16-byte aligned output rows
  int c_vec32;           // 32-byte aligned output rows (one-sector stores)
  int resid;             // ew is the residual program {ADD t, RELU}, t with 32-byte aligned rows
  int64_t budget;
  EwProg ew;             // fused elementwise program (offsets from O)
  int out_bf16;          // O holds BF16 (RNE of the FP32 epilogue result)
  // E4M3 operands: the result is scaled by 1/(s_i s_w), from the device
  // scalars the per-call quantisation wrote (scale_i, scale_w) or, for
  // operands the caller quantised, from alpha
  float alpha;
  const float* scale_i;
  const float* scale_w;
};

// First GEMM row a tap reads: tap (kh, kw) sees the window kh*dh rows down
// and kw*dw columns right.
__device__ __forceinline__ int tap_offset(const HaloTile& t, int tap) {
  const int kh = tap / t.KW, kw = tap - kh * t.KW;
  return kh * t.dh * t.P + kw * t.dw;
}

// STK (kernel-row stacking, one chain): the KW taps of a kernel row sit side
// by side along N, so one MMA of N = 64 * KW per kernel row and 16 channels
// does the work of KW narrow ones.  Accumulator column kw * 64 + f of row m
// holds the tap-kw partial sum of output row m - kw * dw; the epilogue adds
// them with warp shuffles.  The window row pitch P divides 32, so a shifted
// row never leaves its warp.  One accumulator buffer (TMEM for two CTAs), or
// with DB two buffers in all 512 columns (one CTA per SM): the epilogue of a
// tile then overlaps the next tile's MMAs, and the CTA holds the filters
// once beside a deeper ring of window slots.  With one CTA per SM the
// epilogue is the longer half of a tile (a single warp per SM sub-partition
// runs its dependent loads, shuffles and stores with nothing to hide their
// latency), so DB gives it twice the warps: two per TMEM lane quarter, each
// taking every other 32-column segment.
//
// F8: E4M3 operands (stacked rows only): 128-channel K blocks, the same
// 128-byte rows and 32-byte K steps (tcgen05.mma kind::f8f6f4, K = 32), the
// result dequantised by 1/(s_i s_w) in the epilogue.
//
// RES: the output program is the residual ADD t, RELU, applied inline in the
// fast store path.  A separate instantiation, because the residual loads
// raised the double-buffered kernel to spilling registers, which slowed
// every layer without a residual by ~15 %.
template <int MCH, bool STK, bool DB = false, bool F8 = false, bool RES = false>
__global__ void __launch_bounds__(DB ? kThreadsDB : kThreads, 1) halo_conv_kernel(const __grid_constant__ HaloParams p) {
  static_assert(!STK || MCH == 1, "stacked kernel rows use one chain");
  static_assert(!DB || STK, "the double-buffered variant is a stacked-row kernel");
  static_assert(!F8 || STK, "E4M3 window convolutions stack kernel rows");
  static_assert(!RES || (STK && !F8), "the inline residual serves the BF16 stacked kernels");
  constexpr int NACC = (STK && !DB) ? 1 : 2;   // accumulator buffers
  constexpr int EPW = DB ? 2 : 1;              // epilogue warps per TMEM lane quarter
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = ptx::smem_u32(smem_raw);
  const uint32_t base = (raw + 1023) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);
  const HaloTile& t = p.t;
  const int WS = p.wslots, BS = p.bslots;
  const int nst = STK ? t.KW : 1;                                // taps side by side along N
  const int kgroups = STK ? t.KH : t.KH * t.KW;                  // K blocks per 64-channel block
  const uint32_t wbase = base;                                   // window slots
  const uint32_t bbase = wbase + (uint32_t)WS * p.slot_bytes;    // weight slots
  const uint32_t b_tile = (uint32_t)(p.bn * nst) * kRow;
  const uint32_t bar0 = bbase + (uint32_t)BS * b_tile;
  auto wfull = [&](int s) { return bar0 + 8u * s; };
  auto wempty = [&](int s) { return bar0 + 8u * (WS + s); };
  auto bfull = [&](int s) { return bar0 + 8u * (2 * WS + s); };
  auto bempty = [&](int s) { return bar0 + 8u * (2 * WS + BS + s); };
  auto tfull = [&](int b) { return bar0 + 8u * (2 * WS + 2 * BS + b); };
  auto tempty = [&](int b) { return bar0 + 8u * (2 * WS + 2 * BS + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * WS + 2 * BS + 4);
  const uint32_t nbars = (uint32_t)(2 * WS + 2 * BS + 5);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + (bar0 - base) + 8u * nbars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  {
    // The launch must have given this layout enough dynamic shared memory.
    uint32_t dsz;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsz));
    const uint32_t need = (bar0 - raw) + 8u * nbars + 8u;
    if (need > dsz || 8u * nbars + 8u > (uint32_t)kBarBytes) {
      if (threadIdx.x == 0) atomicOr(&g_halo_err, 2u);
      return;
    }
  }
  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  const uint32_t acc_cols = (uint32_t)(MCH * p.bn * nst);
  // 128, 256 or 512 columns: a power of two >= 32 (stacked: 64 * KW rounded
  // up, or all 512 for two buffers)
  const uint32_t tmem_cols = STK ? (DB ? 512u : (acc_cols <= 128u ? 128u : 256u)) : 2u * acc_cols;

  if (threadIdx.x == 0) {
    for (int s = 0; s < WS; ++s) {
      ptx::mbar_init(wfull(s), 1);
      ptx::mbar_init(wempty(s), 1);
    }
    for (int s = 0; s < BS; ++s) {
      ptx::mbar_init(bfull(s), 1);
      ptx::mbar_init(bempty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(tfull(b), 1);
      ptx::mbar_init(tempty(b), 4 * EPW);   // one arrival per epilogue warp
    }
    ptx::mbar_init(drain_bar, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    ptx::tma_prefetch_desc(&p.tmI);
    ptx::tma_prefetch_desc(&p.tmW);
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), tmem_cols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // Set-up above touched no global data; everything below runs after the
  // earlier kernels on the stream have finished.
  nk::pdl_wait();
  nk::pdl_trigger();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int wc = 0, bc = 0;   // window and weight copies issued
      bool ok = true;
      for (int u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
        const int tn = u / p.tiles_m, tm = u - tn * p.tiles_m;
        const int tw = tm % t.tiles_w, th = (tm / t.tiles_w) % t.tiles_h, tb = tm / (t.tiles_w * t.tiles_h);
        const bool load_w = !p.resident || u == (int)blockIdx.x;
        for (int cb = 0; cb < t.cblocks && ok; ++cb) {
          {
            const int s = wc % WS;
            const uint32_t ph = (uint32_t)(wc / WS) & 1u;
            if (!ptx::mbar_wait(wempty(s), ph ^ 1u, p.budget, abort_flag, &g_halo_err)) { ok = false; break; }
            ptx::mbar_arrive_expect_tx(wfull(s), (uint32_t)t.rows * kRow);
            ptx::tma_load_4d(wbase + (uint32_t)s * p.slot_bytes, &p.tmI, wfull(s), cb * t.cblk, tw * t.Q - t.pl,
                             th * t.R - t.pt, tb * t.NB);
            ++wc;
          }
          if (!load_w) continue;
          for (int kg = 0; kg < kgroups; ++kg) {
            const int s = bc % BS;
            const uint32_t ph = (uint32_t)(bc / BS) & 1u;
            if (!ptx::mbar_wait(bempty(s), ph ^ 1u, p.budget, abort_flag, &g_halo_err)) { ok = false; break; }
            ptx::mbar_arrive_expect_tx(bfull(s), b_tile);
            // one box of bn filters per tap; stacked: the KW taps of kernel row kg
            for (int j = 0; j < nst; ++j)
              ptx::tma_load_3d(bbase + (uint32_t)s * b_tile + (uint32_t)(j * p.bn) * kRow, &p.tmW, bfull(s), cb * t.cblk,
                               kg * nst + j, tn * p.bn);
            ++bc;
          }
        }
      }
      // Drain: the last copy issued into each slot lands before exit.
      for (int j = wc - 1; j >= 0 && j >= wc - WS; --j)
        ptx::mbar_drain(wfull(j % WS), (uint32_t)(j / WS) & 1u, 100000000ull);
      for (int j = bc - 1; j >= 0 && j >= bc - BS; --j)
        ptx::mbar_drain(bfull(j % BS), (uint32_t)(j / BS) & 1u, 100000000ull);
    }
  } else if (warp == 1) {
    // -------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t idesc = ptx::make_idesc(F8 ? 0 : 1, 128, p.bn * nst);
      int wc = 0, bc = 0, tc = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < p.units && ok; u += gridDim.x, ++tc) {
        const int acc = tc % NACC;
        const uint32_t aph = (uint32_t)(tc / NACC) & 1u;
        if (!ptx::mbar_wait(tempty(acc), aph ^ 1u, p.budget, abort_flag, &g_halo_err)) break;
        ptx::tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)acc * acc_cols;
        for (int cb = 0; cb < t.cblocks && ok; ++cb) {
          const int ws = wc % WS;
          if (!ptx::mbar_wait(wfull(ws), (uint32_t)(wc / WS) & 1u, p.budget, abort_flag, &g_halo_err)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t win = wbase + (uint32_t)ws * p.slot_bytes;
          for (int kg = 0; kg < kgroups; ++kg) {
            // resident weights: slot = K block, phase 0 completed once and stays so
            const int kb = cb * kgroups + kg;
            const int bs = p.resident ? kb : bc % BS;
            const uint32_t bph = p.resident ? 0u : (uint32_t)(bc / BS) & 1u;
            if (!ptx::mbar_wait(bfull(bs), bph, p.budget, abort_flag, &g_halo_err)) { ok = false; break; }
            ptx::tc_fence_after();
            // stacked: kernel row kg starts kg * dh window rows down (the kw
            // shifts are applied in the epilogue); else tap kg's offset
            const uint32_t a0 = win + (uint32_t)(STK ? kg * t.dh * t.P : tap_offset(t, kg)) * kRow;
            const uint32_t b0 = bbase + (uint32_t)bs * b_tile;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint64_t bd = ptx::sw128_desc(b0 + 32u * k);
              const uint32_t accum = (kb > 0 || k > 0) ? 1u : 0u;
#pragma unroll
              for (int ch = 0; ch < MCH; ++ch)
                ptx::tc_mma<F8>(d + (uint32_t)(ch * p.bn), ptx::sw128_desc(a0 + (uint32_t)(ch * 128 * kRow) + 32u * k),
                               bd, idesc, accum);
            }
            if (!p.resident) {
              ptx::tc_commit(bempty(bs));
              ++bc;
            }
          }
          if (!ok) break;
          ptx::tc_commit(wempty(ws));
          ++wc;
        }
        if (!ok) break;
        ptx::tc_commit(tfull(acc));
      }
      ptx::tc_commit(drain_bar);
      ptx::mbar_drain(drain_bar, 0, 100000000ull);
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;   // TMEM lane quarter this warp may read
    const int img_rows = t.WR * t.P;
    const int cfirst = ((warp - 2) / 4) * 32;     // this warp's first 32-column segment
    float alpha = 1.f;                            // E4M3: 1 / (s_i s_w)
    if constexpr (F8) alpha = p.scale_i ? __frcp_rn(__fmul_rn(*p.scale_i, *p.scale_w)) : p.alpha;
    int tc = 0;
    for (int u = blockIdx.x; u < p.units; u += gridDim.x, ++tc) {
      const int tn = u / p.tiles_m, tm = u - tn * p.tiles_m;
      const int tw = tm % t.tiles_w, th = (tm / t.tiles_w) % t.tiles_h, tb = tm / (t.tiles_w * t.tiles_h);
      const int acc = tc % NACC;
      if (!ptx::mbar_wait(tfull(acc), (uint32_t)(tc / NACC) & 1u, p.budget, abort_flag, &g_halo_err)) break;
      ptx::tc_fence_after();
      for (int ch = 0; ch < MCH; ++ch) {
        // GEMM row m = window pixel (b, y, x); valid when it is an output pixel
        const int m = ch * 128 + q * 32 + lane;
        const int b = m / img_rows, r = m - b * img_rows;
        const int y = r / t.P, x = r - y * t.P;
        const int n = tb * t.NB + b, oh = th * t.R + y, ow = tw * t.Q + x;
        const bool row_ok = b < t.NB && y < t.R && x < t.Q && n < t.N && oh < t.OH && ow < t.OW;
        const int64_t orow_off = ((int64_t)(n * t.OH + oh) * t.OW + ow) * p.F;
        float* orow = p.O + orow_off;
        for (int c0 = cfirst; c0 < p.bn; c0 += 32 * EPW) {
          float v[32];
          const uint32_t lane_base = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)acc * acc_cols;
          if constexpr (DB) {
            // every tap's columns in flight before one wait, then the shifts
            // (the one-buffer variant keeps one tap in flight: its register
            // budget must leave room for two CTAs per SM)
            uint32_t r0[32], rt[3][32];
            ptx::tmem_ld32_async(lane_base + (uint32_t)c0, r0);
#pragma unroll
            for (int j = 1; j < 4; ++j)
              if (j < nst) ptx::tmem_ld32_async(lane_base + (uint32_t)(j * p.bn + c0), rt[j - 1]);
            ptx::tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = __uint_as_float(r0[e]);
#pragma unroll
            // (double-buffered tiles never use whole-width pitches: every
            // shift stays inside its window row)
            for (int j = 1; j < 4; ++j) {
              if (j >= nst) break;
              const int sh = j * t.dw;
#pragma unroll
              for (int e = 0; e < 32; ++e) v[e] += __shfl_down_sync(0xffffffffu, __uint_as_float(rt[j - 1][e]), sh);
            }
          } else {
          ptx::tmem_ld32(lane_base + (uint32_t)(ch * p.bn + c0), v);
          if (STK) {
            // output row m = tap-0 row m + tap-kw row m + kw * dw, same warp;
            // a shift past the window row (whole-width tiles only) reads
            // right padding and adds nothing
            for (int j = 1; j < nst; ++j) {
              float w[32];
              ptx::tmem_ld32(lane_base + (uint32_t)(j * p.bn + c0), w);
              const int sh = j * t.dw;
              const bool in_row = x + sh < t.P;
#pragma unroll
              for (int e = 0; e < 32; ++e) {
                const float s = __shfl_down_sync(0xffffffffu, w[e], sh);
                if (in_row) v[e] += s;
              }
            }
          }
          }
          if constexpr (F8) {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] *= alpha;
          }
          const int col0 = tn * p.bn + c0;
          if (!row_ok || col0 >= p.F) continue;
          if (p.c_vec32 && p.beta == 0.f && col0 + 32 <= p.F && (RES || p.ew.n == 0)) {
            // Full 32-column segment, no accumulate, and no program or the
            // residual program ADD t, RELU (inline, same FP32 steps as the
            // interpreter): one code path for FP32 and BF16 outputs.
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              float xv = v[j];
              if (p.bias) xv += __ldg(p.bias + col0 + j);
              if (p.relu) xv = (xv > 0.f || xv != xv) ? xv : 0.f;
              v[j] = xv;
            }
            if constexpr (RES) {
              const float4* tr = reinterpret_cast<const float4*>(p.ew.t[0] + orow_off + col0);
#pragma unroll
              for (int j = 0; j < 32; j += 4) {
                const float4 r4 = __ldg(tr + j / 4);
                const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const float xv = __fadd_rn(v[j + e], rv[e]);
                  v[j + e] = (xv > 0.f || xv != xv) ? xv : 0.f;
                }
              }
            }
            if (p.out_bf16) store32_bf16_v8(reinterpret_cast<__nv_bfloat16*>(p.O) + orow_off + col0, v);
            else store32_f32_v8(orow + col0, v);
            continue;
          }
          if (p.out_bf16) {
            // BF16 output: the FP32 epilogue, then one RNE rounding per value
            __nv_bfloat16* dh = reinterpret_cast<__nv_bfloat16*>(p.O) + orow_off + col0;
            const int ncol = p.F - col0 < 32 ? p.F - col0 : 32;
            if (p.ew.n) {
              // the program runs out of line on a local buffer (see below)
              float buf[32];
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                float xv = v[j];
                if (j < ncol) {
                  if (p.beta != 0.f) xv = fmaf(p.beta, __bfloat162float(dh[j]), xv);
                  if (p.bias) xv += __ldg(p.bias + col0 + j);
                  if (p.relu) xv = (xv > 0.f || xv != xv) ? xv : 0.f;
                }
                buf[j] = xv;
              }
              ew_apply(p.ew, buf, ncol, orow_off + col0);
              for (int j = 0; j < ncol; ++j) dh[j] = __float2bfloat16_rn(buf[j]);
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                float xv = v[j];
                if (col0 + j < p.F) {
                  if (p.beta != 0.f) xv = fmaf(p.beta, __bfloat162float(dh[j]), xv);
                  if (p.bias) xv += __ldg(p.bias + col0 + j);
                  if (p.relu) xv = (xv > 0.f || xv != xv) ? xv : 0.f;
                }
                v[j] = xv;
              }
              if (p.c_vec32 && ncol == 32) {
                store32_bf16_v8(dh, v);
              } else if (p.c_vec && ncol == 32) {
                store32_bf16(dh, v);
              } else {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                  if (j < ncol) dh[j] = __float2bfloat16_rn(v[j]);
              }
            }
            continue;
          }
          float* dst = orow + col0;
          if (p.ew.n) {
            // A program runs out of line: the segment goes through a local
            // buffer so the program reads its operands (which may alias O)
            // before the store and v[] is not live across the call.
            const int ncol = p.F - col0 < 32 ? p.F - col0 : 32;
            float buf[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              float xv = v[j];
              if (j < ncol) {
                if (p.beta != 0.f) xv = fmaf(p.beta, dst[j], xv);
                if (p.bias) xv += __ldg(p.bias + col0 + j);
                if (p.relu) xv = (xv > 0.f || xv != xv) ? xv : 0.f;
              }
              buf[j] = xv;
            }
            ew_apply(p.ew, buf, ncol, orow_off + col0);
            for (int j = 0; j < ncol; ++j) dst[j] = buf[j];
          } else if (p.c_vec32 && p.beta == 0.f && col0 + 32 <= p.F) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              float xv = v[j];
              if (p.bias) xv += __ldg(p.bias + col0 + j);
              if (p.relu) xv = (xv > 0.f || xv != xv) ? xv : 0.f;
              v[j] = xv;
            }
            store32_f32_v8(dst, v);
          } else if (p.c_vec && col0 + 32 <= p.F) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              float o[4];
              float4 cin = make_float4(0.f, 0.f, 0.f, 0.f);
              if (p.beta != 0.f) cin = *reinterpret_cast<const float4*>(dst + j);
              const float ci[4] = {cin.x, cin.y, cin.z, cin.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                float xv = v[j + e];
                if (p.beta != 0.f) xv = fmaf(p.beta, ci[e], xv);
                if (p.bias) xv += __ldg(p.bias + col0 + j + e);
                if (p.relu) xv = (xv > 0.f || xv != xv) ? xv : 0.f;
                o[e] = xv;
              }
              *reinterpret_cast<float4*>(dst + j) = make_float4(o[0], o[1], o[2], o[3]);
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (col0 + j >= p.F) continue;
              float xv = v[j];
              if (p.beta != 0.f) xv = fmaf(p.beta, dst[j], xv);
              if (p.bias) xv += __ldg(p.bias + col0 + j);
              if (p.relu) xv = (xv > 0.f || xv != xv) ? xv : 0.f;
              dst[j] = xv;
            }
          }
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(tempty(acc));
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc(tmem_base, tmem_cols);
}

// ------------------------------------------------------------------ host
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}

int taps_of(const ConvGeom& g) { return g.kh * g.kw; }

// Channels per K block: one 128-byte row, 64 BF16 or 128 E4M3.
int cblk_of(int kind) { return kind == TC_FP8 ? 128 : 64; }

// Kernel-row stacking: tile_k = cblk * KH (one K block per kernel row and
// channel block) selects the window kernel with the KW taps of a kernel row
// side by side along N (N = 64 * KW <= 256, so 2 <= KW <= 4).  Per-tap
// schedules have tile_k = cblk and plain window schedules 64 * KH * KW
// (BF16 only), so the encodings do not collide.
bool stacked_schedule(const ConvGeom& g, const nk_schedule& s, int kind = TC_BF16) {
  return g.kh >= 2 && g.kw >= 2 && g.kw <= 4 && s.tile_k == cblk_of(kind) * g.kh;
}

// Stacked kernel rows with tile_m 256: one 128-row tile at a time, but two
// accumulator buffers (all 512 TMEM columns, one CTA per SM) so the
// epilogue of a tile overlaps the MMAs of the next.
bool stacked_db(const ConvGeom& g, const nk_schedule& s, int kind = TC_BF16) {
  return stacked_schedule(g, s, kind) && s.tile_m == 256;
}

// Accumulator chains of a window schedule: tile_m / 128 stacked 128-row
// tiles for the plain window; stacked kernel rows always use one.
int chains_of(const ConvGeom& g, const nk_schedule& s, int kind = TC_BF16) {
  return stacked_schedule(g, s, kind) ? 1 : s.tile_m / 128;
}

// Largest row offset the A operand reads, in GEMM rows (stacked: the kw
// shifts move to the epilogue).
int max_offset(const ConvGeom& g, int P, bool stk) {
  return (g.kh - 1) * g.dh * P + (stk ? 0 : (g.kw - 1) * g.dw);
}

// TMEM columns one CTA allocates: two accumulator buffers of mch * bn, or
// (stacked) one buffer of 64 * KW rounded up to a power of two, or (stacked,
// double-buffered) all 512.
int halo_tmem_cols(int mch, int bn, int stk, bool db) {
  return stk > 1 ? (db ? 512 : (bn * stk <= 128 ? 128 : 256)) : 2 * mch * bn;
}

// Window tile for `mch` chains: the fewest tiles whose valid output rows
// all fall inside the first mch*128 GEMM rows; ties go to the smaller window.
// Returns false when no tile fits (box extents <= 256, slot within `max_slot_rows`).
// Stacked (stk > 1): the window row pitch P is 8, 16 or 32, so window rows
// are aligned to warps, and every row a valid output reads through the kw
// shifts (its whole window row) lies inside the first 128 GEMM rows.
//
// Stacked, one column tile: Q may be the whole output width OW <= P instead
// of P - (KW-1)*dw when P - pad_left >= W.  A tap whose shift would leave the
// window row (x + kw*dw >= P) then reads an input column >= W, which is zero
// padding, so the epilogue leaves it out and the sum is exact.  A 7-wide
// image fits a pitch of 8 this way (two images per tile instead of one).
// Only the single-buffered kernel masks those shifts (wrap_ok): in the
// double-buffered one the mask made the epilogue spill registers.
bool choose_halo_tile(const ConvGeom& g, int mch, int max_slot_rows, bool stk, bool wrap_ok, HaloTile* out) {
  const int maxrows = mch * 128;
  const int halo_w = (g.kw - 1) * g.dw, halo_h = (g.kh - 1) * g.dh;
  bool found = false;
  int64_t best_tiles = INT64_MAX;
  int best_slot = INT_MAX;
  HaloTile best{};
  // (Q, P) candidates: P = Q + halo_w, then (stacked) the whole-width tiles
  std::vector<std::pair<int, int>> qp;
  for (int Q = 1; (stk || Q <= g.ow) && Q + halo_w <= 256; ++Q) {
    const int P = Q + halo_w;
    if (Q > maxrows) break;
    if (stk && P != 8 && P != 16 && P != 32) {
      if (P > 32) break;
      continue;
    }
    qp.push_back({Q, P});
  }
  if (stk && wrap_ok)
    for (int P : {8, 16, 32})
      if (g.ow <= P && g.ow > P - halo_w && P - g.pl >= g.w) qp.push_back({g.ow, P});
  for (const auto& c : qp) {
    const int Q = c.first, P = c.second;
    const bool wrap = Q + halo_w > P;   // whole-width tile: chosen only for fewer tiles
    for (int R = 1; R <= g.oh && R + halo_h <= 256; ++R) {
      const int WR = R + halo_h;
      const int last = stk ? R * P : (R - 1) * P + Q;   // rows one image's outputs (and their reads) span
      if (last > maxrows) break;
      int NB = 1 + (maxrows - last) / (WR * P);
      NB = std::min(std::min(NB, g.n), 256);
      const int rows = NB * WR * P;
      const int slot = (std::max(rows, maxrows + max_offset(g, P, stk)) + 7) / 8 * 8;
      if (slot > max_slot_rows) continue;
      const int64_t tiles = (int64_t)((g.n + NB - 1) / NB) * ((g.oh + R - 1) / R) * ((g.ow + Q - 1) / Q);
      if (tiles < best_tiles || (!wrap && tiles == best_tiles && slot < best_slot)) {
        best_tiles = tiles;
        best_slot = slot;
        best.Q = Q; best.R = R; best.NB = NB; best.P = P; best.WR = WR;
        best.rows = rows; best.slot_rows = slot;
        found = true;
      }
    }
  }
  if (!found) return false;
  best.tiles_w = (g.ow + best.Q - 1) / best.Q;
  best.tiles_h = (g.oh + best.R - 1) / best.R;
  best.tiles_b = (g.n + best.NB - 1) / best.NB;
  best.N = g.n; best.OH = g.oh; best.OW = g.ow;
  best.KH = g.kh; best.KW = g.kw; best.dh = g.dh; best.dw = g.dw; best.pt = g.pt; best.pl = g.pl;
  best.cblocks = (g.c + 63) / 64;
  best.stk = stk ? g.kw : 1;
  *out = best;
  return true;
}

// The tile choice is a search over (Q, R); it is cached per geometry so a
// repeated call costs a lookup.
struct TileKey {
  ConvGeom g;
  int mch;
  int stk;
  int wrap_ok;
};
std::mutex g_tile_mu;
std::vector<std::pair<TileKey, std::pair<bool, HaloTile>>> g_tile_cache;

bool cached_halo_tile(const ConvGeom& g, int mch, bool stk, bool wrap_ok, HaloTile* out) {
  // The window slot may use at most what is left beside two weight tiles of
  // 256 rows and the barriers; the real budget is checked per schedule.
  const int max_slot_rows = (kMaxSmem - 1024 - kBarBytes) / kRow;
  std::lock_guard<std::mutex> lk(g_tile_mu);
  for (auto& e : g_tile_cache)
    if (e.first.mch == mch && e.first.stk == (int)stk && e.first.wrap_ok == (int)wrap_ok &&
        std::memcmp(&e.first.g, &g, sizeof g) == 0) {
      *out = e.second.second;
      return e.second.first;
    }
  HaloTile t{};
  const bool ok = choose_halo_tile(g, mch, max_slot_rows, stk, wrap_ok, &t);
  if (g_tile_cache.size() > 4096) g_tile_cache.clear();
  TileKey k;
  std::memset(&k, 0, sizeof k);
  k.g = g;
  k.mch = mch;
  k.stk = (int)stk;
  k.wrap_ok = (int)wrap_ok;
  g_tile_cache.push_back({k, {ok, t}});
  *out = t;
  return ok;
}

struct HaloLayout {
  HaloTile t;
  int wslots, bslots, resident;
  uint32_t slot_bytes;
  int smem;
};

// CTAs of this layout that fit on one SM: shared memory (each CTA also
// costs 1 KB of reserved space) and the TMEM columns each CTA allocates.
int halo_ctas(int smem, int tmem_cols) {
  const bool tmem2 = 2 * tmem_cols <= 512;
  return (tmem2 && 2 * (smem + 1024) <= kMaxSmem + 1024) ? 2 : 1;
}

// Shared-memory layout of a schedule: stages = window slots.  The weights
// stay resident when one N tile holds every filter and all K blocks fit;
// otherwise they stream through a ring of up to 8 tiles (at least two).  Of
// the two, the layout that lets more CTAs (independent MMA chains) share an
// SM wins; on a tie, resident weights.
bool halo_layout(const ConvGeom& g, int F, const nk_schedule& s, HaloLayout* L, int kind = TC_BF16, int sms = 0) {
  const int mch = chains_of(g, s, kind);
  const bool stk = stacked_schedule(g, s, kind);
  if (!cached_halo_tile(g, mch, stk, stk && !stacked_db(g, s, kind), &L->t)) return false;
  L->t.cblk = cblk_of(kind);
  L->t.cblocks = (g.c + L->t.cblk - 1) / L->t.cblk;
  const int tcols = halo_tmem_cols(mch, s.tile_n, L->t.stk, stacked_db(g, s, kind));
  L->slot_bytes = (uint32_t)((L->t.slot_rows * kRow + 1023) / 1024 * 1024);
  L->wslots = s.stages;
  const int fixed = 1024 + s.stages * (int)L->slot_bytes + kBarBytes;
  const int b_tile = s.tile_n * L->t.stk * kRow;   // stacked: KW boxes of tile_n filters
  const int nkb = (stk ? g.kh : taps_of(g)) * L->t.cblocks;
  const int room = (kMaxSmem - fixed) / b_tile;
  if (room < 2) return false;
  // streamed ring: deepest ring that keeps the CTA count of a 2-slot ring,
  // or (sms known, every unit in one wave of one CTA per SM) simply the
  // deepest: a lone CTA's MMA chain waits on its filter loads otherwise
  int ring = std::min(std::min(room, nkb < 2 ? 2 : nkb), 8);
  int want = halo_ctas(fixed + 2 * b_tile, tcols);
  if (sms > 0 && (int64_t)L->t.tiles_b * L->t.tiles_h * L->t.tiles_w * ((F + s.tile_n - 1) / s.tile_n) <= sms)
    want = 1;
  while (ring > 2 && halo_ctas(fixed + ring * b_tile, tcols) < want) --ring;
  L->resident = 0;
  L->bslots = ring;
  const bool one_n = (F + s.tile_n - 1) / s.tile_n == 1;
  if (one_n && room >= nkb && 8 * (2 * s.stages + 2 * nkb + 5) + 8 <= kBarBytes &&
      halo_ctas(fixed + nkb * b_tile, tcols) >= halo_ctas(fixed + ring * b_tile, tcols)) {
    L->resident = 1;
    L->bslots = nkb;
  }
  L->smem = fixed + L->bslots * b_tile;
  if (8 * (2 * L->wslots + 2 * L->bslots + 5) + 8 > kBarBytes) return false;
  return L->smem <= kMaxSmem;
}

template <int MCH, bool STK = false, bool DB = false, bool F8 = false, bool RES = false>
nk_status launch(const HaloParams& p, int grid, int smem, cudaStream_t st) {
  auto kern = halo_conv_kernel<MCH, STK, DB, F8, RES>;
  static int set_bytes[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || set_bytes[dev] < smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(halo_conv_kernel)");
    if (dev >= 0 && dev < 64) set_bytes[dev] = smem;
  }
  (void)nk::launch_k(kern, dim3(grid), dim3(DB ? kThreadsDB : kThreads), smem, st, 1, p);
  return check_launch("halo_conv_kernel");
}

}  // namespace

bool halo_schedule(const ConvGeom& g, const nk_schedule& s, int kind) {
  if (kind == TC_FP8) return stacked_schedule(g, s, kind);   // E4M3: stacked rows only
  return (taps_of(g) > 1 && s.tile_k == 64 * taps_of(g)) || stacked_schedule(g, s);
}

bool halo_schedule_valid(const ConvGeom& g, int F, const nk_schedule& s, int kind) {
  if (!halo_schedule(g, s, kind)) return false;
  if (g.sh != 1 || g.sw != 1) return false;
  if (s.tile_m != 128 && s.tile_m != 256 && s.tile_m != 512) return false;
  if (s.tile_n != 64 && s.tile_n != 128 && s.tile_n != 256) return false;
  if (chains_of(g, s, kind) * s.tile_n > 256) return false;   // two accumulator buffers in 512 TMEM columns
  // stacked: N = 64 * KW; tile_m 128 (one buffer) or 256 (two buffers)
  if (stacked_schedule(g, s, kind) && (s.tile_m > 256 || s.tile_n != 64)) return false;
  if (s.cluster != 1 || s.split_k != 1) return false;
  // window slots: up to 4, up to 8 beside the two buffers of one CTA per SM
  if (s.stages < 1 || s.stages > (stacked_db(g, s, kind) ? 8 : 4)) return false;
  HaloLayout L;
  return halo_layout(g, F, s, &L, kind);
}

// Host-side geometry of a window schedule (see nk_conv_window_tile).
bool halo_tile_info(const ConvGeom& g, int F, const nk_schedule& s, int32_t out[10], int kind) {
  HaloLayout L;
  if (!halo_schedule_valid(g, F, s, kind) || !halo_layout(g, F, s, &L, kind)) return false;
  const HaloTile& t = L.t;
  const int32_t v[10] = {t.P, t.Q, t.R, t.NB, t.WR, t.rows, t.slot_rows, t.stk,
                         t.tiles_w * t.tiles_h * t.tiles_b, chains_of(g, s, kind)};
  for (int i = 0; i < 10; ++i) out[i] = v[i];
  return true;
}

// Measured on GB300 (3x3 ResNet layers, batch 1..32, device time):
// stacked kernel rows beat the plain window and the per-tap kernels on
// every stride-1 layer from 56x56x64 to 7x7x512 (e.g. 8x28x28x128: 8.2 us
// against 14.6 (window) and 20.8 (per-tap); 8x56x56x64: 8.2 against 9.2),
// with one window slot when one 64-channel block covers C and two
// otherwise.  Small grids of deep layers are the exception: with C > 128
// and tiles covering under an eighth of the SMs (batch 1 at 14x14x256 and
// 7x7x512), the per-tap kernel with split-K is as fast or faster, so the
// default leaves them to it.  Where kernel rows cannot be stacked (KW = 1
// or > 4, e.g. 5x5), the tuner's corpus has the per-tap kernel ahead of the
// plain window (which stays in the schedule space).  One chain and one
// window slot keep two CTAs (two independent MMA chains) per SM.
nk_schedule tc_halo_default_schedule(const ConvGeom& g, int F, int sms, bool* ok, int kind) {
  nk_schedule best{};
  *ok = false;
  if (taps_of(g) <= 1 || g.sh != 1 || g.sw != 1) return best;
  // E4M3 reads 128 channels per K block: below C = 128 a window kernel
  // would fill half of every block with zeros, so the per-tap kernel keeps
  // those layers.
  if (kind == TC_FP8 && g.c < 128) return best;
  const int cb = cblk_of(kind);
  for (int st : {g.c <= cb ? 1 : 2, g.c <= cb ? 2 : 1}) {
    nk_schedule s{128, 64, cb * g.kh, 1, st, 1};
    HaloLayout L;
    if (!stacked_schedule(g, s, kind) || !halo_schedule_valid(g, F, s, kind) || !halo_layout(g, F, s, &L, kind))
      continue;
    const int64_t units = (int64_t)L.t.tiles_w * L.t.tiles_h * L.t.tiles_b * ((F + 63) / 64);
    if (g.c > 128 && units * 8 < sms) break;
    // With enough tiles that every CTA of the two-per-SM grid gets two or
    // more, two accumulator buffers on one CTA per SM overlap each tile's
    // epilogue with the next tile's MMAs: 16.0 against 17.4 us at
    // 32x56x56x64 (896 tiles); at 8x56x56x64 (224 tiles) one buffer stays
    // ahead, 8.0 against 8.3 us.
    const nk_schedule d{256, 64, cb * g.kh, 1, 2, 1};
    if (units >= 4 * (int64_t)sms && halo_schedule_valid(g, F, d, kind)) s = d;
    *ok = true;
    return s;
  }
  return best;
}

nk_status tc_halo_conv(const TcConv& c, const nk_schedule& s, cudaStream_t st) {
  int sms = 0;
  nk_status status = require_device(&sms);
  if (status != NK_OK) return status;
  const ConvGeom& g = c.g;
  const int kind = c.kind;
  const bool f8 = kind == TC_FP8;
  const int esz = f8 ? 1 : 2;
  HaloLayout L;
  if (!halo_schedule_valid(g, c.F, s, kind) || !halo_layout(g, c.F, s, &L, kind, sms))
    return fail(NK_ERR_NO_SCHEDULE, "illegal window-conv schedule");
  if ((c.sI_w * esz) % 16 || (c.sI_h * esz) % 16 || (c.sI_n * esz) % 16 || (c.ldw * esz) % 16 ||
      (c.sW_f * esz) % 16 || (reinterpret_cast<uintptr_t>(c.I) & 15) || (reinterpret_cast<uintptr_t>(c.Wt) & 15))
    return fail(NK_ERR_MISALIGNED, "conv operands need 16-byte aligned rows");
  const CUtensorMapDataType dt = f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  auto fn = encode_fn();
  if (!fn) return fail(NK_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  HaloParams p{};
  p.t = L.t;
  const HaloTile& t = L.t;
  {
    cuuint64_t dims[4] = {(cuuint64_t)g.c, (cuuint64_t)g.w, (cuuint64_t)g.h, (cuuint64_t)g.n};
    cuuint64_t strides[3] = {(cuuint64_t)c.sI_w * esz, (cuuint64_t)c.sI_h * esz, (cuuint64_t)c.sI_n * esz};
    cuuint32_t box[4] = {(cuuint32_t)t.cblk, (cuuint32_t)t.P, (cuuint32_t)t.WR, (cuuint32_t)t.NB};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(&p.tmI, dt, 4, const_cast<void*>(c.I), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(NK_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for the conv window", (int)r);
  }
  {
    const int taps = taps_of(g);
    cuuint64_t dims[3] = {(cuuint64_t)g.c, (cuuint64_t)taps, (cuuint64_t)c.F};
    cuuint64_t strides[2] = {(cuuint64_t)c.ldw * esz, (cuuint64_t)c.sW_f * esz};
    cuuint32_t box[3] = {(cuuint32_t)t.cblk, 1, (cuuint32_t)s.tile_n};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(&p.tmW, dt, 3, const_cast<void*>(c.Wt), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(NK_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for the conv filters", (int)r);
  }
  p.F = c.F;
  p.bn = s.tile_n;
  p.wslots = L.wslots;
  p.bslots = L.bslots;
  p.resident = L.resident;
  p.slot_bytes = L.slot_bytes;
  p.tiles_m = t.tiles_w * t.tiles_h * t.tiles_b;
  p.tiles_n = (c.F + s.tile_n - 1) / s.tile_n;
  p.units = p.tiles_m * p.tiles_n;
  p.O = c.O;
  p.bias = c.bias;
  p.relu = c.relu;
  p.beta = c.beta;
  p.ew = c.ew;
  p.out_bf16 = c.out_bf16;
  p.c_vec = ((reinterpret_cast<uintptr_t>(c.O) & 15) == 0 && c.F % (c.out_bf16 ? 8 : 4) == 0) ? 1 : 0;
  p.c_vec32 = ((reinterpret_cast<uintptr_t>(c.O) & 31) == 0 && c.F % (c.out_bf16 ? 16 : 8) == 0) ? 1 : 0;
  p.resid = (c.ew.n == 2 && c.ew.op[0] == NK_EW_ADD && c.ew.op[1] == NK_EW_RELU &&
             (reinterpret_cast<uintptr_t>(c.ew.t[0]) & 31) == 0 && c.F % 8 == 0) ? 1 : 0;
  p.budget = wait_budget();
  p.alpha = c.alpha;
  p.scale_i = c.scale_i;
  p.scale_w = c.scale_w;
  if (p.units == 0) return NK_OK;
  const bool db = stacked_db(g, s, kind);
  const int grid =
      std::min(p.units, sms * halo_ctas(L.smem, halo_tmem_cols(chains_of(g, s, kind), s.tile_n, t.stk, db)));
  if (f8) {
    if (t.stk <= 1) return fail(NK_ERR_NO_SCHEDULE, "E4M3 window convolutions stack kernel rows");
    return db ? launch<1, true, true, true>(p, grid, L.smem, st) : launch<1, true, false, true>(p, grid, L.smem, st);
  }
  if (t.stk > 1 && p.resid)
    return db ? launch<1, true, true, false, true>(p, grid, L.smem, st)
              : launch<1, true, false, false, true>(p, grid, L.smem, st);
  if (t.stk > 1) return db ? launch<1, true, true>(p, grid, L.smem, st) : launch<1, true>(p, grid, L.smem, st);
  switch (chains_of(g, s)) {
    case 1: return launch<1>(p, grid, L.smem, st);
    case 2: return launch<2>(p, grid, L.smem, st);
    default: return launch<4>(p, grid, L.smem, st);
  }
}

}  // namespace nk
