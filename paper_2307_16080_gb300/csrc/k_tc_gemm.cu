// k_tc_gemm.cu -- linalg.matmul on the 5th-generation tensor cores.
//
// C[m,n] (+)= sum_k A[m,k] B[k,n] (Sec. 2.1.1 Listing "linalg-matmul") with
// the bias / ReLU epilogue of the lowered Linear layer (Sec. 2.1.2 Listing
// "listing1").  The paper tiles the loop nest and searches tile sizes
// (Sec. 4.3); here one tile is a 128 x BN block of C computed by one CTA of a
// persistent grid:
//
//   warp 0      TMA producer: A and B tiles (128-byte rows, 128B swizzle) into
//               a STAGES-deep shared-memory ring, one mbarrier pair per slot.
//               Every CTA loads its own tiles: a cluster of two is a CTA pair
//               (below), in which each CTA loads its half of B; no TMA load
//               is multicast.
//   warp 1      allocates TMEM; one thread issues tcgen05.mma (M=128, N=BN,
//               K=16 BF16 / K=32 E4M3 per instruction) into a double-buffered
//               FP32 accumulator in TMEM, and tcgen05.commit frees each slot.
//   warps 2..5  epilogue: tcgen05.ld of their 32-lane quarter, then
//               alpha, beta*C, bias, ReLU and stores -- overlapping the
//               next tile's main loop through the second accumulator.
//
// BF16x3 issues three MMAs per K step (hi*hi, hi*lo, lo*hi) into the same
// accumulator.  Split-K writes each slice's raw tile to the workspace and the
// fixed-order warp-shuffle reduce applies the epilogue.
//
// Every wait is bounded (see tc_ptx.cuh); on a timeout the CTA drains its own
// copies and MMAs, frees TMEM and exits, and the host reports NK_ERR_TIMEOUT.
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

__device__ unsigned int g_tc_err;

uint32_t tc_read_and_clear_errors() {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_err, sizeof v) != cudaSuccess) return 0;
  const unsigned int z = 0;
  cudaMemcpyToSymbol(g_tc_err, &z, sizeof z);
  return v;
}

namespace {

constexpr int kThreads = 192;       // 6 warps
constexpr int kBM = 128;
constexpr int kRowBytes = 128;      // one K block = one 128-byte swizzle row
constexpr int kGroupM = 8;          // rasterisation: 8 (pair-)rows of tiles per band
constexpr int kMaxSmem = 232448;    // 227 KB opt-in limit

// Output tile of the convolution: NB images x R output rows x Q output
// columns (NB*R*Q <= 128 GEMM rows), and the input walk for each filter tap.
struct ConvTile {
  int Q, R, NB;
  int tiles_w, tiles_h;
  int N, OH, OW;
  int sh, sw, dh, dw, pt, pl;
  int KW, cblocks;
  int cblk;               // channels per K block: one 128-byte row (64 BF16, 128 E4M3)
};

struct TcParams {
  CUtensorMap tmA, tmB, tmA2, tmB2;
  int M, N, K;
  int bn, stages;
  int tiles_m, tiles_n;   // tiles_m padded to the cluster size
  int splits, kb_per_split, nkb;
  int units;
  float* C;
  int64_t ldc;
  float* partial;         // [splits][M][N] when splits > 1
  const float* bias;
  int bias_on_m, relu;
  float beta, alpha;
  const float* scale_a;
  const float* scale_b;
  int64_t budget;
  int c_vec;
  // grouped launches: per-group shapes, outputs and TMA descriptors in device memory
  const struct GroupDesc* groups;
  const int* tile_start;        // [G+1] prefix sums of tiles per group
  const int* unit_group;        // [units] group of each unit, or null (binary search)
  const CUtensorMap* gmaps;     // [G][2]: A_g, Bt_g
  const CUtensorMap* gcmaps;    // [G]: C_g for the TMA-store epilogue (c_tma), or null
  int G;
  // implicit-GEMM convolution (tmA: 4-D NHWC input map, tmB: 3-D [F][taps][C] map)
  ConvTile cv;
  uint32_t a_box_bytes;         // bytes TMA writes per A stage (16 KB unless a conv tile is short)
  // epilogue through shared memory and TMA stores (plain GEMM, beta = 0, one K slice)
  CUtensorMap tmC;
  int c_tma;
  EwProg ew;                    // fused elementwise program (offsets from C), single launches
  int out_bf16;                 // single convolutions: C holds BF16 (RNE of the FP32 result)
  int c_vec32;                  // single convolutions: 32-byte aligned output rows
  int resid;                    // single convolutions: ew is {ADD t, RELU}, t with 32-byte aligned rows
};

// Epilogue staging: one 32 x 32 FP32 box (4 KB, 128B-swizzled) per epilogue warp.
constexpr int kStageBox = 4096;
__host__ __device__ inline int staging_bytes(bool wide, int mch = 1) {
  return mch > 1 ? 0 : (wide ? 8 : 4) * kStageBox;   // tall tiles store directly
}

struct GroupDesc {
  int M, N, K, tiles_n;
  float* C;
  int64_t ldc;
  float beta;
  int kblocks;            // K blocks of 64 elements (a conv: taps x channel blocks)
  const float* bias;      // per output column, or null
  int relu;
  int pad;
  ConvTile cv;            // grouped convolutions: the group's output tiling
};

// One pipeline stage: mch A tiles of 128 rows (one per accumulator chain)
// and one B^T tile of bn rows, each row 128 bytes; BF16x3 doubles it (hi, lo).
__host__ __device__ inline int stage_bytes(int kind, int bn, int mch = 1) {
  const int ab = mch * kBM * kRowBytes + bn * kRowBytes;
  return kind == TC_BF16X3 ? 2 * ab : ab;
}

struct Unit {
  int tm, tn, split;
};

// Everything one role needs to know about a unit of work.
struct UnitView {
  int tm, tn, split, kb0, kb1, M, N;
  const CUtensorMap* ma;
  const CUtensorMap* mb;
  const CUtensorMap* mc;   // C map of the TMA-store epilogue
  float* C;
  int64_t ldc;
  float beta;
  const float* bias;
  int relu;
  const ConvTile* cv;    // conv launches: the tiling of this unit's convolution
};

__device__ __forceinline__ Unit decode_unit(const TcParams& p, int u, int cl, int rank) {
  const int tmp_count = p.tiles_m / cl;
  const int per_split = tmp_count * p.tiles_n;
  Unit r;
  r.split = u / per_split;
  const int t = u % per_split;
  const int band = kGroupM * p.tiles_n;
  const int first = (t / band) * kGroupM;
  const int gm = min(tmp_count - first, kGroupM);
  const int tmp = first + (t % band) % gm;
  r.tn = (t % band) / gm;
  r.tm = tmp * cl + rank;
  return r;
}

template <bool GROUPED>
__device__ __forceinline__ UnitView view_unit(const TcParams& p, int u, int cl, int rank) {
  UnitView v;
  if constexpr (GROUPED) {
    // group g with tile_start[g] <= u < tile_start[g+1]: one load from a
    // plan's unit map, else a binary search of the prefix sums.  The map
    // took 0.270 -> 0.245 ms off 512 uneven groups: the search's dependent
    // loads ran in every role for every unit.
    int lo = 0;
    if (p.unit_group) {
      lo = __ldg(p.unit_group + u);
    } else {
      int hi = p.G;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(p.tile_start + mid) <= u) lo = mid;
        else hi = mid;
      }
    }
    const GroupDesc& g = p.groups[lo];
    const int t = u - __ldg(p.tile_start + lo);
    v.tm = (t / g.tiles_n) * cl + rank;   // a pair's tile: its two 128-row halves
    v.tn = t % g.tiles_n;
    v.split = 0;
    v.kb0 = 0;
    v.kb1 = g.kblocks;
    v.M = g.M;
    v.N = g.N;
    v.ma = p.gmaps + 2 * lo;
    v.mb = p.gmaps + 2 * lo + 1;
    v.mc = p.gcmaps ? p.gcmaps + lo : nullptr;
    v.C = g.C;
    v.ldc = g.ldc;
    v.beta = g.beta;
    v.bias = g.bias;
    v.relu = g.relu;
    v.cv = &g.cv;
  } else {
    const Unit t = decode_unit(p, u, cl, rank);
    v.tm = t.tm;
    v.tn = t.tn;
    v.split = t.split;
    v.kb0 = t.split * p.kb_per_split;
    v.kb1 = min(p.nkb, v.kb0 + p.kb_per_split);
    v.M = p.M;
    v.N = p.N;
    v.ma = &p.tmA;
    v.mb = &p.tmB;
    v.mc = &p.tmC;
    v.C = p.C;
    v.ldc = p.ldc;
    v.beta = p.beta;
    v.bias = p.bias;
    v.relu = p.relu;
    v.cv = &p.cv;
  }
  return v;
}

// Output row of GEMM row r (0..127) of conv tile tm, or -1 if it is padding.
__device__ __forceinline__ int conv_row(const ConvTile& c, int tm, int r) {
  if (r >= c.Q * c.R * c.NB) return -1;
  const int tw = tm % c.tiles_w;
  const int th = (tm / c.tiles_w) % c.tiles_h;
  const int tb = tm / (c.tiles_w * c.tiles_h);
  const int q = r % c.Q, rr = (r / c.Q) % c.R, b = r / (c.Q * c.R);
  const int n = tb * c.NB + b, oh = th * c.R + rr, ow = tw * c.Q + q;
  if (n >= c.N || oh >= c.OH || ow >= c.OW) return -1;
  return (n * c.OH + oh) * c.OW + ow;
}

// PAIR: the two CTAs of a cluster form one 2-SM MMA (cta_group::2) computing a
// 256 x BN tile; each holds its 128 rows of A and BN/2 rows of B^T, and the
// even CTA's barriers gate the pair (its MMA thread is the only issuer).
//
// WIDE: a pair computing a 256 x 512 tile as two independent N = 256
// accumulator chains that share the A tile.  One chain of dependent MMAs on a
// single accumulator issues about one instruction per ~190 cycles, while an
// N = 256 MMA holds only 128 cycles of math; interleaving two chains hides
// that latency.  Both chains fill the 512 TMEM columns, so the accumulator is
// single-buffered and eight epilogue warps drain it.
//
// MCH > 1 (tall tile, one CTA): MCH stacked 128-row tiles of A share one B
// tile, each with its own accumulator chain, so narrow problems (N = 64, 128)
// keep several independent MMA chains in flight.
//
// EP8 (grouped launches with one CTA per SM): eight epilogue warps, two per
// TMEM lane quarter, each draining half of a tile's columns -- the
// epilogue of a 128 x 256 tile would otherwise outlast the next tile's MMAs.
// Each warp has its own staging box for the TMA-store epilogue (eight).
//
// Grouped launches store through TMA too (c_tma with a C map per group,
// when every group overwrites a 16-byte aligned C whose rows end on 16-byte
// boundaries): the store clips each group's ragged rows and columns past the
// last 16-byte granule, and one instruction writes a 32 x 32 block where
// per-lane stores touch 32 rows.  On 512 uneven groups (128 x 256 tiles,
// 4 stages) 0.244 -> 0.234 ms.
template <int KIND, int CL, bool GROUPED, bool CONV = false, bool PAIR = false, bool WIDE = false, int MCH = 1,
          bool EP8 = false>
__global__ void __launch_bounds__((WIDE || EP8) ? 320 : 192, 1) tc_gemm_kernel(const __grid_constant__ TcParams p) {
  static_assert(!EP8 || (GROUPED && !WIDE && MCH == 1 && KIND != TC_BF16X3), "eight epilogue warps: grouped tiles");
  static_assert(PAIR == (CL == 2), "a cluster of two is a CTA pair, and a CTA pair is a cluster of two");
  static_assert(!WIDE || (PAIR && KIND != TC_BF16X3 && !GROUPED), "wide tiles are pair tiles");
  static_assert(MCH == 1 || (!PAIR && !GROUPED && KIND != TC_BF16X3 && CL == 1), "tall tiles: one CTA");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = ptx::smem_u32(smem_raw);
  const uint32_t base = (raw + 1023) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw);

  const int b_rows_smem = PAIR ? p.bn / 2 : p.bn;   // rows of B^T this CTA keeps per stage
  const int sb = stage_bytes(KIND, b_rows_smem, MCH);
  const int S = p.stages;
  const uint32_t stg0 = base + S * sb;   // epilogue staging boxes
  const uint32_t bar0 = stg0 + staging_bytes(WIDE || EP8, MCH);   // full[S], empty[S], tfull[2], tempty[2], drain
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * S + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * S + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * S + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + S * sb + staging_bytes(WIDE || EP8, MCH) + 8 * (2 * S + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  {
    // Guard: the launch must have given this layout enough dynamic shared
    // memory; otherwise report and leave before touching any of it.
    uint32_t dsz;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsz));
    const uint32_t need = (base - raw) + (uint32_t)(S * sb + staging_bytes(WIDE || EP8, MCH) + 8 * (2 * S + 5) + 8);
    if (need > dsz) {
      if (threadIdx.x == 0) atomicOr(&g_tc_err, 2u);
      return;
    }
  }

  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  const int rank = CL == 2 ? (int)ptx::cluster_ctarank() : 0;
  const int cluster_id = blockIdx.x / CL;
  const int n_clusters = gridDim.x / CL;
  // Accumulator columns per buffer: BN, or 2*BN for BF16x3 (hi*hi and the
  // hi*lo + lo*hi corrections accumulate apart and meet in the epilogue, so
  // the large term sees K/16 roundings instead of 3K/16).
  const int acc_cols = KIND == TC_BF16X3 ? 2 * p.bn : MCH * p.bn;
  const uint32_t tmem_cols = WIDE ? 512u : 2u * (uint32_t)acc_cols < 32u ? 32u : 2u * (uint32_t)acc_cols;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(full_bar(s), 1);
      ptx::mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(tfull_bar(b), 1);
      ptx::mbar_init(tempty_bar(b), (WIDE || (PAIR && EP8)) ? 16 : (PAIR || EP8) ? 8 : 4);   // every epilogue warp
    }
    ptx::mbar_init(drain_bar, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0 && lane == 0 && !GROUPED) {
    ptx::tma_prefetch_desc(&p.tmA);
    ptx::tma_prefetch_desc(&p.tmB);
    if (KIND == TC_BF16X3) {
      ptx::tma_prefetch_desc(&p.tmA2);
      ptx::tma_prefetch_desc(&p.tmB2);
    }
  }
  if (warp == 1) {
    if (PAIR) {
      ptx::tmem_alloc_pair(ptx::smem_u32(tmem_slot), tmem_cols);
      ptx::tmem_relinquish_pair();
    } else {
      ptx::tmem_alloc(ptx::smem_u32(tmem_slot), tmem_cols);
      ptx::tmem_relinquish();
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (CL == 2) ptx::cluster_sync();
  const uint32_t tmem_base = *tmem_slot;
  // Set-up above touched no global data; everything below runs after the
  // earlier kernels on the stream have finished.
  nk::pdl_wait();
  nk::pdl_trigger();

  const int a_bytes = MCH * kBM * kRowBytes;
  const int b_bytes = b_rows_smem * kRowBytes;
  // Stage layout: [A][B] or, for BF16x3, [A_hi][B_hi][A_lo][B_lo].
  auto a_smem = [&](int s, int part) { return base + s * sb + part * (a_bytes + b_bytes); };
  auto b_smem = [&](int s, int part) { return base + s * sb + part * (a_bytes + b_bytes) + a_bytes; };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int it = 0;
      const int kblk = KIND == TC_FP8 ? 128 : 64;   // elements per 128-byte row
      bool ok = true;
      for (int u = cluster_id; u < p.units && ok; u += n_clusters) {
        const UnitView t = view_unit<GROUPED>(p, u, CL, rank);
        const int kb0 = t.kb0;
        const int kb1 = t.kb1;
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!ptx::mbar_wait(empty_bar(s), ph ^ 1u, p.budget, abort_flag, &g_tc_err)) { ok = false; break; }
          if constexpr (PAIR) {
            // Both CTAs load their own halves; the even CTA's barrier counts both.
            const uint32_t lf = ptx::mapa(full_bar(s), 0);
            const int by = t.tn * p.bn + rank * b_rows_smem;
            if constexpr (CONV) {
              const ConvTile& c = *t.cv;
              if (rank == 0) ptx::mbar_arrive_expect_tx(full_bar(s), 2u * (p.a_box_bytes + (uint32_t)b_bytes));
              const int tap = kb / c.cblocks, c0 = (kb % c.cblocks) * c.cblk;
              const int kh = tap / c.KW, kw = tap % c.KW;
              const int tw = t.tm % c.tiles_w, th = (t.tm / c.tiles_w) % c.tiles_h;
              const int tb = t.tm / (c.tiles_w * c.tiles_h);
              ptx::tma_load_4d_pair(a_smem(s, 0), t.ma, lf, c0, tw * c.Q * c.sw + kw * c.dw - c.pl,
                                    th * c.R * c.sh + kh * c.dh - c.pt, tb * c.NB);
              ptx::tma_load_3d_pair(b_smem(s, 0), t.mb, lf, c0, tap, by);
            } else {
              if (rank == 0) ptx::mbar_arrive_expect_tx(full_bar(s), 2u * (uint32_t)sb);
              const int kx = kb * kblk;
              if (WIDE) {
                // chain h (N columns h*256 .. h*256+255): this CTA holds its 128 rows of B^T
                ptx::tma_load_2d_pair(a_smem(s, 0), t.ma, lf, kx, t.tm * kBM);
                ptx::tma_load_2d_pair(b_smem(s, 0), t.mb, lf, kx, t.tn * p.bn + rank * 128);
                ptx::tma_load_2d_pair(b_smem(s, 0) + 128 * kRowBytes, t.mb, lf, kx, t.tn * p.bn + 256 + rank * 128);
                continue;
              }
              const int nparts = KIND == TC_BF16X3 ? 2 : 1;
              for (int part = 0; part < nparts; ++part) {
                ptx::tma_load_2d_pair(a_smem(s, part), part ? &p.tmA2 : t.ma, lf, kx, t.tm * kBM);
                ptx::tma_load_2d_pair(b_smem(s, part), part ? &p.tmB2 : t.mb, lf, kx, by);
              }
            }
            continue;
          }
          if constexpr (CONV) {
            // K block kb = (filter tap, 64-channel block); the A box is the
            // input window that tap sees, shifted and strided by TMA.
            const ConvTile& c = *t.cv;
            // bytes one A box writes (a short conv tile writes fewer than 16 KB)
            const uint32_t a_box = GROUPED ? (uint32_t)(c.Q * c.R * c.NB * kRowBytes) : p.a_box_bytes;
            ptx::mbar_arrive_expect_tx(full_bar(s), MCH * a_box + (uint32_t)b_bytes);
            const int tap = kb / c.cblocks, c0 = (kb % c.cblocks) * c.cblk;
            const int kh = tap / c.KW, kw = tap % c.KW;
            for (int ch = 0; ch < MCH; ++ch) {
              const int ct = t.tm * MCH + ch;   // conv tile of this chain
              const int tw = ct % c.tiles_w, th = (ct / c.tiles_w) % c.tiles_h;
              const int tb = ct / (c.tiles_w * c.tiles_h);
              ptx::tma_load_4d(a_smem(s, 0) + ch * kBM * kRowBytes, t.ma, full_bar(s), c0,
                               tw * c.Q * c.sw + kw * c.dw - c.pl, th * c.R * c.sh + kh * c.dh - c.pt, tb * c.NB);
            }
            ptx::tma_load_3d(b_smem(s, 0), t.mb, full_bar(s), c0, tap, t.tn * p.bn);
            continue;
          }
          ptx::mbar_arrive_expect_tx(full_bar(s), (uint32_t)sb);
          const int kx = kb * kblk;
          const int ay = t.tm * MCH * kBM;
          const int by = t.tn * p.bn;
          const int nparts = KIND == TC_BF16X3 ? 2 : 1;
          for (int part = 0; part < nparts; ++part) {
            const CUtensorMap* ma = part ? &p.tmA2 : t.ma;
            const CUtensorMap* mb = part ? &p.tmB2 : t.mb;
            for (int ch = 0; ch < MCH; ++ch)
              ptx::tma_load_2d(a_smem(s, part) + ch * kBM * kRowBytes, ma, full_bar(s), kx, ay + ch * kBM);
            ptx::tma_load_2d(b_smem(s, part), mb, full_bar(s), kx, by);
          }
        }
      }
      // Drain: the last copy issued into each slot must land before exit.  In
      // a pair the odd CTA cannot poll the even CTA's barrier; the MMA that
      // consumed its copies frees its own slot, so it waits on that instead.
      const int last = it;
      for (int j = last - 1; j >= 0 && j >= last - S; --j) {
        if (PAIR && rank != 0) ptx::mbar_drain(empty_bar(j % S), (uint32_t)(j / S) & 1u, 100000000ull);
        else ptx::mbar_drain(full_bar(j % S), (uint32_t)(j / S) & 1u, 100000000ull);
      }
    }
  } else if (warp == 1) {
    // -------------------------------------------------------------- MMA
    if (lane == 0 && (!PAIR || rank == 0)) {
      const uint32_t idesc = ptx::make_idesc(KIND == TC_FP8 ? 0 : 1, PAIR ? 2 * kBM : kBM, WIDE ? 256 : p.bn);
      int it = 0, tc = 0;
      bool ok = true;
      for (int u = cluster_id; u < p.units && ok; u += n_clusters, ++tc) {
        const UnitView t = view_unit<GROUPED>(p, u, CL, rank);
        const int kb0 = t.kb0;
        const int kb1 = t.kb1;
        const int acc = WIDE ? 0 : tc & 1;   // a wide tile's two chains fill TMEM: one buffer
        const uint32_t aph = WIDE ? (uint32_t)tc & 1u : (uint32_t)(tc >> 1) & 1u;
        if (!ptx::mbar_wait(tempty_bar(acc), aph ^ 1u, p.budget, abort_flag, &g_tc_err)) break;
        ptx::tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(acc * acc_cols);
        const uint32_t d2 = d + (uint32_t)(WIDE ? 256 : p.bn);   // BF16x3 corrections / second wide chain
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!ptx::mbar_wait(full_bar(s), ph, p.budget, abort_flag, &g_tc_err)) { ok = false; break; }
          ptx::tc_fence_after();
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t koff = (uint32_t)k * 32u;
            const uint64_t ad = ptx::sw128_desc(a_smem(s, 0) + koff);
            const uint64_t bd = ptx::sw128_desc(b_smem(s, 0) + koff);
            const uint32_t accum = (kb > kb0 || k > 0) ? 1u : 0u;
            if (PAIR) ptx::tc_mma_pair<KIND == TC_FP8>(d, ad, bd, idesc, accum);
            else ptx::tc_mma<KIND == TC_FP8>(d, ad, bd, idesc, accum);
#pragma unroll
            for (int ch = 1; ch < MCH; ++ch)   // further chains: their own A rows, the same B
              ptx::tc_mma<KIND == TC_FP8>(d + (uint32_t)(ch * p.bn),
                                          ptx::sw128_desc(a_smem(s, 0) + ch * kBM * kRowBytes + koff), bd, idesc,
                                          accum);
            if (WIDE) {   // second chain: B^T rows 128..255 of this CTA's stage
              const uint64_t bw = ptx::sw128_desc(b_smem(s, 0) + 128 * kRowBytes + koff);
              ptx::tc_mma_pair<KIND == TC_FP8>(d2, ad, bw, idesc, accum);
            }
            if (KIND == TC_BF16X3) {
              const uint64_t ad2 = ptx::sw128_desc(a_smem(s, 1) + koff);
              const uint64_t bd2 = ptx::sw128_desc(b_smem(s, 1) + koff);
              if (PAIR) {
                ptx::tc_mma_pair<0>(d2, ad, bd2, idesc, accum);   // hi * lo
                ptx::tc_mma_pair<0>(d2, ad2, bd, idesc, 1u);      // lo * hi
              } else {
                ptx::tc_mma<0>(d2, ad, bd2, idesc, accum);   // hi * lo
                ptx::tc_mma<0>(d2, ad2, bd, idesc, 1u);      // lo * hi
              }
            }
          }
          if (PAIR) ptx::tc_commit_pair_mc(empty_bar(s), (uint16_t)0x3);
          else ptx::tc_commit(empty_bar(s));
        }
        if (!ok) break;
        if (PAIR) ptx::tc_commit_pair_mc(tfull_bar(acc), (uint16_t)0x3);
        else ptx::tc_commit(tfull_bar(acc));
      }
      // Drain: every MMA this thread issued completes before TMEM is freed.
      if (PAIR) ptx::tc_commit_pair(drain_bar);
      else ptx::tc_commit(drain_bar);
      ptx::mbar_drain(drain_bar, 0, 100000000ull);
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;   // TMEM lane quarter this warp may read
    float alpha = p.alpha;
    if (p.scale_a) alpha = __frcp_rn(__fmul_rn(*p.scale_a, *p.scale_b));
    int tc = 0;
    for (int u = cluster_id; u < p.units; u += n_clusters, ++tc) {
      const UnitView t = view_unit<GROUPED>(p, u, CL, rank);
      const int acc = WIDE ? 0 : tc & 1;
      const uint32_t aph = WIDE ? (uint32_t)tc & 1u : (uint32_t)(tc >> 1) & 1u;
      if (!ptx::mbar_wait(tfull_bar(acc), aph, p.budget, abort_flag, &g_tc_err)) break;
      ptx::tc_fence_after();
      for (int ch = 0; ch < MCH; ++ch) {   // chains of a tall tile (one otherwise)
      const int tmc = t.tm * MCH + ch;
      const int row = CONV ? conv_row(*t.cv, tmc, q * 32 + lane) : tmc * kBM + q * 32 + lane;
      const bool row_ok = CONV ? row >= 0 : row < t.M;
      // a wide tile has two warps per lane quarter, each draining one chain's 256 columns
      const int c_begin = WIDE ? ((warp - 2) / 4) * 256 : EP8 ? ((warp - 2) / 4) * (p.bn / 2) : 0;
      const int c_end = WIDE ? c_begin + 256 : EP8 ? c_begin + p.bn / 2 : p.bn;
      for (int c0 = c_begin; c0 < c_end; c0 += 32) {
        float v[32];
        const uint32_t ta =
            tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * acc_cols + ch * p.bn + c0);
        ptx::tmem_ld32(ta, v);
        if (KIND == TC_BF16X3) {
          float w[32];
          ptx::tmem_ld32(ta + (uint32_t)p.bn, w);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += w[j];
        }
        const int col0 = t.tn * p.bn + c0;
        if (!CONV && p.c_tma) {
          // Coalesced epilogue: registers -> this warp's 128B-swizzled 32 x 32
          // staging box -> one TMA store (rows / columns past C are clipped).
          if (col0 >= t.N) continue;
          const uint32_t stg = stg0 + (uint32_t)((warp - 2) * kStageBox);
          if (lane == 0) ptx::bulk_wait_read0();   // the box's previous store has read it
          __syncwarp();
          const float bm = (t.bias && p.bias_on_m && row_ok) ? __ldg(t.bias + row) : 0.f;
#pragma unroll
          for (int j16 = 0; j16 < 8; ++j16) {
            float o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int j = 4 * j16 + e;
              float x = alpha * v[j];
              if (t.bias) x += p.bias_on_m ? bm : (col0 + j < t.N ? __ldg(t.bias + col0 + j) : 0.f);
              if (t.relu) x = (x > 0.f || x != x) ? x : 0.f;
              o[e] = x;
            }
            const uint32_t addr = stg + (uint32_t)(lane * 128 + ((j16 ^ (lane & 7)) * 16));
            asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(o[0]), "f"(o[1]), "f"(o[2]),
                         "f"(o[3])
                         : "memory");
          }
          ptx::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            ptx::tma_store_2d(t.mc, stg, col0, tmc * kBM + q * 32);
            ptx::bulk_commit();
          }
          continue;
        }
        if (!row_ok || col0 >= t.N) continue;
        if (p.partial) {
          float* dst = p.partial + ((int64_t)t.split * p.M + row) * p.N + col0;
          if (p.c_vec && col0 + 32 <= p.N) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (col0 + j < p.N) dst[j] = v[j];
          }
          continue;
        }
        if constexpr (CONV && !GROUPED) {
          if (p.c_vec32 && t.beta == 0.f && col0 + 32 <= t.N && (p.ew.n == 0 || p.resid)) {
            // Full 32-column segment, no accumulate, and no program or the
            // residual program ADD t, RELU (inline, the interpreter's FP32
            // steps): one code path for FP32 and BF16 outputs.
            const int64_t off = (int64_t)row * t.ldc + col0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              float x = alpha * v[j];
              if (t.bias) x += __ldg(t.bias + col0 + j);
              if (t.relu) x = (x > 0.f || x != x) ? x : 0.f;
              v[j] = x;
            }
            if (p.resid) {
              const float4* tr = reinterpret_cast<const float4*>(p.ew.t[0] + off);
#pragma unroll
              for (int j = 0; j < 32; j += 4) {
                const float4 r4 = __ldg(tr + j / 4);
                const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const float x = __fadd_rn(v[j + e], rv[e]);
                  v[j + e] = (x > 0.f || x != x) ? x : 0.f;
                }
              }
            }
            if (p.out_bf16) store32_bf16_v8(reinterpret_cast<__nv_bfloat16*>(t.C) + off, v);
            else store32_f32_v8(t.C + off, v);
            continue;
          }
          if (p.out_bf16) {
            // BF16 output: the FP32 epilogue, then one RNE rounding per value
            __nv_bfloat16* dh = reinterpret_cast<__nv_bfloat16*>(t.C) + (int64_t)row * t.ldc + col0;
            const int ncol = t.N - col0 < 32 ? t.N - col0 : 32;
            float buf[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              float x = alpha * v[j];
              if (j < ncol) {
                if (t.beta != 0.f) x = fmaf(t.beta, __bfloat162float(dh[j]), x);
                if (t.bias) x += __ldg(t.bias + col0 + j);
                if (t.relu) x = (x > 0.f || x != x) ? x : 0.f;
              }
              buf[j] = x;
            }
            if (p.ew.n) ew_apply(p.ew, buf, ncol, (int64_t)row * t.ldc + col0);
            if (p.c_vec && ncol == 32) {
              store32_bf16(dh, buf);
            } else {
              for (int j = 0; j < ncol; ++j) dh[j] = __float2bfloat16_rn(buf[j]);
            }
            continue;
          }
        }
        float* dst = t.C + (int64_t)row * t.ldc + col0;
        const float bm = (t.bias && p.bias_on_m) ? __ldg(t.bias + row) : 0.f;
        const float beta = t.beta;
        if (!CONV && p.c_vec32 && beta == 0.f && col0 + 32 <= t.N && p.ew.n == 0) {
          // full 32-column segment of 32-byte aligned rows: 32-byte stores
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float x = alpha * v[j];
            if (t.bias) x += p.bias_on_m ? bm : __ldg(t.bias + col0 + j);
            if (t.relu) x = (x > 0.f || x != x) ? x : 0.f;
            v[j] = x;
          }
          store32_f32_v8(dst, v);
          continue;
        }
        if (p.ew.n) {
          // A program runs out of line.  The segment goes through a local
          // buffer: the program reads its operands (which may alias C) before
          // the store, and v[] is not live across the call, so the plain
          // paths below keep their registers.
          const int ncol = t.N - col0 < 32 ? t.N - col0 : 32;
          float buf[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float x = alpha * v[j];
            if (j < ncol) {
              if (beta != 0.f) x = fmaf(beta, dst[j], x);
              if (t.bias) x += p.bias_on_m ? bm : __ldg(t.bias + col0 + j);
              if (t.relu) x = (x > 0.f || x != x) ? x : 0.f;
            }
            buf[j] = x;
          }
          ew_apply(p.ew, buf, ncol, (int64_t)row * t.ldc + col0);
          for (int j = 0; j < ncol; ++j) dst[j] = buf[j];
        } else if (p.c_vec && col0 + 32 <= t.N) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            float o[4];
            float4 cin = make_float4(0.f, 0.f, 0.f, 0.f);
            if (beta != 0.f) cin = *reinterpret_cast<const float4*>(dst + j);
            const float ci[4] = {cin.x, cin.y, cin.z, cin.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              float x = alpha * v[j + e];
              if (beta != 0.f) x = fmaf(beta, ci[e], x);
              if (t.bias) x += p.bias_on_m ? bm : __ldg(t.bias + col0 + j + e);
              if (t.relu) x = (x > 0.f || x != x) ? x : 0.f;
              o[e] = x;
            }
            *reinterpret_cast<float4*>(dst + j) = make_float4(o[0], o[1], o[2], o[3]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (col0 + j >= t.N) continue;
            float x = alpha * v[j];
            if (beta != 0.f) x = fmaf(beta, dst[j], x);
            if (t.bias) x += p.bias_on_m ? bm : __ldg(t.bias + col0 + j);
            if (t.relu) x = (x > 0.f || x != x) ? x : 0.f;
            dst[j] = x;
          }
        }
      }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (PAIR) ptx::mbar_arrive_cluster(ptx::mapa(tempty_bar(acc), 0));   // the issuer's barrier
        else ptx::mbar_arrive(tempty_bar(acc));
      }
    }
    if (!CONV && p.c_tma && lane == 0) ptx::bulk_wait0();   // every store has landed
  }

  ptx::tc_fence_before();
  __syncthreads();
  // A pair frees TMEM only once the even CTA has drained every MMA that
  // writes into either CTA's TMEM.
  if (CL == 2) ptx::cluster_sync();
  ptx::tc_fence_after();
  if (warp == 1) {
    if (PAIR) ptx::tmem_dealloc_pair(tmem_base, tmem_cols);
    else ptx::tmem_dealloc(tmem_base, tmem_cols);
  }
  if (CL == 2) ptx::cluster_sync();
}

// ------------------------------------------------------------------ host
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D K-major operand [rows, K] with row stride ld (elements), 128B swizzle.
nk_status make_kmajor_map(CUtensorMap* m, bool fp8, const void* ptr, int64_t rows, int64_t K,
                          int64_t ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return fail(NK_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  const int esz = fp8 ? 1 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(NK_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for a [%lld, %lld] operand", (int)r,
                (long long)rows, (long long)K);
  return NK_OK;
}

int smem_bytes(int kind, int bn, int stages, bool wide = false, int mch = 1) {
  return 1024 + stages * stage_bytes(kind, bn, mch) + staging_bytes(wide, mch) + 8 * (2 * stages + 5) + 16;
}

// Accumulator chains along M of a one-CTA schedule: tile_m 256 / 512 with
// cluster 1 are tall tiles of 2 / 4 chains (tile_m 256 with cluster 2 is a pair).
int chains_of(const nk_schedule& s) { return (s.cluster == 1 && s.tile_m > 128) ? s.tile_m / 128 : 1; }

// Shared memory of a schedule: a CTA of a pair (tile_m 256) keeps half of B.
int smem_of(int kind, const nk_schedule& s) {
  const bool pair = s.cluster == 2 && s.tile_m == 256;
  return smem_bytes(kind, pair ? s.tile_n / 2 : s.tile_n, s.stages, s.tile_n == 512, chains_of(s));
}

template <int KIND, int CL, bool GROUPED = false, bool CONV = false, bool PAIR = false, bool WIDE = false,
          int MCH = 1, bool EP8 = false>
nk_status launch(const TcParams& p, int grid, int smem, cudaStream_t st) {
  auto kern = tc_gemm_kernel<KIND, CL, GROUPED, CONV, PAIR, WIDE, MCH, EP8>;
  // the attribute is set once per device and size (it stays set on the function)
  static int set_bytes[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || set_bytes[dev] < smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tc_gemm_kernel)");
    if (dev >= 0 && dev < 64) set_bytes[dev] = smem;
  }
  const cudaError_t e = nk::launch_k(kern, dim3(grid), dim3((WIDE || EP8) ? 320 : kThreads), smem, st, CL, p);
  if (e != cudaSuccess) return cuda_fail(e, "launch tc_gemm_kernel");
  return check_launch("tc_gemm_kernel");
}

// CTAs that fit on one SM: shared memory and the 512 TMEM columns.
int ctas_per_sm(int kind, const nk_schedule& s) {
  if (s.tile_n == 512) return 1;   // a wide tile holds all 512 TMEM columns
  const int bn = s.tile_n;
  const int sm = smem_of(kind, s);
  int by_smem = kMaxSmem / sm;
  const int acc = kind == TC_BF16X3 ? 2 * bn : chains_of(s) * bn;
  int cols = 2 * acc < 32 ? 32 : 2 * acc;
  int by_tmem = 512 / cols;
  int r = by_smem < by_tmem ? by_smem : by_tmem;
  return r < 1 ? 1 : (r > 2 ? 2 : r);
}

}  // namespace

bool tc_schedule_valid(int kind, const nk_schedule& s, int M, int N, int K) {
  (void)M; (void)N; (void)K;
  // tile_m 256 with cluster 2 = a CTA pair issuing 2-SM MMAs; tile_m 256 / 512
  // with cluster 1 = a tall tile of 2 / 4 accumulator chains sharing B.  A
  // cluster of two is always a CTA pair: no schedule multicasts a TMA load.
  if (s.tile_m != 128 && s.tile_m != 256 && s.tile_m != 512) return false;
  if (s.cluster == 2 && s.tile_m != 256) return false;
  if (chains_of(s) > 1 && (kind == TC_BF16X3 || chains_of(s) * s.tile_n > 256)) return false;
  if (s.tile_n != 64 && s.tile_n != 128 && s.tile_n != 256 && s.tile_n != 512) return false;
  if (s.tile_n == 512 && (s.tile_m != 256 || kind == TC_BF16X3)) return false;   // wide pair tiles only
  if (kind == TC_BF16X3 && s.tile_n > 128) return false;   // 2 accumulators x 2 buffers <= 512 cols
  if (s.tile_k != (kind == TC_FP8 ? 128 : 64)) return false;
  if (s.cluster != 1 && s.cluster != 2) return false;
  if (s.split_k < 1 || s.split_k > 32) return false;
  if (s.stages < 2 || s.stages > 8) return false;
  if (smem_of(kind, s) > kMaxSmem) return false;
  return true;
}

nk_schedule tc_default_schedule(int kind, int M, int N, int K, int sms) {
  nk_schedule s{};
  s.tile_m = 128;
  s.tile_k = kind == TC_FP8 ? 128 : 64;
  s.tile_n = kind == TC_BF16X3 ? 128 : 256;
  if (N <= 64) s.tile_n = 64;
  else if (N <= 128) s.tile_n = 128;
  s.cluster = 1;
  s.stages = 2;
  while (s.stages < 8 && smem_bytes(kind, s.tile_n, s.stages + 1) <= kMaxSmem) ++s.stages;
  // Large BF16 / FP8 problems: wide pair tiles (256 x 512, two MMA chains)
  // when there are at least two waves of them.
  if (kind != TC_BF16X3 && (int64_t)((M + 255) / 256) * ((N + 511) / 512) >= sms) {
    s.tile_m = 256; s.tile_n = 512; s.cluster = 2; s.stages = 4; s.split_k = 1;
    return s;
  }
  // Split K when the output tiles cannot fill the GPU and K is deep.
  const int tiles = ((M + 127) / 128) * ((N + s.tile_n - 1) / s.tile_n);
  const int nkb = (K + s.tile_k - 1) / s.tile_k;
  s.split_k = 1;
  while (tiles * s.split_k * 2 <= sms && nkb / (s.split_k * 2) >= 4 && s.split_k < 16) s.split_k *= 2;
  return s;
}

size_t tc_gemm_ws(const TcGemm& g, const nk_schedule& s) {
  if (s.split_k <= 1) return 0;
  return (size_t)s.split_k * g.M * g.N * sizeof(float);
}

nk_status tc_gemm(const TcGemm& g, const nk_schedule& s, void* ws, size_t ws_bytes, cudaStream_t st) {
  int sms = 0;
  nk_status status = require_device(&sms);
  if (status != NK_OK) return status;
  if (g.M <= 0 || g.N <= 0) return NK_OK;
  if (!tc_schedule_valid(g.kind, s, g.M, g.N, g.K))
    return fail(NK_ERR_NO_SCHEDULE, "illegal tensor-core schedule");
  if (g.K <= 0) {
    // Empty reduction: the epilogue alone (the CUDA-core kernel with K = 0).
    SimtGemm z{};
    z.A = nullptr; z.sam = 0; z.sak = 1;
    z.B = nullptr; z.sbk = 1; z.sbn = 0;
    z.C = g.C; z.scm = g.ldc; z.scn = 1;
    z.bias = g.bias; z.bias_on_m = g.bias_on_m;
    z.M = g.M; z.N = g.N; z.K = 0;
    z.alpha = 1.f; z.beta = g.beta; z.relu = g.relu;
    z.ew = g.ew;
    return simt_gemm(z, 64, 1, nullptr, 0, st);
  }
  const bool fp8 = g.kind == TC_FP8;
  const int esz = fp8 ? 1 : 2;
  if ((g.lda * esz) % 16 || (g.ldb * esz) % 16)
    return fail(NK_ERR_MISALIGNED, "operand row strides must be multiples of 16 bytes");
  TcParams p;
  memset(&p, 0, sizeof p);
  const int CL = s.cluster;
  if ((status = make_kmajor_map(&p.tmA, fp8, g.A, g.M, g.K, g.lda, kBM)) != NK_OK) return status;
  const int b_box = s.tile_n == 512 ? 128 : s.tile_n / CL;   // a wide tile loads B^T in 128-row boxes
  if ((status = make_kmajor_map(&p.tmB, fp8, g.B, g.N, g.K, g.ldb, b_box)) != NK_OK) return status;
  if (g.kind == TC_BF16X3) {
    if ((status = make_kmajor_map(&p.tmA2, fp8, g.A2, g.M, g.K, g.lda, kBM)) != NK_OK) return status;
    if ((status = make_kmajor_map(&p.tmB2, fp8, g.B2, g.N, g.K, g.ldb, s.tile_n / CL)) != NK_OK) return status;
  }
  p.M = g.M; p.N = g.N; p.K = g.K;
  p.bn = s.tile_n;
  p.stages = s.stages;
  const int mch = chains_of(s);
  const int tm = (g.M + kBM * mch - 1) / (kBM * mch);
  p.tiles_m = (tm + CL - 1) / CL * CL;
  p.tiles_n = (g.N + s.tile_n - 1) / s.tile_n;
  p.nkb = (g.K + s.tile_k - 1) / s.tile_k;
  int splits = s.split_k > p.nkb ? p.nkb : s.split_k;
  p.kb_per_split = (p.nkb + splits - 1) / splits;
  splits = (p.nkb + p.kb_per_split - 1) / p.kb_per_split;
  p.splits = splits;
  p.units = (p.tiles_m / CL) * p.tiles_n * splits;
  p.C = g.C;
  p.ldc = g.ldc;
  p.partial = nullptr;
  if (splits > 1) {
    const size_t need = (size_t)splits * g.M * g.N * sizeof(float);
    if (!ws || ws_bytes < need) return fail(NK_ERR_WORKSPACE, "split-K needs %zu bytes of workspace", need);
    p.partial = static_cast<float*>(ws);
  }
  p.bias = g.bias;
  p.bias_on_m = g.bias_on_m;
  p.relu = g.relu;
  p.beta = g.beta;
  p.alpha = g.alpha;
  p.scale_a = g.scale_a;
  p.scale_b = g.scale_b;
  p.ew = g.ew;
  p.budget = wait_budget();
  const bool cvec = ((reinterpret_cast<uintptr_t>(g.C) & 15) == 0) && (g.ldc % 4 == 0) &&
                    (splits == 1 || (g.N % 4 == 0 && (reinterpret_cast<uintptr_t>(ws) & 15) == 0));
  p.c_vec = cvec ? 1 : 0;
  p.c_vec32 = (splits == 1 && (reinterpret_cast<uintptr_t>(g.C) & 31) == 0 && g.ldc % 8 == 0) ? 1 : 0;
  // TMA-store epilogue: plain overwrite of a 16-byte aligned C in one K slice.
  // Rows must also end on a 16-byte boundary (N % 4 == 0): a TMA store clips
  // the innermost dimension only to 16-byte granules, so with N % 4 != 0 and
  // a padded row stride it wrote the row's padding (caught by canaries).
  p.c_tma = 0;
  if (mch == 1 && splits == 1 && g.beta == 0.f && g.ew.n == 0 && (reinterpret_cast<uintptr_t>(g.C) & 15) == 0 &&
      (g.ldc * 4) % 16 == 0 && g.N % 4 == 0) {
    auto fn = encode_fn();
    cuuint64_t dims[2] = {(cuuint64_t)g.N, (cuuint64_t)g.M};
    cuuint64_t strides[1] = {(cuuint64_t)(g.ldc * 4)};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t es[2] = {1, 1};
    if (fn && fn(&p.tmC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, g.C, dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      p.c_tma = 1;
  }
  const int smem = smem_of(g.kind, s);
  int grid = sms * ctas_per_sm(g.kind, s);
  grid = grid / CL * CL;
  const int need_ctas = p.units * CL;
  if (grid > need_ctas) grid = need_ctas;
  if (grid < CL) grid = CL;
  const bool pair = s.tile_m == 256;
  if (s.tile_n == 512) {
    if (g.kind == TC_FP8) status = launch<TC_FP8, 2, false, false, true, true>(p, grid, smem, st);
    else status = launch<TC_BF16, 2, false, false, true, true>(p, grid, smem, st);
  } else if (mch == 2) {
    if (g.kind == TC_FP8) status = launch<TC_FP8, 1, false, false, false, false, 2>(p, grid, smem, st);
    else status = launch<TC_BF16, 1, false, false, false, false, 2>(p, grid, smem, st);
  } else if (mch == 4) {
    if (g.kind == TC_FP8) status = launch<TC_FP8, 1, false, false, false, false, 4>(p, grid, smem, st);
    else status = launch<TC_BF16, 1, false, false, false, false, 4>(p, grid, smem, st);
  } else
  switch (g.kind * 2 + (pair ? 1 : 0)) {
    case TC_BF16 * 2 + 0: status = launch<TC_BF16, 1>(p, grid, smem, st); break;
    case TC_BF16 * 2 + 1: status = launch<TC_BF16, 2, false, false, true>(p, grid, smem, st); break;
    case TC_FP8 * 2 + 0: status = launch<TC_FP8, 1>(p, grid, smem, st); break;
    case TC_FP8 * 2 + 1: status = launch<TC_FP8, 2, false, false, true>(p, grid, smem, st); break;
    case TC_BF16X3 * 2 + 0: status = launch<TC_BF16X3, 1>(p, grid, smem, st); break;
    default: status = launch<TC_BF16X3, 2, false, false, true>(p, grid, smem, st); break;
  }
  if (status != NK_OK || splits == 1) return status;
  SplitReduce r{};
  r.partial = p.partial;
  r.splits = splits;
  r.M = g.M;
  r.N = g.N;
  r.C = g.C;
  r.scm = g.ldc;
  r.scn = 1;
  r.bias = g.bias;
  r.bias_on_m = g.bias_on_m;
  r.alpha = g.alpha;
  r.beta = g.beta;
  r.relu = g.relu;
  r.scale_a = g.scale_a;
  r.scale_b = g.scale_b;
  r.ew = g.ew;
  return splitk_reduce(r, st);
}

}  // namespace nk

// ===================================================================== conv
namespace nk {
namespace {

// Output tile (Q columns x R rows x NB images, <= 128 GEMM rows) with the
// fewest tiles; ties go to the widest rows.
ConvTile search_conv_tile(const ConvGeom& g, int maxrows) {
  ConvTile best{};
  int64_t best_tiles = INT64_MAX;
  for (int Q = 1; Q <= maxrows && Q <= g.ow; ++Q) {
    if (Q * g.sw > 256) break;
    for (int R = 1; Q * R <= maxrows && R <= g.oh; ++R) {
      if (R * g.sh > 256) break;
      const int NB = std::max(1, std::min(g.n, maxrows / (Q * R)));
      const int64_t tiles = (int64_t)((g.n + NB - 1) / NB) * ((g.oh + R - 1) / R) * ((g.ow + Q - 1) / Q);
      if (tiles < best_tiles || (tiles == best_tiles && Q > best.Q)) {
        best_tiles = tiles;
        best.Q = Q; best.R = R; best.NB = NB;
      }
    }
  }
  best.tiles_w = (g.ow + best.Q - 1) / best.Q;
  best.tiles_h = (g.oh + best.R - 1) / best.R;
  best.N = g.n; best.OH = g.oh; best.OW = g.ow;
  best.sh = g.sh; best.sw = g.sw; best.dh = g.dh; best.dw = g.dw; best.pt = g.pt; best.pl = g.pl;
  best.KW = g.kw;
  best.cblk = 64;
  best.cblocks = (g.c + 63) / 64;
  return best;
}

// The search above runs per call; its answer is cached per geometry.
std::mutex g_ctile_mu;
std::vector<std::pair<ConvGeom, ConvTile>> g_ctile_cache;

ConvTile cached_conv_tile(const ConvGeom& g) {
  std::lock_guard<std::mutex> lk(g_ctile_mu);
  for (auto& e : g_ctile_cache)
    if (std::memcmp(&e.first, &g, sizeof g) == 0) return e.second;
  const ConvTile t = search_conv_tile(g, 128);
  if (g_ctile_cache.size() > 4096) g_ctile_cache.clear();
  g_ctile_cache.push_back({g, t});
  return t;
}

// The tile of a geometry, with K blocks of one 128-byte row of channels.
ConvTile choose_conv_tile(const ConvGeom& g, int kind) {
  ConvTile t = cached_conv_tile(g);
  t.cblk = kind == TC_FP8 ? 128 : 64;
  t.cblocks = (g.c + t.cblk - 1) / t.cblk;
  return t;
}

nk_status make_conv_maps(CUtensorMap* map_a, CUtensorMap* map_b, const TcConv& c, const ConvTile& t, int bn_box) {
  auto fn = encode_fn();
  if (!fn) return fail(NK_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  const ConvGeom& g = c.g;
  const bool fp8 = c.kind == TC_FP8;
  const int esz = fp8 ? 1 : 2;
  const CUtensorMapDataType dt = fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  {
    cuuint64_t dims[4] = {(cuuint64_t)g.c, (cuuint64_t)g.w, (cuuint64_t)g.h, (cuuint64_t)g.n};
    cuuint64_t strides[3] = {(cuuint64_t)c.sI_w * esz, (cuuint64_t)c.sI_h * esz, (cuuint64_t)c.sI_n * esz};
    cuuint32_t box[4] = {(cuuint32_t)t.cblk, (cuuint32_t)(t.Q * g.sw), (cuuint32_t)(t.R * g.sh), (cuuint32_t)t.NB};
    cuuint32_t es[4] = {1, (cuuint32_t)g.sw, (cuuint32_t)g.sh, 1};
    CUresult r = fn(map_a, dt, 4, const_cast<void*>(c.I), dims, strides, box,
                    es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(NK_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for the conv input", (int)r);
  }
  {
    const int taps = g.kh * g.kw;
    cuuint64_t dims[3] = {(cuuint64_t)g.c, (cuuint64_t)taps, (cuuint64_t)c.F};
    cuuint64_t strides[2] = {(cuuint64_t)c.ldw * esz, (cuuint64_t)c.sW_f * esz};
    cuuint32_t box[3] = {(cuuint32_t)t.cblk, 1, (cuuint32_t)bn_box};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(map_b, dt, 3, const_cast<void*>(c.Wt), dims, strides, box,
                    es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(NK_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for the conv weights", (int)r);
  }
  return NK_OK;
}

}  // namespace

bool tc_conv_schedule_valid(const ConvGeom& g, int F, const nk_schedule& s, int kind) {
  if (kind != TC_BF16 && kind != TC_FP8) return false;
  if (halo_schedule(g, s, kind)) return halo_schedule_valid(g, F, s, kind);
  if (g.sw > 8 || g.sh > 8 || s.tile_n == 512) return false;
  // E4M3 convolutions: one CTA per tile, tall tiles included (no CTA pairs)
  if (kind == TC_FP8 && s.cluster == 2) return false;
  return tc_schedule_valid(kind, s, g.n * g.oh * g.ow, F, g.kh * g.kw * g.c);
}

// The shared-window kernel where it wins (see tc_halo_default_schedule).
// Otherwise one 128 x 64 tile per CTA for BF16 (128 x 128 for E4M3 when F >
// 64) -- more, narrower tiles keep more independent MMA chains busy: over the
// tuner's BF16 corpus (100 conv problems, every legal schedule timed) 64-wide
// tiles took the mean regret of this default from 16 % to 6 %, mostly on
// strided and 1x1 layers with F >= 128 -- with as many stages as leave room
// for two CTAs per SM (short K loops gain more from a second CTA than from
// deeper rings), and split-K while the grid would leave half the SMs idle.
nk_schedule tc_conv_default_schedule(const ConvGeom& g, int F, int sms, int kind) {
  bool ok = false;
  if (kind == TC_BF16 || kind == TC_FP8) {
    nk_schedule h = tc_halo_default_schedule(g, F, sms, &ok, kind);
    if (ok) return h;
  }
  nk_schedule s{};
  s.tile_m = 128;
  s.tile_k = kind == TC_FP8 ? 128 : 64;
  s.tile_n = (kind == TC_BF16 || F <= 64) ? 64 : 128;
  s.cluster = 1;
  s.split_k = 1;
  s.stages = 2;
  const bool two = 4 * s.tile_n <= 512;   // two CTAs' double-buffered accumulators fit in TMEM
  for (;;) {
    nk_schedule n = s;
    n.stages = s.stages + 1;
    const int need = smem_of(kind, n);
    if (n.stages > 8 || need > kMaxSmem || (two && 2 * (need + 1024) > kMaxSmem + 1024)) break;
    s = n;
  }
  const ConvTile t = choose_conv_tile(g, kind);
  const int ctiles = t.tiles_w * t.tiles_h * ((g.n + t.NB - 1) / t.NB);
  const int tiles = ctiles * ((F + s.tile_n - 1) / s.tile_n);
  const int nkb = g.kh * g.kw * t.cblocks;
  while (tiles * s.split_k * 2 <= sms && nkb / (s.split_k * 2) >= 4 && s.split_k < 16) s.split_k *= 2;
  return s;
}

size_t tc_conv_ws(const TcConv& c, const nk_schedule& s) {
  if (s.split_k <= 1 || halo_schedule(c.g, s, c.kind)) return 0;
  return (size_t)s.split_k * c.g.n * c.g.oh * c.g.ow * c.F * sizeof(float);
}

nk_status tc_conv(const TcConv& c, const nk_schedule& s, void* ws, size_t ws_bytes, cudaStream_t st) {
  int sms = 0;
  nk_status status = require_device(&sms);
  if (status != NK_OK) return status;
  const ConvGeom& g = c.g;
  const int kind = c.kind;
  if ((kind == TC_BF16 || kind == TC_FP8) && halo_schedule(g, s, kind)) return tc_halo_conv(c, s, st);
  const int M = g.n * g.oh * g.ow;
  if (g.sw > 8 || g.sh > 8) return fail(NK_ERR_UNSUPPORTED, "conv stride above 8");
  if (!tc_conv_schedule_valid(g, c.F, s, kind))
    return fail(NK_ERR_NO_SCHEDULE, "illegal tensor-core schedule for conv");
  const int esz = kind == TC_FP8 ? 1 : 2;
  if ((c.sI_w * esz) % 16 || (c.sI_h * esz) % 16 || (c.sI_n * esz) % 16 || (c.ldw * esz) % 16 ||
      (c.sW_f * esz) % 16 || (reinterpret_cast<uintptr_t>(c.I) & 15) || (reinterpret_cast<uintptr_t>(c.Wt) & 15))
    return fail(NK_ERR_MISALIGNED, "conv operands need 16-byte aligned bases and strides");
  const ConvTile t = choose_conv_tile(g, kind);
  TcParams p;
  memset(&p, 0, sizeof p);
  const int CL = s.cluster;
  if ((status = make_conv_maps(&p.tmA, &p.tmB, c, t, s.tile_n / CL)) != NK_OK) return status;
  p.cv = t;
  p.a_box_bytes = (uint32_t)(t.Q * t.R * t.NB * kRowBytes);
  p.M = M; p.N = c.F; p.K = g.kh * g.kw * g.c;
  p.bn = s.tile_n;
  p.stages = s.stages;
  const int mch = chains_of(s);
  const int ctiles = t.tiles_w * t.tiles_h * ((g.n + t.NB - 1) / t.NB);
  const int tm = (ctiles + mch - 1) / mch;
  p.tiles_m = (tm + CL - 1) / CL * CL;
  p.tiles_n = (c.F + s.tile_n - 1) / s.tile_n;
  p.nkb = g.kh * g.kw * t.cblocks;
  int splits = s.split_k > p.nkb ? p.nkb : s.split_k;
  p.kb_per_split = (p.nkb + splits - 1) / splits;
  splits = (p.nkb + p.kb_per_split - 1) / p.kb_per_split;
  p.splits = splits;
  p.units = (p.tiles_m / CL) * p.tiles_n * splits;
  p.C = c.O;
  p.ldc = c.F;
  if (splits > 1) {
    const size_t need = (size_t)splits * M * c.F * sizeof(float);
    if (!ws || ws_bytes < need) return fail(NK_ERR_WORKSPACE, "split-K needs %zu bytes of workspace", need);
    p.partial = static_cast<float*>(ws);
  }
  p.bias = c.bias;
  p.relu = c.relu;
  p.beta = c.beta;
  // E4M3 operands the caller quantised carry 1/(s_i s_w) in alpha
  p.alpha = (kind == TC_FP8 && !c.scale_i) ? c.alpha : 1.f;
  p.scale_a = c.scale_i;   // E4M3: alpha = 1 / (s_i * s_w), read on the device
  p.scale_b = c.scale_w;
  p.ew = c.ew;
  p.budget = wait_budget();
  p.out_bf16 = c.out_bf16;
  p.c_vec32 = (splits == 1 && (reinterpret_cast<uintptr_t>(c.O) & 31) == 0 && c.F % (c.out_bf16 ? 16 : 8) == 0) ? 1 : 0;
  p.resid = (c.ew.n == 2 && c.ew.op[0] == NK_EW_ADD && c.ew.op[1] == NK_EW_RELU &&
             (reinterpret_cast<uintptr_t>(c.ew.t[0]) & 31) == 0 && c.F % 8 == 0) ? 1 : 0;
  // vector stores: 16-byte aligned rows (FP32: F % 4, BF16: F % 8) and partials
  p.c_vec = ((reinterpret_cast<uintptr_t>(c.O) & 15) == 0 && c.F % (c.out_bf16 ? 8 : 4) == 0 &&
             (splits == 1 || (reinterpret_cast<uintptr_t>(ws) & 15) == 0)) ? 1 : 0;
  const int smem = smem_of(kind, s);
  if (smem > kMaxSmem) return fail(NK_ERR_NO_SCHEDULE, "conv schedule needs %d bytes of shared memory", smem);
  int grid = sms * ctas_per_sm(kind, s);
  grid = grid / CL * CL;
  if (grid > p.units * CL) grid = p.units * CL;
  if (grid < CL) grid = CL;
  if (kind == TC_FP8) {
    if (mch == 2) status = launch<TC_FP8, 1, false, true, false, false, 2>(p, grid, smem, st);
    else if (mch == 4) status = launch<TC_FP8, 1, false, true, false, false, 4>(p, grid, smem, st);
    else status = launch<TC_FP8, 1, false, true>(p, grid, smem, st);
  } else if (mch == 2) status = launch<TC_BF16, 1, false, true, false, false, 2>(p, grid, smem, st);
  else if (mch == 4) status = launch<TC_BF16, 1, false, true, false, false, 4>(p, grid, smem, st);
  else if (CL == 2) status = launch<TC_BF16, 2, false, true, true>(p, grid, smem, st);
  else status = launch<TC_BF16, 1, false, true>(p, grid, smem, st);
  if (status != NK_OK || splits == 1) return status;
  SplitReduce r{};
  r.partial = p.partial;
  r.splits = splits;
  r.M = M;
  r.N = c.F;
  r.C = c.O;
  r.scm = c.F;
  r.scn = 1;
  r.bias = c.bias;
  r.alpha = (kind == TC_FP8 && !c.scale_i) ? c.alpha : 1.f;
  r.beta = c.beta;
  r.relu = c.relu;
  r.scale_a = c.scale_i;
  r.scale_b = c.scale_w;
  r.ew = c.ew;
  r.out_bf16 = c.out_bf16;
  return splitk_reduce(r, st);
}

}  // namespace nk

// ====================================================================== grouped
// linalg.batch_matmul generalised to G independent GEMMs of uneven shapes, all
// in one persistent launch: a device table holds each group's shape, output
// and TMA descriptors, and a prefix sum of tiles per group lets every CTA map
// its running unit index to (group, tile).  A plan also holds the group of
// every unit (one load); a launch from a caller's workspace searches the
// prefix sums instead.  Groups are ordered by decreasing K so the longest
// tiles start first.
struct nk_grouped_plan {
  void* dev = nullptr;     // device table (owned when built by nk_grouped_plan_create)
  int* umap = nullptr;     // [units] group of each unit (plans only)
  bool owned = false;
  bool pair = false;       // 256-row tiles on CTA pairs (cta_group::2)
  bool ep8 = false;        // GEMM groups on one CTA per SM: eight epilogue warps
  bool conv = false;       // groups are convolutions (implicit GEMM, per-tap loads)
  int units = 0;
  int grid = 0;
  int smem = 0;
  nk::TcParams p;
};

namespace nk {
namespace {

// One persistent launch of a grouped GEMM plan: CTA pairs or one CTA per
// tile, with eight epilogue warps when a CTA has the SM to itself.
nk_status run_grouped_gemm(const nk_grouped_plan& plan, cudaStream_t st) {
  if (plan.pair) {
    if (plan.ep8) return launch<TC_BF16, 2, true, false, true, false, 1, true>(plan.p, plan.grid, plan.smem, st);
    return launch<TC_BF16, 2, true, false, true>(plan.p, plan.grid, plan.smem, st);
  }
  if (plan.ep8) return launch<TC_BF16, 1, true, false, false, false, 1, true>(plan.p, plan.grid, plan.smem, st);
  return launch<TC_BF16, 1, true>(plan.p, plan.grid, plan.smem, st);
}

size_t grouped_bytes(int G) {
  size_t maps = (size_t)G * 2 * sizeof(CUtensorMap);
  size_t descs = (size_t)G * sizeof(GroupDesc);
  size_t starts = (size_t)(G + 1) * sizeof(int);
  size_t cmaps = (size_t)G * sizeof(CUtensorMap);   // C maps of the TMA-store epilogue (GEMM groups)
  return maps + ((descs + 127) / 128 * 128) + ((starts + 127) / 128 * 128) + cmaps;
}

nk_schedule grouped_schedule(const nk_schedule* user) {
  nk_schedule s{128, 128, 64, 1, 0, 1};
  if (user) {
    if (user->tile_n) s.tile_n = user->tile_n;
    if (user->stages) s.stages = user->stages;
    if (user->cluster) s.cluster = user->cluster;
    if (user->split_k) s.split_k = user->split_k;
    if (user->tile_m) s.tile_m = user->tile_m;
    if (user->tile_k) s.tile_k = user->tile_k;
  }
  if (s.stages == 0) {
    s.stages = 2;
    while (s.stages < 8 && smem_bytes(TC_BF16, s.tile_n, s.stages + 1) <= kMaxSmem) ++s.stages;
  }
  return s;
}

// Fills `host` (grouped_bytes(G) bytes) with the table for a device buffer at
// `dev_base`, and the launch parameters.
nk_status build_grouped(int G, const nk_gemm_group* groups, int precision, const nk_schedule* user,
                        void* dev_base, std::vector<uint8_t>& host, nk_grouped_plan& plan) {
  if (G < 0) return fail(NK_ERR_INVALID_ARG, "negative group count");
  if (G > 0 && !groups) return fail(NK_ERR_INVALID_ARG, "groups is NULL");
  if (precision != NK_PREC_BF16)
    return fail(NK_ERR_UNSUPPORTED, "grouped GEMM runs BF16 operands (NK_PREC_BF16) only");
  const nk_schedule s = grouped_schedule(user);
  // tile_m 128 on one CTA, or tile_m 256 on a CTA pair (each CTA holds its
  // 128 rows of A and half of the B tile)
  const bool pair = s.tile_m == 256 && s.cluster == 2;
  if (s.split_k != 1 || s.tile_n == 512 || !(pair || (s.tile_m == 128 && s.cluster == 1)) ||
      !tc_schedule_valid(TC_BF16, s, 1, 1, 1))
    return fail(NK_ERR_NO_SCHEDULE,
                "grouped schedule needs split_k 1 and tile_m 128 on one CTA or 256 on a CTA pair");
  const int rows = pair ? 2 * kBM : kBM;   // GEMM rows of one unit
  int sms = 0;
  nk_status st = require_device(&sms);
  if (st != NK_OK) return st;
  // A single-row operand's leading dimension is never stepped over; give TMA
  // a legal one (row padded to 16 bytes) whatever the caller passed.
  auto ld_a = [](const nk_gemm_group& q) { return q.M == 1 ? (int64_t)(q.K + 7) / 8 * 8 : q.lda; };
  auto ld_b = [](const nk_gemm_group& q) { return q.N == 1 ? (int64_t)(q.K + 7) / 8 * 8 : q.ldb; };
  auto ld_c = [](const nk_gemm_group& q) { return q.M == 1 ? (int64_t)(q.N + 3) / 4 * 4 : q.ldc; };
  for (int g = 0; g < G; ++g) {
    nk_gemm_group q = groups[g];
    q.lda = ld_a(q); q.ldb = ld_b(q); q.ldc = ld_c(q);
    if (q.M < 1 || q.N < 1 || q.K < 1) return fail(NK_ERR_INVALID_ARG, "group %d has an empty extent", g);
    if (!q.A || !q.Bt || !q.C) return fail(NK_ERR_INVALID_ARG, "group %d has a NULL pointer", g);
    if (q.lda < q.K || q.ldb < q.K || q.ldc < q.N)
      return fail(NK_ERR_INVALID_ARG, "group %d: leading dimension smaller than the row", g);
    if ((q.lda * 2) % 16 || (q.ldb * 2) % 16 || (reinterpret_cast<uintptr_t>(q.A) & 15) ||
        (reinterpret_cast<uintptr_t>(q.Bt) & 15))
      return fail(NK_ERR_MISALIGNED, "group %d: BF16 operands need 16-byte aligned rows", g);
  }
  std::vector<int> order(G);
  for (int g = 0; g < G; ++g) order[g] = g;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return groups[a].K > groups[b].K; });
  host.assign(grouped_bytes(G), 0);
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(host.data());
  const size_t off_desc = (size_t)G * 2 * sizeof(CUtensorMap);
  const size_t off_start = off_desc + ((size_t)G * sizeof(GroupDesc) + 127) / 128 * 128;
  GroupDesc* descs = reinterpret_cast<GroupDesc*>(host.data() + off_desc);
  int* starts = reinterpret_cast<int*>(host.data() + off_start);
  const size_t off_cmap = off_start + ((size_t)(G + 1) * sizeof(int) + 127) / 128 * 128;
  CUtensorMap* cmaps = reinterpret_cast<CUtensorMap*>(host.data() + off_cmap);
  bool cvec = true, cvec32 = true, ctma = true;
  auto fn = encode_fn();
  int64_t total = 0;
  for (int i = 0; i < G; ++i) {
    nk_gemm_group q = groups[order[i]];
    q.lda = ld_a(q); q.ldb = ld_b(q); q.ldc = ld_c(q);
    if ((st = make_kmajor_map(&maps[2 * i], false, q.A, q.M, q.K, q.lda, kBM)) != NK_OK) return st;
    if ((st = make_kmajor_map(&maps[2 * i + 1], false, q.Bt, q.N, q.K, q.ldb, pair ? s.tile_n / 2 : s.tile_n)) !=
        NK_OK)
      return st;
    GroupDesc& d = descs[i];
    d.M = q.M; d.N = q.N; d.K = q.K;
    d.tiles_n = (q.N + s.tile_n - 1) / s.tile_n;
    d.C = q.C;
    d.ldc = q.ldc;
    d.beta = q.accumulate ? 1.f : 0.f;
    d.kblocks = (q.K + 63) / 64;
    starts[i] = (int)total;
    total += (int64_t)((q.M + rows - 1) / rows) * d.tiles_n;
    if (total > INT32_MAX) return fail(NK_ERR_UNSUPPORTED, "too many tiles");
    cvec = cvec && ((reinterpret_cast<uintptr_t>(q.C) & 15) == 0) && (q.ldc % 4 == 0);
    cvec32 = cvec32 && ((reinterpret_cast<uintptr_t>(q.C) & 31) == 0) && (q.ldc % 8 == 0);
    // TMA-store epilogue: every group a plain overwrite of a 16-byte aligned C
    // whose rows end on 16-byte boundaries (a TMA store clips the innermost
    // dimension to 16-byte granules only)
    ctma = ctma && fn && !q.accumulate && ((reinterpret_cast<uintptr_t>(q.C) & 15) == 0) && (q.ldc * 4) % 16 == 0 &&
           q.N % 4 == 0;
    if (ctma) {
      cuuint64_t dims[2] = {(cuuint64_t)q.N, (cuuint64_t)q.M};
      cuuint64_t strides[1] = {(cuuint64_t)(q.ldc * 4)};
      cuuint32_t box[2] = {32, 32};
      cuuint32_t es[2] = {1, 1};
      ctma = fn(&cmaps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, q.C, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
  }
  starts[G] = (int)total;
  TcParams& p = plan.p;
  memset(&p, 0, sizeof p);
  p.bn = s.tile_n;
  p.stages = s.stages;
  p.units = (int)total;
  p.splits = 1;
  p.alpha = 1.f;
  p.budget = wait_budget();
  p.c_vec = cvec ? 1 : 0;
  p.c_vec32 = cvec32 ? 1 : 0;
  p.G = G;
  uint8_t* db = static_cast<uint8_t*>(dev_base);
  p.gmaps = reinterpret_cast<const CUtensorMap*>(db);
  p.groups = reinterpret_cast<const GroupDesc*>(db + off_desc);
  p.tile_start = reinterpret_cast<const int*>(db + off_start);
  plan.units = (int)total;
  plan.pair = pair;
  plan.ep8 = ctas_per_sm(TC_BF16, s) == 1;
  plan.smem = smem_of(TC_BF16, s);
  // eight epilogue warps stage through eight boxes (four are budgeted)
  if (plan.ep8 && plan.smem + 4 * kStageBox > kMaxSmem) plan.ep8 = false;
  if (plan.ep8) plan.smem += 4 * kStageBox;
  if (ctma) {
    p.gcmaps = reinterpret_cast<const CUtensorMap*>(db + off_cmap);
    p.c_tma = 1;
  }
  const int CL = pair ? 2 : 1;
  int grid = sms * ctas_per_sm(TC_BF16, s) / CL * CL;
  if (grid > plan.units * CL) grid = plan.units * CL;
  plan.grid = grid < CL ? CL : grid;
  return NK_OK;
}

// Grouped convolutions: each group a linalg.conv_2d_nhwc_hwcf on BF16 NHWC
// input and packed BF16 weights, with its own output tiling (ConvTile), 4-D
// input and 3-D weight maps, bias and ReLU in the device table.
nk_status build_grouped_conv(int G, const nk_conv_group* groups, const nk_schedule* user, void* dev_base,
                             std::vector<uint8_t>& host, nk_grouped_plan& plan) {
  if (G < 0) return fail(NK_ERR_INVALID_ARG, "negative group count");
  if (G > 0 && !groups) return fail(NK_ERR_INVALID_ARG, "groups is NULL");
  const nk_schedule s = grouped_schedule(user);
  if (s.tile_m != 128 || s.cluster != 1 || s.split_k != 1 || s.tile_n == 512 || s.tile_k != 64 ||
      !tc_schedule_valid(TC_BF16, s, 1, 1, 1))
    return fail(NK_ERR_NO_SCHEDULE, "grouped conv schedule needs tile_m 128, tile_k 64, cluster 1, split_k 1");
  int sms = 0;
  nk_status st = require_device(&sms);
  if (st != NK_OK) return st;
  std::vector<TcConv> convs(G);
  std::vector<int> kblocks(G);
  for (int i = 0; i < G; ++i) {
    const nk_conv_group& q = groups[i];
    const nk_tensor &I = q.I, &W = q.W, &O = q.O;
    if (I.rank != 4 || W.rank != 4 || O.rank != 4 || I.dtype != NK_BF16 || W.dtype != NK_BF16 || O.dtype != NK_F32)
      return fail(NK_ERR_UNSUPPORTED, "conv group %d: BF16 NHWC I, packed BF16 W and FP32 NHWC O", i);
    for (int d = 0; d < 2; ++d)
      if (q.stride[d] < 1 || q.dilation[d] < 1) return fail(NK_ERR_INVALID_ARG, "conv group %d: stride, dilation", i);
    for (int d = 0; d < 4; ++d)
      if (q.pad[d] < 0) return fail(NK_ERR_INVALID_ARG, "conv group %d: negative padding", i);
    ConvGeom g{};
    g.n = (int)I.shape[0]; g.h = (int)I.shape[1]; g.w = (int)I.shape[2]; g.c = (int)I.shape[3];
    g.kh = (int)W.shape[0]; g.kw = (int)W.shape[1];
    g.sh = (int)q.stride[0]; g.sw = (int)q.stride[1]; g.dh = (int)q.dilation[0]; g.dw = (int)q.dilation[1];
    g.pt = (int)q.pad[0]; g.pl = (int)q.pad[2];
    const int64_t oh = (g.h + q.pad[0] + q.pad[1] - g.dh * (g.kh - 1) - 1) / g.sh + 1;
    const int64_t ow = (g.w + q.pad[2] + q.pad[3] - g.dw * (g.kw - 1) - 1) / g.sw + 1;
    if (oh < 1 || ow < 1 || g.n < 1 || g.c < 1 || W.shape[3] < 1)
      return fail(NK_ERR_INVALID_ARG, "conv group %d: empty problem", i);
    if (W.shape[2] != g.c) return fail(NK_ERR_INVALID_ARG, "conv group %d: I channels != W channels", i);
    if (O.shape[0] != g.n || O.shape[1] != oh || O.shape[2] != ow || O.shape[3] != W.shape[3])
      return fail(NK_ERR_INVALID_ARG, "conv group %d: O must be [%d,%lld,%lld,%lld]", i, g.n, (long long)oh,
                  (long long)ow, (long long)W.shape[3]);
    if (g.sh > 8 || g.sw > 8) return fail(NK_ERR_UNSUPPORTED, "conv group %d: stride above 8", i);
    g.oh = (int)oh; g.ow = (int)ow;
    g.sin_n = I.stride[0]; g.sin_h = I.stride[1]; g.sin_w = I.stride[2];
    const int64_t ldw = W.stride[1], sF = W.stride[3];
    if (I.stride[3] != 1 || W.stride[2] != 1 || ldw < g.c || ldw % 8 || W.stride[0] != W.shape[1] * ldw ||
        sF % 8 || sF < W.shape[0] * W.shape[1] * ldw)
      return fail(NK_ERR_UNSUPPORTED, "conv group %d: I needs unit channel stride, W the packed layout", i);
    if (O.stride[3] != 1 || O.stride[2] != O.shape[3] || O.stride[1] != O.shape[2] * O.stride[2] ||
        O.stride[0] != O.shape[1] * O.stride[1])
      return fail(NK_ERR_UNSUPPORTED, "conv group %d: O must be contiguous NHWC", i);
    if ((g.sin_w * 2) % 16 || (g.sin_h * 2) % 16 || (g.sin_n * 2) % 16 ||
        (reinterpret_cast<uintptr_t>(I.ptr) & 15) || (reinterpret_cast<uintptr_t>(W.ptr) & 15))
      return fail(NK_ERR_MISALIGNED, "conv group %d: operands need 16-byte aligned bases and rows", i);
    if ((int64_t)g.n * g.oh * g.ow > INT32_MAX) return fail(NK_ERR_UNSUPPORTED, "conv group %d: too large", i);
    TcConv& c = convs[i];
    c.kind = TC_BF16;
    c.I = I.ptr; c.sI_n = g.sin_n; c.sI_h = g.sin_h; c.sI_w = g.sin_w;
    c.Wt = W.ptr; c.ldw = ldw; c.sW_f = sF;
    c.g = g;
    c.F = (int)W.shape[3];
    c.O = static_cast<float*>(O.ptr);
    kblocks[i] = g.kh * g.kw * ((g.c + 63) / 64);
  }
  std::vector<int> order(G);
  for (int g = 0; g < G; ++g) order[g] = g;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return kblocks[a] > kblocks[b]; });
  host.assign(grouped_bytes(G), 0);
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(host.data());
  const size_t off_desc = (size_t)G * 2 * sizeof(CUtensorMap);
  const size_t off_start = off_desc + ((size_t)G * sizeof(GroupDesc) + 127) / 128 * 128;
  GroupDesc* descs = reinterpret_cast<GroupDesc*>(host.data() + off_desc);
  int* starts = reinterpret_cast<int*>(host.data() + off_start);
  bool cvec = true;
  int64_t total = 0;
  for (int i = 0; i < G; ++i) {
    const int gi = order[i];
    const TcConv& c = convs[gi];
    const ConvTile t = choose_conv_tile(c.g, TC_BF16);
    if ((st = make_conv_maps(&maps[2 * i], &maps[2 * i + 1], c, t, s.tile_n)) != NK_OK) return st;
    GroupDesc& d = descs[i];
    d.M = c.g.n * c.g.oh * c.g.ow;
    d.N = c.F;
    d.K = c.g.kh * c.g.kw * c.g.c;
    d.tiles_n = (c.F + s.tile_n - 1) / s.tile_n;
    d.C = c.O;
    d.ldc = c.F;
    d.beta = groups[gi].accumulate ? 1.f : 0.f;
    d.kblocks = kblocks[gi];
    d.bias = groups[gi].bias;
    d.relu = groups[gi].relu;
    d.cv = t;
    starts[i] = (int)total;
    total += (int64_t)t.tiles_w * t.tiles_h * ((c.g.n + t.NB - 1) / t.NB) * d.tiles_n;
    if (total > INT32_MAX) return fail(NK_ERR_UNSUPPORTED, "too many tiles");
    cvec = cvec && ((reinterpret_cast<uintptr_t>(c.O) & 15) == 0) && (c.F % 4 == 0);
  }
  starts[G] = (int)total;
  TcParams& p = plan.p;
  memset(&p, 0, sizeof p);
  p.bn = s.tile_n;
  p.stages = s.stages;
  p.units = (int)total;
  p.splits = 1;
  p.alpha = 1.f;
  p.budget = wait_budget();
  p.c_vec = cvec ? 1 : 0;
  p.G = G;
  uint8_t* db = static_cast<uint8_t*>(dev_base);
  p.gmaps = reinterpret_cast<const CUtensorMap*>(db);
  p.groups = reinterpret_cast<const GroupDesc*>(db + off_desc);
  p.tile_start = reinterpret_cast<const int*>(db + off_start);
  plan.units = (int)total;
  plan.pair = false;
  plan.conv = true;
  plan.smem = smem_of(TC_BF16, s);
  int grid = sms * ctas_per_sm(TC_BF16, s);
  if (grid > plan.units) grid = plan.units;
  plan.grid = grid < 1 ? 1 : grid;
  return NK_OK;
}

}  // namespace
}  // namespace nk

using namespace nk;

extern "C" {

nk_status nk_grouped_workspace_size(int32_t G, const nk_gemm_group* groups, int32_t precision,
                                    const nk_schedule* sched, size_t* bytes) {
  (void)groups; (void)precision; (void)sched;
  if (!bytes) return fail(NK_ERR_INVALID_ARG, "bytes is NULL");
  if (G < 0) return fail(NK_ERR_INVALID_ARG, "negative group count");
  *bytes = grouped_bytes(G);
  return NK_OK;
}

namespace nk {
namespace {
// The group of every unit, from the tile prefix sums of the host table.
nk_status attach_unit_map(nk_grouped_plan& plan, const std::vector<uint8_t>& host, int G) {
  if (plan.units <= 0) return NK_OK;
  const size_t off_start = (size_t)G * 2 * sizeof(CUtensorMap) + ((size_t)G * sizeof(GroupDesc) + 127) / 128 * 128;
  const int* starts = reinterpret_cast<const int*>(host.data() + off_start);
  std::vector<int> m((size_t)plan.units);
  int g = 0;
  for (int u = 0; u < plan.units; ++u) {
    while (g + 1 < G && starts[g + 1] <= u) ++g;
    m[(size_t)u] = g;
  }
  cudaError_t e = cudaMalloc(&plan.umap, m.size() * sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(unit map)");
  e = cudaMemcpy(plan.umap, m.data(), m.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(plan.umap); plan.umap = nullptr; return cuda_fail(e, "cudaMemcpy(unit map)"); }
  plan.p.unit_group = plan.umap;
  return NK_OK;
}
}  // namespace
}  // namespace nk

nk_status nk_grouped_plan_create(int32_t G, const nk_gemm_group* groups, int32_t precision,
                                 const nk_schedule* sched, nk_grouped_plan** out) {
  nk::NvtxRange nvtx_range_("nk_grouped_plan_create");
  if (!out) return fail(NK_ERR_INVALID_ARG, "plan is NULL");
  *out = nullptr;
  auto* plan = new nk_grouped_plan();
  void* dev = nullptr;
  const size_t bytes = grouped_bytes(G);
  cudaError_t e = cudaMalloc(&dev, bytes > 0 ? bytes : 1);
  if (e != cudaSuccess) { delete plan; return cuda_fail(e, "cudaMalloc(grouped plan)"); }
  std::vector<uint8_t> host;
  nk_status s = build_grouped(G, groups, precision, sched, dev, host, *plan);
  if (s == NK_OK && bytes) {
    e = cudaMemcpy(dev, host.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpy(grouped plan)");
  }
  if (s == NK_OK) s = nk::attach_unit_map(*plan, host, G);
  if (s != NK_OK) { cudaFree(dev); delete plan; return s; }
  plan->dev = dev;
  plan->owned = true;
  *out = plan;
  return NK_OK;
}

nk_status nk_conv2d_grouped_plan_create(int32_t G, const nk_conv_group* groups, const nk_schedule* sched,
                                        nk_grouped_plan** out) {
  nk::NvtxRange nvtx_range_("nk_conv2d_grouped_plan_create");
  if (!out) return fail(NK_ERR_INVALID_ARG, "plan is NULL");
  *out = nullptr;
  auto* plan = new nk_grouped_plan();
  void* dev = nullptr;
  const size_t bytes = grouped_bytes(G);
  cudaError_t e = cudaMalloc(&dev, bytes > 0 ? bytes : 1);
  if (e != cudaSuccess) { delete plan; return cuda_fail(e, "cudaMalloc(grouped conv plan)"); }
  std::vector<uint8_t> host;
  nk_status s = build_grouped_conv(G, groups, sched, dev, host, *plan);
  if (s == NK_OK && bytes) {
    e = cudaMemcpy(dev, host.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpy(grouped conv plan)");
  }
  if (s == NK_OK) s = nk::attach_unit_map(*plan, host, G);
  if (s != NK_OK) { cudaFree(dev); delete plan; return s; }
  plan->dev = dev;
  plan->owned = true;
  *out = plan;
  return NK_OK;
}

nk_status nk_grouped_plan_run(const nk_grouped_plan* plan, void* stream) {
  nk::NvtxRange nvtx_range_("nk_grouped_plan_run");
  if (!plan) return fail(NK_ERR_INVALID_ARG, "plan is NULL");
  if (plan->units == 0) return NK_OK;
  if (plan->conv)
    return launch<TC_BF16, 1, true, true>(plan->p, plan->grid, plan->smem, static_cast<cudaStream_t>(stream));
  return run_grouped_gemm(*plan, static_cast<cudaStream_t>(stream));
}

nk_status nk_grouped_plan_destroy(nk_grouped_plan* plan) {
  if (!plan) return NK_OK;
  if (plan->owned && plan->dev) cudaFree(plan->dev);
  if (plan->umap) cudaFree(plan->umap);
  delete plan;
  return NK_OK;
}

nk_status nk_batch_matmul_grouped(int32_t G, const nk_gemm_group* groups, int32_t precision,
                                  const nk_schedule* sched, void* ws, size_t ws_bytes, void* stream) {
  nk::NvtxRange nvtx_range_("nk_batch_matmul_grouped");
  const size_t bytes = grouped_bytes(G);
  if (G > 0 && (!ws || ws_bytes < bytes))
    return fail(NK_ERR_WORKSPACE, "grouped GEMM needs %zu bytes of workspace", bytes);
  if (ws && (reinterpret_cast<uintptr_t>(ws) & 127))
    return fail(NK_ERR_MISALIGNED, "grouped workspace must be 128-byte aligned");
  nk_grouped_plan plan;
  std::vector<uint8_t> host;
  nk_status s = build_grouped(G, groups, precision, sched, ws, host, plan);
  if (s != NK_OK || plan.units == 0) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(ws, host.data(), bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(grouped table)");
  // a pageable source is staged before cudaMemcpyAsync returns, so `host` may go
  return run_grouped_gemm(plan, st);
}

}  // extern "C"
