// K1 (tensor-core form): the probe blend of Section 3.2 of arXiv 2103.05875 as
// a tcgen05 contraction with a fused epilogue, for sm_103a.
//
// The blend is a dense contraction because every probe of a volume shares the
// frame's ray directions: per texel t and probe row x (a colour channel, d or
// d^2), acc[t, x] = sum_r W[t, r] x[r]. Texels form the MMA's M dimension (one
// tensor-memory lane per texel), the probe rows of a work item (np <= 32
// probes per row group) its N dimension, rays its K dimension:
//
//   A (shared memory, K-major): the weights from the weights kernel, one
//     combined texel list in 128-row tiles: visibility texels in rows
//     0..Tv-1, colour texels from the next multiple of 8. The weights kernel
//     writes each K chunk as the exact (swizzled) shared-memory image of its
//     tiles, so a chunk arrives with one bulk copy per plane; rows past the
//     texels are zero and the lanes they produce are ignored.
//   B (shared memory, K-major, one row per probe row, row groups of 32):
//     [ d | d^2 (hi) | d^2 lo (16-bit forms) | R | G | B ]
//     d and the colour planes come straight from HBM by TMA; d^2 is formed on
//     chip by two converter warps (its rounding to the operand format is split
//     into hi + lo parts so that it costs no accuracy).
//   D (tensor memory, FP32): one MMA per tile and K step, with the B rows its
//     texels need: the visibility rows, the colour rows, or all of B for the
//     tile that holds both. An MMA with M = 128 costs the same up to N = 112,
//     so a few wide MMAs beat many narrow ones.
//
// Operand forms (pv_desc.operand_fmt):
//   F16  kind::f16, binary16 inputs; visibility weights scaled by 2^15 and
//        d^2 by 2^-4 (both undone exactly) to stay in range.
//   BF16 kind::f16 with bfloat16; W = W_hi + W_lo (two MMAs) because one
//        bfloat16 weight only carries 8 bits.
//   F32  kind::tf32, float32 inputs; x = x_hi + x_lo and W = W_hi + W_lo with
//        TF32 parts, three MMAs (hi*hi + hi*lo + lo*hi) recover float32
//        accuracy.
//
// Warp roles (512 threads, one CTA per SM, persistent over work items):
//   warp 0     producer: ray tiles (TMA) and weight images (bulk copies) into
//              a ring of stages
//   warp 1     TMEM allocation and the single MMA-issuing thread
//   warps 2-3  converters: d^2 rows, TF32 hi/lo split
//   warps 4-15 epilogue. A lane owns one texel (its TMEM lane) and a task is
//              one channel of a 32-texel group over the item's probe rows,
//              loaded from TMEM eight columns at a time. Per row the fused
//              work of Sections 3.2-3.4 runs with every per-texel constant in
//              registers (weight-sum normalisation, hysteresis, storage
//              rounding, transmitted code, comparison with the
//              last-transmitted code, changed flags) on the item's tiles in
//              shared memory; each new code replaces the last one in the code
//              tile. The guard band is copied afterwards for all rows, and the
//              tiles and the current codes (which select/pack sends) go back
//              to HBM by bulk copies. The item's old texels and codes are
//              streamed in by bulk copies while the previous item is still
//              being processed; when every CTA has one item and the separate
//              layout would leave a shallow ring, they live in the ring's
//              first stages instead and are loaded once those stages are free.
// Programmatic dependent launch: the kernel lets its successor launch at its
// start and runs its set-up (barriers, TMEM, tensor-map prefetch, parameter
// reads) before waiting for its predecessor; each role waits only before its
// first read of memory a predecessor wrote.
// Accumulators are double-buffered in TMEM (columns 0 and 256) when a buffer
// needs at most 256 columns, so an item's epilogue overlaps the next item's
// MMAs. Every mbarrier wait is
// bounded in time; on expiry the kernel raises the volume's error word and
// every role leaves its loop, so no wait can hang the GPU.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdio.h>
#include <type_traits>
#include <stdlib.h>
#include <string.h>

#include "pv_codes.cuh"
#include "pv_internal.h"

namespace {

enum Form { kF16 = 0, kBF16 = 1, kF32 = 2 };

constexpr int NT = 512;
constexpr int EPI_WARPS = 12;            // warps 4..15, three per TMEM lane quarter
constexpr int EPI_THREADS = 32 * EPI_WARPS;
// bytes per K-chunk row in shared memory: 64 (SWIZZLE_64B) for every form,
// i.e. 32 rays per chunk for 16-bit operands and 16 for TF32. Per-chunk
// latency dominates the main loop, so fewer, larger chunks win over a deeper
// ring (the FP32 form then fits two stages)
template <int FORM>
__host__ __device__ constexpr int row_bytes() { return 64; }
constexpr int GRP = 32;                  // probe rows per row group of the B tile
constexpr int MT = 128;                  // texels per MMA tile (M)
constexpr int kMaxStages = 8;            // deepest ring of K stages (shared memory permitting)
enum TileKind { kTileVis = 0, kTileCol = 1, kTileBoth = 2 };
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s
// binary16 operand form: d^2 enters the MMA scaled by 2^-4 (exact), which
// keeps the high part of d^2 for hit distances up to 2^10 in binary16 range
constexpr float kD2ScaleF16 = 0.0625f;

struct TcParams {
  pv_dev k;
  int np, items, iters, stages, kc;
  int ntiles, bufcols, nbuf;             // 128-row texel tiles; TMEM columns a buffer uses
  int vb;                                // tile row of colour texel 0 (visibility texels: rows 0..Tv-1)
  int nvc;                               // B rows (and TMEM columns) of the visibility block
  int crow;                              // first B row of the colour block
  int a_rows;                            // rows of the ray (B) tile
  int tkind[4], tbase[4];                // per tile: which B rows (kTileVis/Col/Both); first TMEM column
  uint32_t tidesc[4];
  int off_a_lo, off_w, off_w_lo, stage_bytes;
  int off_state, off_last, off_rsum, off_pos, off_gb, off_flags, off_bar;
  int alias_stages;                      // > 0: one item per CTA, whose old texels and codes live in
                                         // the first alias_stages stages of the ring (loaded at its end)
  int gb_c, gb_v;                        // guard-band texels per tile: 4n + 4
  uint32_t stage_tx, w_tx;               // bytes per stage: all, weight tiles only
};

// One volume of a launch: its tensor maps, its buffers and its work items.
// Every volume of a launch shares the tile shapes, state and operand formats
// (the fields of TcParams); rays and probe counts may differ.
struct BlendVol {
  CUtensorMap rad, dist;
  pv_dev k;                              // k.w_op: the weight tile images, one bulk copy per chunk and plane
  int item0;                             // first work item of the volume in the launch
  int nchunks;                           // ray chunks of kc rays
};

template <int MAXV>
struct BlendArgs {
  TcParams tp;                           // tp.k: shape of the volumes, error word
  int nvol;
  BlendVol v[MAXV];
};

// Volume of global work item `item` (items are numbered volume by volume).
template <int MAXV>
__device__ __forceinline__ int vol_of(const BlendArgs<MAXV>& a, int item) {
  int v = 0;
  while (v + 1 < a.nvol && item >= a.v[v + 1].item0) ++v;
  return v;
}

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000000;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false if it expired or
// another role already gave up.
__device__ __noinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = gtime();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 128; ++i)
      if (mbar_try(b, parity)) return true;
    if (*(volatile int*)err) return false;
    if (gtime() - t0 > kWaitNs) {
      atomicExch(err, 1);
      return false;
    }
  }
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 384;" ::: "memory"); }
__device__ __forceinline__ void conv_bar() { asm volatile("bar.sync 2, 64;" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
template <int FORM>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (FORM == kF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// 8 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major rows of RB bytes with the matching
// swizzle (64 B: SWIZZLE_64B, 32 B: SWIZZLE_32B), 8-row groups RB*8 bytes apart
// (SBO); LBO unused for these layouts; descriptor version 1.
template <int RB>
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  const uint64_t a = smem_u32(p);
  uint64_t d = 0;
  d |= (a & 0x3FFFFull) >> 4;            // start address
  d |= (uint64_t)1 << 16;                // leading byte offset (16 B, ignored)
  d |= (uint64_t)((RB * 8) >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;                // version
  d |= (uint64_t)(RB == 64 ? 4 : 6) << 61;   // SWIZZLE_64B / SWIZZLE_32B
  return d;
}

// ------------------------------------------------------------------ epilogue
// State format as a compile-time choice: 0 binary16, 1 binary32.
template <int SF>
struct StateOps {
  static constexpr int SB = SF == 0 ? 2 : 4;         // bytes per stored texel
  static __device__ __forceinline__ float value(uint32_t b) {
    return SF == 0 ? __half2float(__ushort_as_half((unsigned short)b)) : __uint_as_float(b);
  }
  static __device__ __forceinline__ uint32_t bits(float v) {
    return SF == 0 ? (uint32_t)__half_as_ushort(__float2half_rn(v)) : __float_as_uint(v);
  }
};

// Shared-memory loads and stores of 2- or 4-byte elements at 32-bit shared
// addresses.
template <int B>
__device__ __forceinline__ uint32_t lds(uint32_t a) {
  uint32_t v;
  if constexpr (B == 2) asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a));
  else asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
// Store only where `on` is set. The predicate lives inside the instruction,
// so a row's store does not split the surrounding code into branches and the
// rows of a group stay free to overlap.
template <int B>
__device__ __forceinline__ void sts_if(bool on, uint32_t a, uint32_t v) {
  if constexpr (B == 2)
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q st.shared.u16 [%0], %1;\n}\n" ::"r"(a),
                 "h"((unsigned short)v), "r"((uint32_t)on));
  else
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q st.shared.u32 [%0], %1;\n}\n" ::"r"(a), "r"(v),
                 "r"((uint32_t)on));
}

// Transmitted code of a stored texel (Section 3.4): visibility as binary16
// bits, colour as UF10 or UNORM10.
template <int SF, int KIND, bool VIS>
__device__ __forceinline__ uint32_t texel_code(uint32_t b) {
  if (VIS) return SF == 0 ? b : (uint32_t)__half_as_ushort(__float2half_rn(__uint_as_float(b)));
  if (KIND == PV_CODE_UNORM10) return pv::unorm10_from_float(StateOps<SF>::value(b));
  return SF == 0 ? pv::uf10_from_half_bits(b) : pv::uf10_from_float_bits(b);
}

// One epilogue task: the 32 accumulator columns at taddr (plus those at
// taddr_lo for an operand split into two parts) are probe rows p = 0..31 of
// one channel, and this lane's TMEM lane is one texel, whose
// stored value in row p sits at s_tile + p * row_b and whose last-transmitted
// code at s_code + p * code_b (shared addresses). Rows go in groups of U: one
// TMEM load per group, then the group's old texels and last codes, then the
// arithmetic and stores. The group loop stays rolled so that the epilogue's
// code is small enough to stay in the instruction cache. Returns the rows
// whose transmitted code changed as a bit mask (bit p).
template <int SF, int KIND, bool VIS, bool LO>
__device__ __forceinline__ uint32_t epi_task(uint32_t taddr, uint32_t taddr_lo, bool has, uint32_t s_tile,
                                             uint32_t s_code, float rS, float h, float omh, float scale,
                                             uint32_t row_b, uint32_t code_b, int npi) {
  constexpr int SB = StateOps<SF>::SB;
  constexpr int U = 8;
  const float c = omh * (rS * scale);
  const bool upd = rS > 0.0f;
  uint32_t ro[U], co[U];                             // row offsets within a group
#pragma unroll
  for (int u = 0; u < U; ++u) {
    ro[u] = (uint32_t)u * row_b;
    co[u] = (uint32_t)u * code_b;
  }
  uint32_t m = 0;
#pragma unroll 1
  for (int g = 0; g < npi; g += U) {
    float v[U];
    tmem_ld8(taddr + (uint32_t)g, v);
    if (LO) {                                          // accumulator of the operand's low part
      float w[U];
      tmem_ld8(taddr_lo + (uint32_t)g, w);
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] += w[u];
    }
    const uint32_t tb = s_tile + (uint32_t)g * row_b, cb = s_code + (uint32_t)g * code_b;
    // rows of this group inside the item (none for lanes without a texel);
    // rows past the item still load (the shared regions are padded for it)
    const int lim = has ? npi - g : 0;
    uint32_t old[U], last[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      old[u] = lds<SB>(tb + ro[u]);
      last[u] = lds<2>(cb + co[u]);
    }
    uint32_t mg = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool live = u < lim;
      const float nv = fmaf(h, StateOps<SF>::value(old[u]), v[u] * c);
      const uint32_t nb = upd ? StateOps<SF>::bits(nv) : old[u];
      sts_if<SB>(live, tb + ro[u], nb);
      const uint32_t code = texel_code<SF, KIND, VIS>(nb);
      mg |= (live && code != last[u]) ? (1u << u) : 0u;
      sts_if<2>(live, cb + co[u], code);             // the code tile now holds the current codes
    }
    m |= mg << g;
  }
  return m;
}

// Shared-memory addresses and sizes the epilogue tasks of an item use.
struct EpiCtx {
  uint32_t s_rsum, s_pos;                // per-texel tables: colour texels first, then visibility
  uint32_t s_st_c, s_st_v, s_ls_c, s_ls_v;
  int sc_stride, sv_stride, lc_stride, lv_stride;
  int Tc, Tv, np, npi;
  float h, omh, d2_scale;
};

// Tasks of a group of 32 texels of one texture for this warp: the channels
// (32 TMEM columns each from `col`) dealt round-robin to the three warps of
// the lane quarter. `t0` is the texture's texel index of lane 0 (lanes
// outside 0..T-1 have no texel).
template <int SF, int KIND, bool VIS, bool D2LO>
__device__ __forceinline__ uint32_t epi_group(const EpiCtx& x, uint32_t col, int t0, int lane, int slot,
                                              int& task) {
  constexpr int NCH = VIS ? 2 : 3;
  constexpr int SB = StateOps<SF>::SB;
  const int T = VIS ? x.Tv : x.Tc;
  const int t = t0 + lane;
  const bool has = t >= 0 && t < T;
  const int tt = has ? t : (t0 < 0 ? 0 : t0);      // a valid texel for the loads of idle lanes
  const uint32_t ti = (uint32_t)(VIS ? x.Tc + tt : tt);
  const float rS = has ? __uint_as_float(lds<4>(x.s_rsum + 4u * ti)) : 0.0f;
  const uint32_t pos = lds<2>(x.s_pos + 2u * ti);
  const int tile_elems = VIS ? x.sv_stride : x.sc_stride, code_elems = VIS ? x.lv_stride : x.lc_stride;
  const uint32_t row_b = (uint32_t)tile_elems * SB, code_b = (uint32_t)code_elems * 2;
  const uint32_t s_tiles = VIS ? x.s_st_v : x.s_st_c, s_codes = VIS ? x.s_ls_v : x.s_ls_c;
  uint32_t m = 0;
#pragma unroll 1
  for (int ch = 0; ch < NCH; ++ch) {
    const int mine = task++ % 3;
    if (mine != slot) continue;
    const uint32_t st = s_tiles + (uint32_t)(ch * x.np) * row_b + pos * SB;
    const uint32_t sc = s_codes + (uint32_t)(ch * x.np) * code_b + (uint32_t)tt * 2;
    const uint32_t c = col + GRP * ch;
    if (VIS && ch == 1) {
      if (D2LO) m |= epi_task<SF, KIND, VIS, true>(c, c + GRP, has, st, sc, rS, x.h, x.omh, x.d2_scale, row_b, code_b, x.npi);
      else m |= epi_task<SF, KIND, VIS, false>(c, 0, has, st, sc, rS, x.h, x.omh, x.d2_scale, row_b, code_b, x.npi);
    } else {
      m |= epi_task<SF, KIND, VIS, false>(c, 0, has, st, sc, rS, x.h, x.omh, 1.0f, row_b, code_b, x.npi);
    }
  }
  return m;
}

// All tasks of one item in one TMEM buffer (lane quarter of this warp, TMEM
// address `tq` of column 0): per 128-row tile, the visibility texels and the
// colour texels that fall into this quarter. Returns the changed-probe masks
// (colour, visibility).
template <int SF, int KIND, bool D2LO>
__device__ __forceinline__ void epi_item(const TcParams& tp, const EpiCtx& x, uint32_t tq, int quarter, int lane,
                                         int slot, uint32_t& mc, uint32_t& mv) {
  int task = 0;
  mc = 0;
  mv = 0;
  for (int j = 0; j < tp.ntiles; ++j) {
    const int r0 = MT * j + GRP * quarter;             // tile row of lane 0
    const uint32_t col = tq + (uint32_t)tp.tbase[j];
    if (tp.tkind[j] != kTileCol && r0 < x.Tv) mv |= epi_group<SF, 0, true, D2LO>(x, col, r0, lane, slot, task);
    const int c0 = r0 - tp.vb;                         // colour texel of lane 0
    if (tp.tkind[j] != kTileVis && c0 + GRP > 0 && c0 < x.Tc)
      mc |= epi_group<SF, KIND, false, false>(x, col + (tp.tkind[j] == kTileBoth ? (uint32_t)tp.crow : 0u), c0,
                                             lane, slot, task);
  }
}

// The item's old texels and last-transmitted codes, into shared memory.
__device__ __forceinline__ void prefetch_item(const pv_dev& k, int np, int p0, int sb, uint8_t* st_c, uint8_t* st_v,
                                              uint16_t* ls_c, uint16_t* ls_v, uint64_t* bar) {
  const int npi = min(np, k.P - p0);
  const uint32_t sc_b = (uint32_t)npi * k.sc_stride * sb, sv_b = (uint32_t)npi * k.sv_stride * sb;
  const uint32_t lc_b = (uint32_t)npi * k.lc_stride * 2, lv_b = (uint32_t)npi * k.lv_stride * 2;
  mbar_expect_tx(bar, 3 * (sc_b + lc_b) + 2 * (sv_b + lv_b));
  for (int c = 0; c < 3; ++c) {
    bulk_g2s(st_c + (size_t)c * np * k.sc_stride * sb,
             (const uint8_t*)k.state_c + ((size_t)c * k.P + p0) * k.sc_stride * sb, sc_b, bar);
    bulk_g2s(ls_c + (size_t)c * np * k.lc_stride, k.last_c + ((size_t)c * k.P + p0) * k.lc_stride, lc_b, bar);
  }
  for (int c = 0; c < 2; ++c) {
    bulk_g2s(st_v + (size_t)c * np * k.sv_stride * sb,
             (const uint8_t*)k.state_v + ((size_t)c * k.P + p0) * k.sv_stride * sb, sv_b, bar);
    bulk_g2s(ls_v + (size_t)c * np * k.lv_stride, k.last_v + ((size_t)c * k.P + p0) * k.lv_stride, lv_b, bar);
  }
}

// Guard band (Section 3.3) of every row of an item, from the interior texels
// just written. A lane keeps its guard-band table entries in registers; the
// epilogue warps share the rows, four rows in flight per lane.
template <int SF>
__device__ __forceinline__ void guard_band(uint32_t s_base, uint32_t s_g, int ng, int nch, int tile_elems,
                                           int np, int npi, int ew, int lane) {
  constexpr int SB = StateOps<SF>::SB;
  const uint32_t row_b = (uint32_t)tile_elems * SB;
  for (int q0 = 0; q0 < ng; q0 += 32) {
    const int q = q0 + lane;
    const bool ok = q < ng;
    const uint32_t ent = ok ? lds<4>(s_g + 4u * q) : 0u;
    const uint32_t dst = (ent & 0xFFFFu) * SB, src = (ent >> 16) * SB;
    for (int ch = 0; ch < nch; ++ch) {
      const uint32_t rb = s_base + (uint32_t)(ch * np) * row_b;
      for (int p0 = ew; p0 < npi; p0 += 4 * EPI_WARPS) {
        uint32_t val[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int p = p0 + u * EPI_WARPS;
          const uint32_t r = rb + (uint32_t)(p < npi ? p : p0) * row_b;
          val[u] = lds<SB>(r + src);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int p = p0 + u * EPI_WARPS;
          sts_if<SB>(ok && p < npi, rb + (uint32_t)p * row_b + dst, val[u]);
        }
      }
    }
  }
}

// Guard-band table slot of border position (r, c) of an (n+2)^2 tile: the
// ring in the order top row, bottom row, left column, right column.
__device__ __forceinline__ int ring_slot(int r, int c, int n) {
  if (r == 0) return c;
  if (r == n + 1) return (n + 2) + c;
  if (c == 0) return 2 * (n + 2) + (r - 1);
  return 2 * (n + 2) + n + (r - 1);
}

// ------------------------------------------------------------------ kernel
template <int FORM, int MAXV>
__global__ void __launch_bounds__(NT, 1) k_blend_tc(const __grid_constant__ BlendArgs<MAXV> a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  pv_grid_launch_dependents();
  const TcParams& tp = a.tp;
  const pv_dev& k = tp.k;                          // shapes and formats shared by the volumes
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool kSplitW = FORM != kF16;
  constexpr bool kSplitA = FORM == kF32;
  constexpr int ROWB = row_bytes<FORM>();
  constexpr int CPR = ROWB / 16;                   // 16-byte chunks per row

  uint64_t* bars = (uint64_t*)(smem + tp.off_bar);
  uint64_t* full = bars;                           // [stages]
  uint64_t* conv = bars + tp.stages;               // [stages]
  uint64_t* empty = bars + 2 * tp.stages;          // [stages]
  uint64_t* tfull = bars + 3 * tp.stages;          // [2]
  uint64_t* tempty = tfull + 2;                    // [2]
  uint64_t* efull = tempty + 2;                    // [1]: an item's texels and codes arrived
  uint32_t* tmem_holder = (uint32_t*)(efull + 1);
  float* rsum = (float*)(smem + tp.off_rsum);      // [Tc + Tv]: 1 / weight sum (0: no weight)
  uint16_t* tab_pos = (uint16_t*)(smem + tp.off_pos);   // [Tc + Tv]: texel position in its tile
  uint32_t* gb = (uint32_t*)(smem + tp.off_gb);    // [gb_c + gb_v]: guard-band dst | src << 16
  uint32_t* flag_mask = (uint32_t*)(smem + tp.off_flags);   // [2][2]: changed probes, by item parity
  uint8_t* state_s = smem + tp.off_state;
  uint16_t* last_s = (uint16_t*)(smem + tp.off_last);

  const int sb = k.state_fmt == PV_FMT_F16 ? 2 : 4;
  const int np = tp.np;
  // shared-memory layout of an item's texels and codes: [ch][np][stride]
  uint8_t* st_c = state_s;
  uint8_t* st_v = state_s + (size_t)3 * np * k.sc_stride * sb;
  uint16_t* ls_c = last_s;
  uint16_t* ls_v = last_s + (size_t)3 * np * k.lc_stride;

  if (threadIdx.x == 0) {
    for (int s = 0; s < tp.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 64);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EPI_THREADS);
    }
    mbar_init(efull, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_holder))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  // Everything above runs while the previous kernel may still be running.
  // Each role waits for it (pv_grid_wait) just before its first read of
  // memory a predecessor wrote: the producer before its first load, the
  // epilogue before it reads sums, hysteresis and old tiles. The MMA issuer
  // and the converters touch only shared memory and TMEM. Parameter reads
  // before the wait overlap the predecessor's tail.
  int* err = k.err;
  // rounds of this CTA: its items
  const int rounds = tp.items > (int)blockIdx.x ? (tp.items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      for (int v = 0; v < a.nvol; ++v) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(&a.v[v].dist) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&a.v[v].rad) : "memory");
      }
      {  // the first item's parameters, fetched before the wait
        const BlendVol& b0 = a.v[vol_of(a, (int)blockIdx.x < tp.items ? (int)blockIdx.x : tp.items - 1)];
        asm volatile("" ::"r"(b0.nchunks), "r"(b0.item0), "r"(b0.k.P), "l"(b0.k.w_op), "r"(b0.k.w_chunks),
                     "r"(tp.stage_tx), "r"(tp.w_tx), "r"(tp.kc), "r"(tp.crow), "r"(tp.ntiles), "r"(tp.off_w),
                     "r"(tp.off_w_lo), "r"(tp.stages), "r"(tp.stage_bytes));
      }
      pv_grid_wait();
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int it = 0; it < rounds && ok; ++it) {
        const int item = blockIdx.x + it * gridDim.x;
        const bool real = item < tp.items;
        const BlendVol& bv = a.v[vol_of(a, real ? item : tp.items - 1)];
        const int p0 = (item - bv.item0) * np;
        for (int kc = 0; kc < bv.nchunks; ++kc) {
          ok = mbar_wait(&empty[s], ph ^ 1, err);
          if (!ok) break;
          uint8_t* st = smem + (size_t)s * tp.stage_bytes;
          const int x = kc * tp.kc;
          mbar_expect_tx(&full[s], real ? tp.stage_tx : tp.w_tx);
          if (real) {
            tma_load_2d(st, &bv.dist, x, p0, &full[s]);
            for (int c = 0; c < 3; ++c)
              tma_load_2d(st + (size_t)(tp.crow + c * GRP) * ROWB, &bv.rad, x, c * bv.k.P + p0, &full[s]);
          }
          // the chunk's weight tile images (hi and, split forms, lo), one bulk
          // copy each, straight into the MMA's swizzled layout
          const uint32_t wbytes = (uint32_t)tp.ntiles * MT * ROWB;
          const uint8_t* wsrc = (const uint8_t*)bv.k.w_op + (size_t)kc * wbytes;
          const size_t wplane = (size_t)bv.k.w_chunks * wbytes;
          bulk_g2s(st + tp.off_w, wsrc, wbytes, &full[s]);
          if (kSplitW) bulk_g2s(st + tp.off_w_lo, wsrc + wplane, wbytes, &full[s]);
          if (++s == tp.stages) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      // one item per CTA: its old texels and codes go into the first
      // alias_stages stages once the MMAs that read those stages are done
      if (tp.alias_stages > 0 && rounds > 0 && ok) {
        const uint32_t need = (1u << tp.alias_stages) - 1u;
        uint32_t got = 0u;
        for (int i = 0; i < tp.stages && ok && (got & need) != need; ++i) {
          ok = mbar_wait(&empty[s], ph ^ 1, err);
          got |= 1u << s;
          if (++s == tp.stages) {
            s = 0;
            ph ^= 1;
          }
        }
        if (ok) {
          const BlendVol& bv = a.v[vol_of(a, blockIdx.x)];
          prefetch_item(bv.k, np, ((int)blockIdx.x - bv.item0) * np, sb, st_c, st_v, ls_c, ls_v, efull);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int s = 0, b = 0;
      uint32_t ph = 0, tph = 0;
      bool ok = true;
      for (int it = 0; it < rounds && ok; ++it) {
        const int item = blockIdx.x + it * gridDim.x;
        const bool real = item < tp.items;
        const int nchunks = a.v[vol_of(a, real ? item : tp.items - 1)].nchunks;
        if (real) {
          ok = mbar_wait(&tempty[b], tph ^ 1, err);
          if (!ok) break;
          tc_fence_after();
        }
        const uint32_t dbase = tmem + b * 256;
        for (int kc = 0; kc < nchunks; ++kc) {
          ok = mbar_wait(&conv[s], ph, err);
          if (!ok) break;
          tc_fence_after();
          uint8_t* st = smem + (size_t)s * tp.stage_bytes;
#pragma unroll
          for (int ks = 0; ks < ROWB / 32 && real; ++ks) {   // one MMA K step per 32 bytes of row
            const int kb = ks * 32;
            const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
            // one MMA per tile (per weight / ray part): visibility tiles take the
            // visibility rows of the ray tile, colour tiles the colour rows, a
            // tile holding both takes the whole ray tile
            for (int j = 0; j < tp.ntiles; ++j) {
              const uint32_t d = dbase + tp.tbase[j];
              const size_t brow = tp.tkind[j] == kTileCol ? (size_t)tp.crow : 0;
              const uint64_t a = sdesc<ROWB>(st + tp.off_w + (size_t)j * MT * ROWB + kb);
              const uint64_t bb = sdesc<ROWB>(st + brow * ROWB + kb);
              mma<FORM>(d, a, bb, tp.tidesc[j], acc);
              if (kSplitW) mma<FORM>(d, sdesc<ROWB>(st + tp.off_w_lo + (size_t)j * MT * ROWB + kb), bb, tp.tidesc[j], 1u);
              if (kSplitA) mma<FORM>(d, a, sdesc<ROWB>(st + tp.off_a_lo + brow * ROWB + kb), tp.tidesc[j], 1u);
            }
          }
          // stage free once these MMAs finish
          mma_commit(&empty[s]);
          if (++s == tp.stages) {
            s = 0;
            ph ^= 1;
          }
        }
        if (!ok) break;
        if (!real) continue;
        mma_commit(&tfull[b]);                         // accumulators ready for the epilogue
        if (++b == tp.nbuf) {
          b = 0;
          tph ^= 1;
        }
      }
    }
  } else if (warp < 4) {
    // ------------------------------------------------------------ converters
    const int ct = threadIdx.x - 64;
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int it = 0; it < rounds && ok; ++it) {
      const int item = blockIdx.x + it * gridDim.x;
      const int nchunks = a.v[vol_of(a, item < tp.items ? item : tp.items - 1)].nchunks;
      for (int kc = 0; kc < nchunks; ++kc) {
        ok = mbar_wait(&full[s], ph, err);
        if (!ok) break;
        uint8_t* st = smem + (size_t)s * tp.stage_bytes;
        if constexpr (FORM == kF32) {
          // d^2 rows from full-precision d, then every row split into TF32 hi + lo;
          // each thread loads all of its chunks before it stores any
          constexpr int DCH = GRP * CPR / 64;          // d chunks per thread
          float4 d[DCH];
#pragma unroll
          for (int u = 0; u < DCH; ++u) d[u] = *(const float4*)(st + (size_t)(ct + 64 * u) * 16);
#pragma unroll
          for (int u = 0; u < DCH; ++u)
            *(float4*)(st + (size_t)(GRP * CPR + ct + 64 * u) * 16) =
                make_float4(d[u].x * d[u].x, d[u].y * d[u].y, d[u].z * d[u].z, d[u].w * d[u].w);
          conv_bar();
          constexpr int ACH = 160 * CPR / 64;          // chunks per thread over the B tile's 160 rows
          uint4 x[ACH];
#pragma unroll
          for (int u = 0; u < ACH; ++u) x[u] = *(const uint4*)(st + (size_t)(ct + 64 * u) * 16);
#pragma unroll
          for (int u = 0; u < ACH; ++u) {
            const uint4 hi = make_uint4(x[u].x & 0xFFFFE000u, x[u].y & 0xFFFFE000u, x[u].z & 0xFFFFE000u,
                                        x[u].w & 0xFFFFE000u);
            const float4 lo = make_float4(__uint_as_float(x[u].x) - __uint_as_float(hi.x),
                                          __uint_as_float(x[u].y) - __uint_as_float(hi.y),
                                          __uint_as_float(x[u].z) - __uint_as_float(hi.z),
                                          __uint_as_float(x[u].w) - __uint_as_float(hi.w));
            *(uint4*)(st + (size_t)(ct + 64 * u) * 16) = hi;
            *(float4*)(st + tp.off_a_lo + (size_t)(ct + 64 * u) * 16) = lo;
          }
        } else {
          // d^2 = hi + lo in the operand format (binary16 scaled by 2^-4): the low
          // part keeps the rounding of d^2 out of the visibility moments
          for (int q = ct; q < GRP * CPR; q += 64) {
            const uint4 raw = *(const uint4*)(st + (size_t)q * 16);
            const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
            uint32_t oh[4], ol[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if constexpr (FORM == kF16) {
                const __half2 h2 = *reinterpret_cast<const __half2*>(&w[e]);
                const float d0 = __low2float(h2), d1 = __high2float(h2);
                const float q0 = d0 * d0 * kD2ScaleF16, q1 = d1 * d1 * kD2ScaleF16;
                const __half h0 = __float2half_rn(q0), h1 = __float2half_rn(q1);
                const __half l0 = __float2half_rn(q0 - __half2float(h0));
                const __half l1 = __float2half_rn(q1 - __half2float(h1));
                oh[e] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
                ol[e] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
              } else {
                const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&w[e]);
                const float d0 = __low2float(h2), d1 = __high2float(h2);
                const float q0 = d0 * d0, q1 = d1 * d1;
                const __nv_bfloat16 h0 = __float2bfloat16_rn(q0), h1 = __float2bfloat16_rn(q1);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(q0 - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(q1 - __bfloat162float(h1));
                oh[e] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                ol[e] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
              }
            }
            *(uint4*)(st + (size_t)(GRP * CPR + q) * 16) = make_uint4(oh[0], oh[1], oh[2], oh[3]);
            *(uint4*)(st + (size_t)(2 * GRP * CPR + q) * 16) = make_uint4(ol[0], ol[1], ol[2], ol[3]);
          }
        }
        fence_proxy_async();
        mbar_arrive(&conv[s]);
        if (++s == tp.stages) {
          s = 0;
          ph ^= 1;
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int e = threadIdx.x - 128;                   // 0..EPI_THREADS-1
    const int ew = e >> 5;                             // epilogue warp 0..EPI_WARPS-1
    const int quarter = warp & 3;                      // TMEM lanes 32*quarter .. +32
    const int slot = ew >> 2;                          // which of the quarter's three warps
    // per-texel tables, built while the first stages load (the weight sums,
    // which differ per volume, when an item of a new volume starts)
    for (int t = e; t < k.Tc + k.Tv; t += EPI_THREADS) {
      const bool vis = t >= k.Tc;
      const int n = vis ? k.nv : k.nc, tt = vis ? t - k.Tc : t;
      const int i = tt / n, j = tt % n;
      const int src = (i + 1) * (n + 2) + (j + 1);
      tab_pos[t] = (uint16_t)src;
      int tr[8], tc[8];
      const int nb = pv::border_targets(i, j, n, tr, tc);
      uint32_t* g = vis ? gb + tp.gb_c : gb;
      for (int q = 0; q < nb; ++q)
        g[ring_slot(tr[q], tc[q], n)] = (uint32_t)(tr[q] * (n + 2) + tc[q]) | ((uint32_t)src << 16);
    }
    if (e < 4) flag_mask[e] = 0;
    pv_grid_wait();
    // thread 0 streams each item's old texels and codes into shared memory as
    // soon as the previous item's tiles have been written back
    if (e == 0 && blockIdx.x < tp.items && tp.alias_stages == 0) {
      const BlendVol& bv = a.v[vol_of(a, blockIdx.x)];
      prefetch_item(bv.k, np, ((int)blockIdx.x - bv.item0) * np, sb, st_c, st_v, ls_c, ls_v, efull);
    }
    constexpr bool kSplitD2 = FORM != kF32;         // d^2 as hi + lo columns
    const int kind = k.color_code;
    const bool f16 = k.state_fmt == PV_FMT_F16;
    const uint32_t s_st_c = smem_u32(st_c), s_st_v = smem_u32(st_v);
    const uint32_t s_ls_c = smem_u32(ls_c), s_ls_v = smem_u32(ls_v);
    const uint32_t s_rsum = smem_u32(rsum), s_pos = smem_u32(tab_pos), s_gb = smem_u32(gb);
    EpiCtx x;
    x.s_rsum = s_rsum;
    x.s_pos = s_pos;
    x.s_st_c = s_st_c;
    x.s_st_v = s_st_v;
    x.s_ls_c = s_ls_c;
    x.s_ls_v = s_ls_v;
    x.sc_stride = k.sc_stride;
    x.sv_stride = k.sv_stride;
    x.lc_stride = k.lc_stride;
    x.lv_stride = k.lv_stride;
    x.Tc = k.Tc;
    x.Tv = k.Tv;
    x.np = np;
    x.npi = np;
    x.d2_scale = FORM == kF16 ? 1.0f / kD2ScaleF16 : 1.0f;
    int b = 0, par = 0, cur = -1;
    uint32_t tph = 0, eph = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < tp.items && ok; item += gridDim.x) {
      const int vi = vol_of(a, item);
      const pv_dev& kv = a.v[vi].k;
      const int p0 = (item - a.v[vi].item0) * np;      // first probe of the item in its volume
      const int npi = min(np, kv.P - p0);
      if (vi != cur) {                                 // this volume's weight sums and hysteresis
        for (int t = e; t < k.Tc + k.Tv; t += EPI_THREADS) {
          const float S = kv.sums[t];
          rsum[t] = S > 0.0f ? 1.0f / S : 0.0f;
        }
        x.h = *kv.hy;
        x.omh = 1.0f - x.h;
        cur = vi;
      }
      epi_bar();
      ok = mbar_wait(efull, eph, err);
      if (ok) ok = mbar_wait(&tfull[b], tph, err);
      if (!ok) break;
      eph ^= 1;
      tc_fence_after();
      const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16) + b * 256;
      x.npi = npi;
      uint32_t mv, mc;
      if (f16) {
        if (kind == PV_CODE_UNORM10) epi_item<0, PV_CODE_UNORM10, kSplitD2>(tp, x, tq, quarter, lane, slot, mc, mv);
        else epi_item<0, PV_CODE_UF10, kSplitD2>(tp, x, tq, quarter, lane, slot, mc, mv);
      } else {
        if (kind == PV_CODE_UNORM10) epi_item<1, PV_CODE_UNORM10, kSplitD2>(tp, x, tq, quarter, lane, slot, mc, mv);
        else epi_item<1, PV_CODE_UF10, kSplitD2>(tp, x, tq, quarter, lane, slot, mc, mv);
      }
      // accumulators consumed: hand the TMEM buffer back to the MMA thread
      tc_fence_before();
      mbar_arrive(&tempty[b]);
      if (++b == tp.nbuf) {
        b = 0;
        tph ^= 1;
      }
      mc = __reduce_or_sync(0xffffffffu, mc);
      mv = __reduce_or_sync(0xffffffffu, mv);
      uint32_t* fm = flag_mask + 2 * par;
      if (lane == 0) {
        if (mc) atomicOr(&fm[0], mc);
        if (mv) atomicOr(&fm[1], mv);
      }
      epi_bar();                                       // interior texels and flags of the item done
      if (e < 2) {                                     // changed-probe bits of this item
        const uint32_t m = fm[e];
        fm[e] = 0;                                     // this parity's masks are next used two items on
        const int sh = p0 & 31;
        uint32_t* w = &kv.chg[e * kv.chg_words + (p0 >> 5)];
        if (m << sh) atomicOr(w, m << sh);
        if (sh && (m >> (32 - sh))) atomicOr(w + 1, m >> (32 - sh));
      }
      par ^= 1;
      if (f16) {
        guard_band<0>(s_st_c, s_gb, tp.gb_c, 3, k.sc_stride, np, npi, ew, lane);
        guard_band<0>(s_st_v, s_gb + 4u * tp.gb_c, tp.gb_v, 2, k.sv_stride, np, npi, ew, lane);
      } else {
        guard_band<1>(s_st_c, s_gb, tp.gb_c, 3, k.sc_stride, np, npi, ew, lane);
        guard_band<1>(s_st_v, s_gb + 4u * tp.gb_c, tp.gb_v, 2, k.sv_stride, np, npi, ew, lane);
      }
      fence_proxy_async();
      epi_bar();
      if (e == 0) {
        const uint32_t sc_b = (uint32_t)npi * k.sc_stride * sb, sv_b = (uint32_t)npi * k.sv_stride * sb;
        for (int c = 0; c < 3; ++c)
          bulk_s2g((uint8_t*)kv.state_c + ((size_t)c * kv.P + p0) * k.sc_stride * sb,
                   st_c + (size_t)c * np * k.sc_stride * sb, sc_b);
        for (int c = 0; c < 2; ++c)
          bulk_s2g((uint8_t*)kv.state_v + ((size_t)c * kv.P + p0) * k.sv_stride * sb,
                   st_v + (size_t)c * np * k.sv_stride * sb, sv_b);
        if (kv.cur_c) {                                // the item's current codes
          const uint32_t lc_b = (uint32_t)npi * k.lc_stride * 2, lv_b = (uint32_t)npi * k.lv_stride * 2;
          for (int c = 0; c < 3; ++c)
            bulk_s2g(kv.cur_c + ((size_t)c * kv.P + p0) * k.lc_stride, ls_c + (size_t)c * np * k.lc_stride, lc_b);
          for (int c = 0; c < 2; ++c)
            bulk_s2g(kv.cur_v + ((size_t)c * kv.P + p0) * k.lv_stride, ls_v + (size_t)c * np * k.lv_stride, lv_b);
        }
        bulk_commit();
        bulk_wait_read();                              // shared tiles may be refilled now
        const int next = item + gridDim.x;
        if (next < tp.items) {
          const BlendVol& nv = a.v[vol_of(a, next)];
          prefetch_item(nv.k, np, (next - nv.item0) * np, sb, st_c, st_v, ls_c, ls_v, efull);
        }
      }
    }
    if (e == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ------------------------------------------------------------------ host plan
constexpr int kMaxBatch = PV_MAX_BATCH;

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encoder() {
  if (g_encode) return cudaSuccess;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return cudaSuccess;
}

CUtensorMapDataType dtype_of(int fmt) {
  if (fmt == PV_FMT_F16) return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  if (fmt == PV_FMT_BF16) return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
}

cudaError_t encode_2d(CUtensorMap* m, int fmt, const void* base, uint64_t inner, uint64_t rows,
                      uint64_t row_bytes, uint32_t box_inner, uint32_t box_rows) {
  const CUtensorMapSwizzle swz = box_inner * (fmt == PV_FMT_F32 ? 4u : 2u) == 64u ? CU_TENSOR_MAP_SWIZZLE_64B
                                                                                : CU_TENSOR_MAP_SWIZZLE_32B;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(m, dtype_of(fmt), 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// kind::f16 / kind::tf32 instruction descriptor: F32 accumulate, K-major A and B.
uint32_t make_idesc(int form, int M, int N) {
  const uint32_t ab = form == kF32 ? 2u : (form == kBF16 ? 1u : 0u);
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

size_t align1k(size_t x) { return (x + 1023) & ~(size_t)1023; }

int form_of(int operand_fmt) {
  return operand_fmt == PV_FMT_F16 ? kF16 : (operand_fmt == PV_FMT_BF16 ? kBF16 : kF32);
}

template <int MAXV>
cudaError_t set_smem_attr_v(int form, int bytes) {
  if (form == kF16)
    return cudaFuncSetAttribute(k_blend_tc<kF16, MAXV>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (form == kBF16)
    return cudaFuncSetAttribute(k_blend_tc<kBF16, MAXV>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return cudaFuncSetAttribute(k_blend_tc<kF32, MAXV>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

struct DevInfo {
  int sms, smem_max;
};

cudaError_t dev_info(DevInfo* d) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d->smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return e;
}

// Tile layout, stage ring and epilogue regions for volumes shaped like k, with
// work items of at most np_want probes (fewer when shared memory demands).
// Fills every field of tp except items, iters and the volume-dependent ones.
cudaError_t make_layout(const pv_dev& k, int form, int np_want, int smem_max, bool alias_ok,
                        TcParams& tp, size_t* smem) {
  const int sb = k.state_fmt == PV_FMT_F16 ? 2 : 4;
  const int ROWB = form == kF32 ? row_bytes<kF32>() : row_bytes<kF16>();
  tp.k = k;
  tp.kc = k.w_kc;                              // = ROWB / operand bytes
  // ray (B) tile rows: d | d^2 (| d^2 lo, 16-bit forms) | R | G | B, 32 each
  tp.nvc = form != kF32 ? 3 * GRP : 2 * GRP;
  tp.crow = tp.nvc;
  tp.a_rows = tp.crow + 3 * GRP;
  // texel (A) tiles: the weight images' rows, visibility texels in rows
  // 0..Tv-1 and colour texels from row vb; one MMA per 128-row tile, with the
  // B rows its texels need
  if (k.w_rb != ROWB || k.w_rows % MT != 0) return cudaErrorInvalidValue;
  tp.vb = k.w_vb;
  tp.ntiles = k.w_rows / MT;
  int col = 0;
  for (int j = 0; j < tp.ntiles; ++j) {
    const int r0 = j * MT, r1 = r0 + MT;
    const bool has_v = r0 < k.Tv, has_c = r1 > tp.vb && r0 < tp.vb + k.Tc;
    tp.tkind[j] = has_v && has_c ? kTileBoth : (has_v ? kTileVis : kTileCol);
    const int n = tp.tkind[j] == kTileBoth ? tp.a_rows : (tp.tkind[j] == kTileVis ? tp.nvc : 3 * GRP);
    tp.tbase[j] = col;
    tp.tidesc[j] = make_idesc(form, MT, n);
    col += n;
  }
  tp.bufcols = col;
  tp.nbuf = tp.bufcols <= 256 ? 2 : 1;         // buffers at TMEM columns 0 and 256
  tp.gb_c = 4 * k.nc + 4;
  tp.gb_v = 4 * k.nv + 4;
  // stage layout: ray tile, its TF32 low parts (FP32 form), then the weight
  // tile(s): ntiles * 128 rows each, of which the MMAs read all (rows past
  // the texels hold whatever was there; the lanes they produce are ignored)
  size_t off = 0;
  const size_t a_b = align1k((size_t)tp.a_rows * ROWB);
  off += a_b;
  tp.off_a_lo = (int)off;
  if (form == kF32) off += a_b;
  const size_t w_b = (size_t)tp.ntiles * MT * ROWB;
  tp.off_w = (int)off;
  off += w_b;
  tp.off_w_lo = tp.off_w;
  if (form != kF16) {
    tp.off_w_lo = (int)off;
    off += w_b;
  }
  tp.stage_bytes = (int)off;
  // probes per work item: np_want, fewer when the item's tiles would leave
  // room for less than two stages
  const size_t n_rsum = (size_t)(k.Tc + k.Tv) * 4, n_pos = (size_t)(k.Tc + k.Tv) * 2;
  const size_t n_gb = (size_t)(tp.gb_c + tp.gb_v) * 4;
  tp.alias_stages = 0;
  tp.w_tx = (uint32_t)((form != kF16 ? 2 : 1) * tp.ntiles * MT * ROWB);
  int np = np_want;
  int stages = 0;
  size_t epi_state = 0, epi_last = 0;
  for (; np >= 1; --np) {
    // the epilogue's last row group of a channel reads up to 7 rows past the
    // item, so each region ends with 8 spare rows
    epi_state = ((size_t)np * (3 * k.sc_stride + 2 * k.sv_stride) + 8 * (size_t)k.sv_stride) * sb;
    epi_last = ((size_t)np * (3 * k.lc_stride + 2 * k.lv_stride) + 8 * (size_t)k.lv_stride) * 2;
    const size_t epi = align1k(epi_state) + align1k(epi_last) + align1k(n_rsum) + align1k(n_pos) +
                       align1k(n_gb) + 1024 + 1024;
    const size_t need = 1024 + epi;
    stages = need < (size_t)smem_max ? (int)(((size_t)smem_max - need) / tp.stage_bytes) : 0;
    if (stages >= 2) break;
  }
  if (alias_ok && stages < 3) {
    // One item per CTA and a shallow ring (the FP32 form): the ring takes all
    // of shared memory but the tables, and the item's old texels and codes go
    // into its first stages once the main loop no longer needs them, so the
    // ring is about twice as deep. (With three or more stages the separate
    // layout is faster: its old tiles load early, not behind the last chunks.)
    const size_t es = ((size_t)np_want * (3 * k.sc_stride + 2 * k.sv_stride) + 8 * (size_t)k.sv_stride) * sb;
    const size_t el = ((size_t)np_want * (3 * k.lc_stride + 2 * k.lv_stride) + 8 * (size_t)k.lv_stride) * 2;
    const size_t tables = align1k(n_rsum) + align1k(n_pos) + align1k(n_gb) + 1024 + 1024;
    const size_t region = align1k(es) + align1k(el);
    int st = tables + 2048 < (size_t)smem_max ? (int)(((size_t)smem_max - 2048 - tables) / tp.stage_bytes) : 0;
    if (st > kMaxStages) st = kMaxStages;
    if (st >= 2 && (size_t)st * tp.stage_bytes >= region) {
      tp.np = np_want;
      tp.stages = st;
      tp.alias_stages = (int)((region + tp.stage_bytes - 1) / tp.stage_bytes);
      tp.stage_tx = (uint32_t)(4 * np_want * ROWB) + tp.w_tx;
      tp.off_state = 0;
      tp.off_last = (int)align1k(es);
      size_t off = (size_t)st * tp.stage_bytes;
      tp.off_rsum = (int)off;
      off += align1k(n_rsum);
      tp.off_pos = (int)off;
      off += align1k(n_pos);
      tp.off_gb = (int)off;
      off += align1k(n_gb);
      tp.off_flags = (int)off;
      off += 1024;
      tp.off_bar = (int)off;
      off += 1024;
      *smem = off + 1024;                      // slack for aligning the dynamic base
      return cudaSuccess;
    }
  }
  if (stages < 2) return cudaErrorInvalidConfiguration;
  if (stages > kMaxStages) stages = kMaxStages;
  tp.np = np;
  tp.stages = stages;
  tp.stage_tx = (uint32_t)(4 * np * ROWB) + tp.w_tx;
  off = (size_t)stages * tp.stage_bytes;
  tp.off_state = (int)off;
  off += align1k(epi_state);
  tp.off_last = (int)off;
  off += align1k(epi_last);
  tp.off_rsum = (int)off;
  off += align1k(n_rsum);
  tp.off_pos = (int)off;
  off += align1k(n_pos);
  tp.off_gb = (int)off;
  off += align1k(n_gb);
  tp.off_flags = (int)off;
  off += 1024;
  tp.off_bar = (int)off;
  off += 1024;
  *smem = off + 1024;                          // slack for aligning the dynamic base
  return cudaSuccess;
}

// Tensor maps of one frame's rays (radiance [3][P][R], dist [P][R]).
cudaError_t encode_ray_maps(const pv_dev& k, int form, const TcParams& tp, const void* rad, const void* dist,
                            BlendVol& bv) {
  const int ob = form == kF32 ? 4 : 2;
  cudaError_t e = encode_2d(&bv.rad, k.operand_fmt, rad, k.R, (uint64_t)3 * k.P, (uint64_t)k.R * ob, tp.kc, tp.np);
  if (e == cudaSuccess) e = encode_2d(&bv.dist, k.operand_fmt, dist, k.R, k.P, (uint64_t)k.R * ob, tp.kc, tp.np);
  return e;
}

template <int MAXV>
cudaError_t launch_blend(const BlendArgs<MAXV>& a, int form, int grid, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0] = pv_pdl_attr();
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (form == kF16) e = cudaLaunchKernelEx(&cfg, k_blend_tc<kF16, MAXV>, a);
  else if (form == kBF16) e = cudaLaunchKernelEx(&cfg, k_blend_tc<kBF16, MAXV>, a);
  else e = cudaLaunchKernelEx(&cfg, k_blend_tc<kF32, MAXV>, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

struct TcPlan {
  BlendArgs<1> args;
  size_t smem;
  int grid;
  int form;
};

}  // namespace

// Batch plan (opaque to the API layer).
struct pv_tc_batch {
  BlendArgs<kMaxBatch> args;
  size_t smem;
  int grid;
  int form;
  int n;
  pv_volume* vols[kMaxBatch];
};

bool pv_tc_supported(const pv_desc* d, const char** why) {
  const int ob = d->operand_fmt == PV_FMT_F32 ? 4 : 2;
  const int nc = d->color_interior, nv = d->vis_interior;
  if (nc < 2 || nv < 2) {
    if (why) *why = "tile interiors below 2x2 (guard-band table holds three copies per texel)";
    return false;
  }
  if ((d->rays_per_probe * ob) % 16 != 0) {
    if (why) *why = "rays_per_probe * operand bytes must be a multiple of 16 (TMA row pitch)";
    return false;
  }
  // The library is built for sm_103a only, so the device needs no check
  // here: on any other GPU no kernel of the library can launch at all.
  return true;
}

cudaError_t pv_tc_plan_create(pv_volume* v) {
  cudaError_t e = get_encoder();
  DevInfo di;
  if (e == cudaSuccess) e = dev_info(&di);
  if (e != cudaSuccess) return e;
  const pv_dev& k = v->k;
  const int form = form_of(k.operand_fmt);
  e = set_smem_attr_v<1>(form, di.smem_max);
  if (e != cudaSuccess) return e;
  // one CTA per SM
  const int resident = di.sms;
  // one item per resident CTA where possible
  const int np_max = v->state_bytes == 2 ? 32 : 16;
  int np = (k.P + resident - 1) / resident;
  np = np < 1 ? 1 : (np > np_max ? np_max : np);
  TcPlan* pl = new TcPlan();
  memset(pl, 0, sizeof(TcPlan));
  TcParams& tp = pl->args.tp;
  // a volume whose items all fit in one wave keeps each item's old tiles in
  // its CTA's stage ring (a deeper ring)
  const bool one_wave = (k.P + np - 1) / np <= resident;
  e = make_layout(k, form, np, di.smem_max, one_wave, tp, &pl->smem);
  if (e == cudaSuccess) {
    tp.items = (k.P + tp.np - 1) / tp.np;
    pl->grid = tp.items < resident ? tp.items : resident;
    tp.iters = (tp.items + pl->grid - 1) / pl->grid;
    if (tp.alias_stages > 0 && tp.iters != 1) e = cudaErrorInvalidConfiguration;   // cannot happen: np kept
    pl->form = form;
    pl->args.nvol = 1;
    BlendVol& bv = pl->args.v[0];
    bv.k = k;
    bv.item0 = 0;
    bv.nchunks = k.w_chunks;
  }
  if (e != cudaSuccess) {
    delete pl;
    return e;
  }
  v->tc_plan = pl;
  return cudaSuccess;
}

void pv_tc_plan_destroy(pv_volume* v) {
  if (v && v->tc_plan) {
    delete (TcPlan*)v->tc_plan;
    v->tc_plan = nullptr;
  }
}

cudaError_t pv_launch_blend_tc(pv_volume* v, const void* rad, const void* dist, cudaStream_t st) {
  TcPlan* pl = (TcPlan*)v->tc_plan;
  if (!pl) return cudaErrorNotSupported;
  BlendArgs<1> a = pl->args;
  a.tp.k = v->k;
  a.v[0].k = v->k;
  cudaError_t e = encode_ray_maps(v->k, pl->form, a.tp, rad, dist, a.v[0]);
  if (e != cudaSuccess) return e;
  return launch_blend(a, pl->form, pl->grid, pl->smem, st);
}

cudaError_t pv_tc_batch_create(pv_volume* const* vols, int n, int np_want, pv_tc_batch** out) {
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  cudaError_t e = get_encoder();
  DevInfo di;
  if (e == cudaSuccess) e = dev_info(&di);
  if (e != cudaSuccess) return e;
  const pv_dev& k0 = vols[0]->k;
  const int form = form_of(k0.operand_fmt);
  e = set_smem_attr_v<kMaxBatch>(form, di.smem_max);
  if (e != cudaSuccess) return e;
  int total = 0;
  for (int i = 0; i < n; ++i) total += vols[i]->k.P;
  const int np_max = vols[0]->state_bytes == 2 ? 32 : 16;
  int np = np_want > 0 ? np_want : (total + di.sms - 1) / di.sms;
  np = np < 1 ? 1 : (np > np_max ? np_max : np);
  pv_tc_batch* b = new pv_tc_batch();
  memset(b, 0, sizeof(pv_tc_batch));
  TcParams& tp = b->args.tp;
  e = make_layout(k0, form, np, di.smem_max, false, tp, &b->smem);
  if (e == cudaSuccess) {
    int items = 0;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
      const pv_dev& k = vols[i]->k;
      BlendVol& bv = b->args.v[i];
      bv.k = k;
      bv.item0 = items;
      bv.nchunks = k.w_chunks;
      items += (k.P + tp.np - 1) / tp.np;
      b->vols[i] = vols[i];
    }
    tp.items = items;
    b->grid = items < di.sms ? items : di.sms;
    tp.iters = (items + b->grid - 1) / b->grid;
    b->args.nvol = n;
    b->form = form;
    b->n = n;
  }
  if (e != cudaSuccess) {
    delete b;
    return e;
  }
  *out = b;
  return cudaSuccess;
}

void pv_tc_batch_destroy(pv_tc_batch* b) { delete b; }

int pv_tc_batch_np(const pv_tc_batch* b) { return b->args.tp.np; }

cudaError_t pv_tc_batch_launch(pv_tc_batch* b, const void* const* rad, const void* const* dist, cudaStream_t st) {
  // the launch arguments live on the host stack for the duration of the call
  BlendArgs<kMaxBatch>* a = new BlendArgs<kMaxBatch>(b->args);
  cudaError_t e = cudaSuccess;
  a->tp.k = b->vols[0]->k;
  for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
    a->v[i].k = b->vols[i]->k;
    e = encode_ray_maps(b->vols[i]->k, b->form, a->tp, rad[i], dist[i], a->v[i]);
  }
  if (e == cudaSuccess) e = launch_blend(*a, b->form, b->grid, b->smem, st);
  delete a;
  return e;
}
