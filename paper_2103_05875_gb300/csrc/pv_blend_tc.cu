// K1 (tensor-core form): the probe blend of Section 3.2 of arXiv 2103.05875 as
// a tcgen05 contraction with a fused epilogue, for sm_103a.
//
// The blend is a dense contraction because every probe of a volume shares the
// frame's ray directions: per probe row x (a colour channel, d or d^2) and
// texel t, acc[t] = sum_r W[t, r] x[r]. Rows of a work item (np <= 32 probes)
// form the MMA's M dimension, texels its N dimension, rays its K dimension:
//
//   A (shared memory, K-major, 64-byte rows, SWIZZLE_64B), row groups of 32:
//     [ d | d^2 (hi) | d^2 lo (16-bit forms) | R | G | B ]
//     d and the colour planes come straight from HBM by TMA; d^2 is formed on
//     chip by two converter warps (its rounding to the operand format is split
//     into hi + lo parts so that it costs no accuracy).
//   B (shared memory): W_v [Nv x K] and W_c [Nc x K] from the weights kernel.
//   D (tensor memory, FP32): vis MMA over A rows 0..127 with N = Nv, colour
//     MMA over the 128 rows that end with the B plane, N = Nc. Accumulator
//     lanes: vis d = 0..31, d^2 = 32..63 (+64..95 lo); colour R, G, B = 32..127.
//
// Operand forms (pv_desc.operand_fmt):
//   F16  kind::f16, binary16 inputs; visibility weights scaled by 2^15 and
//        d^2 by 2^-8 (both undone exactly) to stay in range.
//   BF16 kind::f16 with bfloat16; W = W_hi + W_lo (two MMAs) because one
//        bfloat16 weight only carries 8 bits.
//   F32  kind::tf32, float32 inputs; x = x_hi + x_lo and W = W_hi + W_lo with
//        TF32 parts, three MMAs (hi*hi + hi*lo + lo*hi) recover float32
//        accuracy.
//
// Warp roles (384 threads, one CTA per SM, persistent over work items):
//   warp 0     TMA producer: ray tiles and weight tiles into a ring of stages;
//              the item's old texels and last-transmitted codes (bulk copies)
//   warp 1     TMEM allocation and the single MMA-issuing thread
//   warps 2-3  converters: d^2 rows, TF32 hi/lo split
//   warps 4-11 epilogue: TMEM -> registers -> shared (transposed), then the
//              fused per-texel work of Sections 3.2-3.4 (weight-sum
//              normalisation, hysteresis, storage rounding, guard band,
//              transmitted code, comparison with the last-transmitted code,
//              changed flags) on the item's tiles in shared memory, one probe
//              row per warp and one texel per lane, written back by bulk copies.
// Accumulators are double-buffered in TMEM when both fit in 256 columns, so
// an item's epilogue overlaps the next item's MMAs. Every mbarrier wait is
// bounded in time; on expiry the kernel raises the volume's error word and
// every role leaves its loop, so no wait can hang the GPU.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdio.h>
#include <type_traits>
#include <string.h>

#include "pv_codes.cuh"
#include "pv_internal.h"

namespace {

enum Form { kF16 = 0, kBF16 = 1, kF32 = 2 };

constexpr int NT = 384;
constexpr int EPI_THREADS = 256;         // warps 4..11
// bytes per K-chunk row in shared memory: 64 (SWIZZLE_64B) for the 16-bit
// forms, 32 (SWIZZLE_32B) for TF32, which keeps the FP32 form's stages small
// enough for a four-deep ring
template <int FORM>
__host__ __device__ constexpr int row_bytes() { return FORM == 2 ? 32 : 64; }
constexpr int GRP = 32;                  // rows per row group of the A tile
constexpr int MS_LD = 129;               // odd leading dimension of the transpose buffer
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

struct TcParams {
  pv_dev k;
  int np, items, stages, kc, nchunks;
  int Nc, Nv, nbuf, col_v, col_c;
  int crow;                              // first A row of the colour block
  int a_rows;                            // rows of the A tile
  int off_a_lo, off_wc, off_wc_lo, off_wv, off_wv_lo, stage_bytes;
  int off_state, off_last, off_ms, off_invs, off_flags, off_bar, off_tab;
  uint32_t stage_tx;
  uint32_t idesc_c, idesc_v;
};

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
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
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
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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

// ------------------------------------------------------------------ epilogue texel
// Per-texel constants of the epilogue, built once per launch: the texel's
// position in its tile and the guard-band positions that copy it (at most
// three for n >= 2, packed 16 bits each, count in the top 16 bits).
__device__ __forceinline__ uint64_t pack_border(int i, int j, int n) {
  int tr[8], tc[8];
  const int nb = pv::border_targets(i, j, n, tr, tc);
  uint64_t v = 0;
  int m = nb < 3 ? nb : 3;
  for (int b = 0; b < m; ++b) v |= (uint64_t)(tr[b] * (n + 2) + tc[b]) << (16 * b);
  return v | ((uint64_t)m << 48);
}

// State format as a compile-time choice: 0 binary16, 1 binary32. Tiles are
// addressed in elements through typed shared-memory pointers so the compiler
// can schedule the epilogue's loads and stores freely.
template <int SF>
struct StateOps {
  using T = typename std::conditional<SF == 0, uint16_t, uint32_t>::type;
  static __device__ __forceinline__ float value(uint32_t b) {
    return SF == 0 ? __half2float(__ushort_as_half((unsigned short)b)) : __uint_as_float(b);
  }
  static __device__ __forceinline__ uint32_t bits(float v) {
    return SF == 0 ? (uint32_t)__half_as_ushort(__float2half_rn(v)) : __float_as_uint(v);
  }
};

// Per-lane constants of the texel a lane handles in an epilogue pass.
struct LaneTexel {
  uint32_t pos, b0, b1, b2;   // element offsets in the tile: the texel and its guard-band copies
  int nb;                     // number of guard-band copies (0 for lanes without a texel)
  float rS;                   // 1 / weight sum (0: no weight, the texel keeps its value)
  int t;                      // texel index (code offset in a code row)
  bool has;
};

// One pass of the fused epilogue for a block of up to 32 texels (one per
// lane): each warp owns a fixed share of this texture's probe rows (ch, p) and
// loops over them, so a lane's rows are independent chains with all per-texel
// constants in registers. Per row the shared tile is updated in place
// (weight-sum normalisation, hysteresis, storage rounding, guard band) and the
// transmitted code is compared with the last-transmitted one; changed rows are
// collected in per-channel 32-bit probe masks, OR-reduced once per pass.
template <int SF, int KIND, bool VIS, bool D2LO>
__device__ __forceinline__ void epi_pass(const LaneTexel lt, const float* __restrict__ mcol, int npi, int np,
                                         void* tiles_v, int tile_elems, const uint16_t* __restrict__ codes,
                                         int code_elems, float h, float omh, float d2_scale, int ew, int lane,
                                         uint32_t* flag_mask) {
  using ST = typename StateOps<SF>::T;
  ST* __restrict__ tiles = reinterpret_cast<ST*>(tiles_v);
  constexpr int NCH = VIS ? 2 : 3;
  constexpr int PER = NCH * GRP / 8;                   // row slots per warp: 8 (vis), 12 (colour)
  constexpr int U = 4;                                 // rows in flight per lane
  uint32_t m0 = 0, m1 = 0, m2 = 0;
#pragma unroll
  for (int i0 = 0; i0 < PER; i0 += U) {
    // all loads of U rows first (branch-free), so the rows' chains overlap
    float acc[U];
    uint32_t old[U], last[U];
    int off[U], chs[U], ps[U];
    bool live[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int sl = ew * PER + i0 + u;
      const int ch = sl >> 5, p = sl & 31;
      live[u] = lt.has && p < npi;
      chs[u] = ch;
      ps[u] = p;
      const int pc = live[u] ? p : 0;
      off[u] = (ch * np + pc) * tile_elems;
      float a;
      if (VIS) {
        a = ch == 0 ? mcol[pc] : mcol[32 + pc];
        if (ch == 1) a = (D2LO ? a + mcol[64 + pc] : a) * d2_scale;
      } else {
        a = mcol[32 + 32 * ch + pc];
      }
      acc[u] = a;
      old[u] = (uint32_t)tiles[off[u] + lt.pos];
      last[u] = (uint32_t)codes[(ch * np + pc) * code_elems + lt.t];
    }
    // math, then stores
    uint32_t nb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t upd = StateOps<SF>::bits(fmaf(h, StateOps<SF>::value(old[u]), omh * (acc[u] * lt.rS)));
      nb[u] = lt.rS > 0.0f ? upd : old[u];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (live[u]) {
        tiles[off[u] + lt.pos] = (ST)nb[u];
        if (lt.nb > 0) tiles[off[u] + lt.b0] = (ST)nb[u];
        if (lt.nb > 1) tiles[off[u] + lt.b1] = (ST)nb[u];
        if (lt.nb > 2) tiles[off[u] + lt.b2] = (ST)nb[u];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      uint32_t code;
      if (VIS) code = SF == 0 ? nb[u] : (uint32_t)__half_as_ushort(__float2half_rn(__uint_as_float(nb[u])));
      else if (KIND == PV_CODE_UNORM10) code = pv::unorm10_from_float(StateOps<SF>::value(nb[u]));
      else code = SF == 0 ? pv::uf10_from_half_bits(nb[u]) : pv::uf10_from_float_bits(nb[u]);
      const uint32_t bit = (live[u] && code != last[u]) ? (1u << ps[u]) : 0u;
      m0 |= chs[u] == 0 ? bit : 0u;
      m1 |= chs[u] == 1 ? bit : 0u;
      m2 |= chs[u] == 2 ? bit : 0u;
    }
  }
  m0 = __reduce_or_sync(0xffffffffu, m0);
  m1 = __reduce_or_sync(0xffffffffu, m1);
  if (!VIS) m2 = __reduce_or_sync(0xffffffffu, m2);
  if (lane == 0) {
    const int base = VIS ? 3 : 0;
    if (m0) atomicOr(&flag_mask[base + 0], m0);
    if (m1) atomicOr(&flag_mask[base + 1], m1);
    if (!VIS && m2) atomicOr(&flag_mask[base + 2], m2);
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

// ------------------------------------------------------------------ kernel
template <int FORM>
__global__ void __launch_bounds__(NT, 1)
    k_blend_tc(const __grid_constant__ TcParams tp, const __grid_constant__ CUtensorMap map_rad,
               const __grid_constant__ CUtensorMap map_dist, const __grid_constant__ CUtensorMap map_wc,
               const __grid_constant__ CUtensorMap map_wv, const __grid_constant__ CUtensorMap map_wc_lo,
               const __grid_constant__ CUtensorMap map_wv_lo) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const pv_dev& k = tp.k;
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
  float* rsum = (float*)(smem + tp.off_invs);      // [Nc + Nv]: 1 / weight sum (0: no weight)
  uint64_t* tab_border = (uint64_t*)(smem + tp.off_tab);           // [Tc + Tv]
  uint16_t* tab_pos = (uint16_t*)(tab_border + k.Tc + k.Tv);       // [Tc + Tv]
  uint32_t* flag_mask = (uint32_t*)(smem + tp.off_flags);   // [5]: changed probes of the item, per channel
  uint8_t* state_s = smem + tp.off_state;
  uint16_t* last_s = (uint16_t*)(smem + tp.off_last);
  float* ms = (float*)(smem + tp.off_ms);          // [32][MS_LD]: accumulators, transposed

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
  for (int t = threadIdx.x; t < k.Tc + k.Tv; t += NT) {
    const bool vis = t >= k.Tc;
    const float S = k.sums[t];
    rsum[vis ? tp.Nc + (t - k.Tc) : t] = S > 0.0f ? 1.0f / S : 0.0f;
    const int n = vis ? k.nv : k.nc, tt = vis ? t - k.Tc : t;
    const int i = tt / n, j = tt % n;
    tab_pos[t] = (uint16_t)((i + 1) * (n + 2) + (j + 1));
    tab_border[t] = pack_border(i, j, n);
  }
  for (int q = threadIdx.x; q < 5; q += NT) flag_mask[q] = 0;
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
  int* err = k.err;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < tp.items && ok; item += gridDim.x) {
        const int p0 = item * np;
        // ray and weight tiles, chunk by chunk
        for (int kc = 0; kc < tp.nchunks; ++kc) {
          ok = mbar_wait(&empty[s], ph ^ 1, err);
          if (!ok) break;
          uint8_t* st = smem + (size_t)s * tp.stage_bytes;
          const int x = kc * tp.kc;
          mbar_expect_tx(&full[s], tp.stage_tx);
          tma_load_2d(st, &map_dist, x, p0, &full[s]);
          for (int c = 0; c < 3; ++c)
            tma_load_2d(st + (size_t)(tp.crow + c * GRP) * ROWB, &map_rad, x, c * k.P + p0, &full[s]);
          tma_load_2d(st + tp.off_wc, &map_wc, x, 0, &full[s]);
          tma_load_2d(st + tp.off_wv, &map_wv, x, 0, &full[s]);
          if (kSplitW) {
            tma_load_2d(st + tp.off_wc_lo, &map_wc_lo, x, 0, &full[s]);
            tma_load_2d(st + tp.off_wv_lo, &map_wv_lo, x, 0, &full[s]);
          }
          if (++s == tp.stages) {
            s = 0;
            ph ^= 1;
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int s = 0, b = 0;
      uint32_t ph = 0, tph = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < tp.items && ok; item += gridDim.x) {
        ok = mbar_wait(&tempty[b], tph ^ 1, err);
        if (!ok) break;
        tc_fence_after();
        const uint32_t dv = tmem + b * 256 + tp.col_v;
        const uint32_t dc = tmem + b * 256 + tp.col_c;
        for (int kc = 0; kc < tp.nchunks; ++kc) {
          ok = mbar_wait(&conv[s], ph, err);
          if (!ok) break;
          tc_fence_after();
          uint8_t* st = smem + (size_t)s * tp.stage_bytes;
#pragma unroll
          for (int ks = 0; ks < ROWB / 32; ++ks) {     // one MMA K step per 32 bytes of row
            const int kb = ks * 32;
            const uint64_t av = sdesc<ROWB>(st + kb);
            const uint64_t ac = sdesc<ROWB>(st + (size_t)(tp.crow + 3 * GRP - 128) * ROWB + kb);
            const uint64_t bv = sdesc<ROWB>(st + tp.off_wv + kb);
            const uint64_t bc = sdesc<ROWB>(st + tp.off_wc + kb);
            const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
            mma<FORM>(dv, av, bv, tp.idesc_v, acc);
            mma<FORM>(dc, ac, bc, tp.idesc_c, acc);
            if (kSplitW) {
              mma<FORM>(dv, av, sdesc<ROWB>(st + tp.off_wv_lo + kb), tp.idesc_v, 1u);
              mma<FORM>(dc, ac, sdesc<ROWB>(st + tp.off_wc_lo + kb), tp.idesc_c, 1u);
            }
            if (kSplitA) {
              uint8_t* lo = st + tp.off_a_lo;
              mma<FORM>(dv, sdesc<ROWB>(lo + kb), bv, tp.idesc_v, 1u);
              mma<FORM>(dc, sdesc<ROWB>(lo + (size_t)(tp.crow + 3 * GRP - 128) * ROWB + kb), bc, tp.idesc_c, 1u);
            }
          }
          mma_commit(&empty[s]);                       // stage free once these MMAs finish
          if (++s == tp.stages) {
            s = 0;
            ph ^= 1;
          }
        }
        if (!ok) break;
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
    for (int item = blockIdx.x; item < tp.items && ok; item += gridDim.x) {
      for (int kc = 0; kc < tp.nchunks; ++kc) {
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
          constexpr int ACH = 160 * CPR / 64;          // chunks per thread over the A tile's 160 rows
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
          // d^2 = hi + lo in the operand format (binary16 scaled by 2^-8)
          for (int q = ct; q < GRP * CPR; q += 64) {
            const uint4 raw = *(const uint4*)(st + (size_t)q * 16);
            const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
            uint32_t oh[4], ol[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              float d0, d1;
              if constexpr (FORM == kF16) {
                const __half2 h2 = *reinterpret_cast<const __half2*>(&w[e]);
                d0 = __low2float(h2);
                d1 = __high2float(h2);
              } else {
                const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&w[e]);
                d0 = __low2float(h2);
                d1 = __high2float(h2);
              }
              const float sc = FORM == kF16 ? 0.00390625f : 1.0f;
              const float q0 = d0 * d0 * sc, q1 = d1 * d1 * sc;
              if constexpr (FORM == kF16) {
                const __half h0 = __float2half_rn(q0), h1 = __float2half_rn(q1);
                const __half l0 = __float2half_rn(q0 - __half2float(h0));
                const __half l1 = __float2half_rn(q1 - __half2float(h1));
                oh[e] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
                ol[e] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
              } else {
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
    const int e = threadIdx.x - 128;                   // 0..255
    const int ew = e >> 5;                             // epilogue warp 0..7
    const int quarter = warp & 3;                      // TMEM lanes 32*quarter .. +32
    const int half = ew >> 2;                          // which 16-column half of a pass it loads
    const float h = *k.hy, omh = 1.0f - h;
    const float d2_scale = FORM == kF16 ? 256.0f : 1.0f;
    constexpr bool d2_lo = FORM != kF32;               // d^2 lo rows at lanes 64..95
    const int kind = k.color_code;
    int b = 0;
    uint32_t tph = 0, eph = 0;
    bool ok = true;
    // thread 0 streams each item's old texels and codes into shared memory as
    // soon as the previous item's tiles have been written back
    if (e == 0 && blockIdx.x < tp.items) prefetch_item(k, np, blockIdx.x * np, sb, st_c, st_v, ls_c, ls_v, efull);
    for (int item = blockIdx.x; item < tp.items && ok; item += gridDim.x) {
      const int p0 = item * np;
      const int npi = min(np, k.P - p0);
      ok = mbar_wait(efull, eph, err);
      if (ok) ok = mbar_wait(&tfull[b], tph, err);
      if (!ok) break;
      eph ^= 1;
      tc_fence_after();
      const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + b * 256;
      const int npass_c = (k.Tc + 31) / 32, npass_v = (k.Tv + 31) / 32;
      for (int pass = 0; pass < npass_c + npass_v; ++pass) {
        const bool vis = pass >= npass_c;
        const int blk = vis ? pass - npass_c : pass;
        const int N = vis ? tp.Nv : tp.Nc;
        const int c16 = 32 * blk + 16 * half;          // first of the 16 columns this warp loads
        if (c16 < N) {
          float v[16];
          tmem_ld16(trow + (vis ? tp.col_v : tp.col_c) + c16, v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) ms[(16 * half + j) * MS_LD + quarter * 32 + lane] = v[j];
        }
        epi_bar();
        // lane <-> texel t of this pass; constants of that texel
        const int T = vis ? k.Tv : k.Tc;
        const int t = 32 * blk + lane;
        LaneTexel lt;
        lt.has = t < T;
        const int tg = lt.has ? (vis ? k.Tc + t : t) : 0;
        const uint64_t bord = tab_border[tg];
        lt.pos = tab_pos[tg];
        lt.nb = lt.has ? (int)(bord >> 48) : 0;
        lt.b0 = (uint32_t)(bord & 0xFFFFu);
        lt.b1 = (uint32_t)((bord >> 16) & 0xFFFFu);
        lt.b2 = (uint32_t)((bord >> 32) & 0xFFFFu);
        lt.rS = lt.has ? rsum[(vis ? tp.Nc : 0) + t] : 0.0f;
        lt.t = lt.has ? t : 0;
        const float* mcol = ms + lane * MS_LD;
        void* tiles = vis ? (void*)st_v : (void*)st_c;
        const int tile_elems = vis ? k.sv_stride : k.sc_stride;
        const uint16_t* codes = vis ? ls_v : ls_c;
        const int code_elems = vis ? k.lv_stride : k.lc_stride;
        const bool f16 = k.state_fmt == PV_FMT_F16;
        if (vis) {
          if (f16) epi_pass<0, 0, true, d2_lo>(lt, mcol, npi, np, tiles, tile_elems, codes, code_elems, h, omh, d2_scale, ew, lane, flag_mask);
          else epi_pass<1, 0, true, d2_lo>(lt, mcol, npi, np, tiles, tile_elems, codes, code_elems, h, omh, d2_scale, ew, lane, flag_mask);
        } else if (kind == PV_CODE_UNORM10) {
          if (f16) epi_pass<0, PV_CODE_UNORM10, false, false>(lt, mcol, npi, np, tiles, tile_elems, codes, code_elems, h, omh, 1.0f, ew, lane, flag_mask);
          else epi_pass<1, PV_CODE_UNORM10, false, false>(lt, mcol, npi, np, tiles, tile_elems, codes, code_elems, h, omh, 1.0f, ew, lane, flag_mask);
        } else {
          if (f16) epi_pass<0, PV_CODE_UF10, false, false>(lt, mcol, npi, np, tiles, tile_elems, codes, code_elems, h, omh, 1.0f, ew, lane, flag_mask);
          else epi_pass<1, PV_CODE_UF10, false, false>(lt, mcol, npi, np, tiles, tile_elems, codes, code_elems, h, omh, 1.0f, ew, lane, flag_mask);
        }
        epi_bar();
      }
      // accumulators consumed: hand the TMEM buffer back to the MMA thread
      tc_fence_before();
      mbar_arrive(&tempty[b]);
      if (++b == tp.nbuf) {
        b = 0;
        tph ^= 1;
      }
      if (e < 2) {                                     // changed-probe bits of this item
        const uint32_t m = e == 0 ? (flag_mask[0] | flag_mask[1] | flag_mask[2]) : (flag_mask[3] | flag_mask[4]);
        const int sh = p0 & 31;
        uint32_t* w = &k.chg[e * k.chg_words + (p0 >> 5)];
        if (m << sh) atomicOr(w, m << sh);
        if (sh && (m >> (32 - sh))) atomicOr(w + 1, m >> (32 - sh));
      }
      epi_bar();
      if (e < 5) flag_mask[e] = 0;
      fence_proxy_async();
      epi_bar();
      if (e == 0) {
        const uint32_t sc_b = (uint32_t)npi * k.sc_stride * sb, sv_b = (uint32_t)npi * k.sv_stride * sb;
        for (int c = 0; c < 3; ++c)
          bulk_s2g((uint8_t*)k.state_c + ((size_t)c * k.P + p0) * k.sc_stride * sb,
                   st_c + (size_t)c * np * k.sc_stride * sb, sc_b);
        for (int c = 0; c < 2; ++c)
          bulk_s2g((uint8_t*)k.state_v + ((size_t)c * k.P + p0) * k.sv_stride * sb,
                   st_v + (size_t)c * np * k.sv_stride * sb, sv_b);
        bulk_commit();
        bulk_wait_read();                              // shared tiles may be refilled now
        const int next = item + gridDim.x;
        if (next < tp.items) prefetch_item(k, np, next * np, sb, st_c, st_v, ls_c, ls_v, efull);
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
struct TcPlan {
  TcParams tp;
  CUtensorMap wc, wv, wc_lo, wv_lo;
  size_t smem;
  int grid;
  int form;
};

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

}  // namespace

bool pv_tc_supported(const pv_desc* d, const char** why) {
  const int ob = d->operand_fmt == PV_FMT_F32 ? 4 : 2;
  const int nc = d->color_interior, nv = d->vis_interior;
  const int Nc = ((nc * nc + 15) / 16) * 16, Nv = ((nv * nv + 15) / 16) * 16;
  if (nc < 2 || nv < 2) {
    if (why) *why = "tile interiors below 2x2 (guard-band table holds three copies per texel)";
    return false;
  }
  if ((d->rays_per_probe * ob) % 16 != 0) {
    if (why) *why = "rays_per_probe * operand bytes must be a multiple of 16 (TMA row pitch)";
    return false;
  }
  if (Nc + Nv > 512 || Nv > 256 || Nc > 256) {
    if (why) *why = "tile interiors too large for the tensor-memory accumulators";
    return false;
  }
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaGetLastError();
  if (!(major == 10 && minor == 3)) {
    if (why) *why = "needs an sm_103 GPU (GB300)";
    return false;
  }
  return true;
}

cudaError_t pv_tc_plan_create(pv_volume* v) {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  TcPlan* pl = new TcPlan();
  memset(pl, 0, sizeof(TcPlan));
  TcParams& tp = pl->tp;
  const pv_dev& k = v->k;
  tp.k = k;
  const int form = k.operand_fmt == PV_FMT_F16 ? kF16 : (k.operand_fmt == PV_FMT_BF16 ? kBF16 : kF32);
  pl->form = form;
  const int ob = form == kF32 ? 4 : 2;
  int dev = 0, sms = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int sb = v->state_bytes;
  const int np_max = sb == 2 ? 32 : 16;
  int np = (k.P + sms - 1) / sms;
  np = np < 1 ? 1 : (np > np_max ? np_max : np);
  tp.np = np;
  tp.items = (k.P + np - 1) / np;
  pl->grid = tp.items < sms ? tp.items : sms;
  const int ROWB = form == kF32 ? row_bytes<kF32>() : row_bytes<kF16>();
  tp.kc = ROWB / ob;
  tp.nchunks = (k.R + tp.kc - 1) / tp.kc;
  tp.Nc = k.tc_pad;
  tp.Nv = k.tv_pad;
  tp.nbuf = tp.Nc + tp.Nv <= 256 ? 2 : 1;
  tp.col_v = 0;
  tp.col_c = tp.Nv;
  tp.a_rows = form == kF32 ? 160 : 192;
  tp.crow = form == kF32 ? 64 : 96;
  // stage layout
  size_t off = 0;
  const size_t a_b = align1k((size_t)tp.a_rows * ROWB);
  off += a_b;
  tp.off_a_lo = (int)off;
  if (form == kF32) off += a_b;
  tp.off_wc = (int)off;
  off += align1k((size_t)tp.Nc * ROWB);
  tp.off_wv = (int)off;
  off += align1k((size_t)tp.Nv * ROWB);
  tp.off_wc_lo = (int)off;
  if (form != kF16) off += align1k((size_t)tp.Nc * ROWB);
  tp.off_wv_lo = (int)off;
  if (form != kF16) off += align1k((size_t)tp.Nv * ROWB);
  tp.stage_bytes = (int)off;
  tp.stage_tx = (uint32_t)((4 * np + (form != kF16 ? 2 : 1) * (tp.Nc + tp.Nv)) * ROWB);
  // epilogue region
  const size_t epi_state = (size_t)np * (3 * k.sc_stride + 2 * k.sv_stride) * sb;
  const size_t epi_last = (size_t)np * (3 * k.lc_stride + 2 * k.lv_stride) * 2;
  const size_t tab = (size_t)(k.Tc + k.Tv) * 10;
  const size_t epi = align1k(epi_state) + align1k(epi_last) + align1k((size_t)32 * MS_LD * 4) +
                     align1k((size_t)(tp.Nc + tp.Nv) * 4) + align1k(5 * GRP * 4) + align1k(tab) + 1024;
  const size_t budget = (size_t)smem_max - 1024 - epi;
  int stages = (int)(budget / tp.stage_bytes);
  if (stages > 4) stages = 4;
  if (stages < 2) {
    delete pl;
    return cudaErrorInvalidConfiguration;
  }
  tp.stages = stages;
  off = (size_t)stages * tp.stage_bytes;
  tp.off_state = (int)off;
  off += align1k(epi_state);
  tp.off_last = (int)off;
  off += align1k(epi_last);
  tp.off_ms = (int)off;
  off += align1k((size_t)32 * MS_LD * 4);
  tp.off_invs = (int)off;
  off += align1k((size_t)(tp.Nc + tp.Nv) * 4);
  tp.off_flags = (int)off;
  off += align1k(5 * GRP * 4);
  tp.off_tab = (int)off;
  off += align1k(tab);
  tp.off_bar = (int)off;
  off += 1024;
  pl->smem = off + 1024;                       // slack for aligning the dynamic base
  tp.idesc_c = make_idesc(form, 128, tp.Nc);
  tp.idesc_v = make_idesc(form, 128, tp.Nv);
  // weight tensor maps (fixed for the volume's life)
  const size_t plane = (size_t)(k.tc_pad + k.tv_pad) * k.r_pad;
  const uint8_t* w = (const uint8_t*)k.w_op;
  e = encode_2d(&pl->wc, k.operand_fmt, w, k.r_pad, k.tc_pad, (uint64_t)k.r_pad * ob, tp.kc, tp.Nc);
  if (e == cudaSuccess)
    e = encode_2d(&pl->wv, k.operand_fmt, w + (size_t)k.tc_pad * k.r_pad * ob, k.r_pad, k.tv_pad,
                  (uint64_t)k.r_pad * ob, tp.kc, tp.Nv);
  if (e == cudaSuccess && form != kF16) {
    e = encode_2d(&pl->wc_lo, k.operand_fmt, w + plane * ob, k.r_pad, k.tc_pad, (uint64_t)k.r_pad * ob,
                  tp.kc, tp.Nc);
    if (e == cudaSuccess)
      e = encode_2d(&pl->wv_lo, k.operand_fmt, w + (plane + (size_t)k.tc_pad * k.r_pad) * ob, k.r_pad,
                    k.tv_pad, (uint64_t)k.r_pad * ob, tp.kc, tp.Nv);
  } else {
    pl->wc_lo = pl->wc;
    pl->wv_lo = pl->wv;
  }
  if (e == cudaSuccess) {
    if (form == kF16)
      e = cudaFuncSetAttribute(k_blend_tc<kF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl->smem);
    else if (form == kBF16)
      e = cudaFuncSetAttribute(k_blend_tc<kBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl->smem);
    else
      e = cudaFuncSetAttribute(k_blend_tc<kF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl->smem);
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
  const pv_dev& k = v->k;
  const int ob = pl->form == kF32 ? 4 : 2;
  CUtensorMap mr, md;
  cudaError_t e = encode_2d(&mr, k.operand_fmt, rad, k.R, (uint64_t)3 * k.P, (uint64_t)k.R * ob,
                            pl->tp.kc, pl->tp.np);
  if (e == cudaSuccess)
    e = encode_2d(&md, k.operand_fmt, dist, k.R, k.P, (uint64_t)k.R * ob, pl->tp.kc, pl->tp.np);
  if (e != cudaSuccess) return e;
  TcParams tp = pl->tp;
  tp.k = k;
  switch (pl->form) {
    case kF16:
      k_blend_tc<kF16><<<pl->grid, NT, pl->smem, st>>>(tp, mr, md, pl->wc, pl->wv, pl->wc_lo, pl->wv_lo);
      break;
    case kBF16:
      k_blend_tc<kBF16><<<pl->grid, NT, pl->smem, st>>>(tp, mr, md, pl->wc, pl->wv, pl->wc_lo, pl->wv_lo);
      break;
    default:
      k_blend_tc<kF32><<<pl->grid, NT, pl->smem, st>>>(tp, mr, md, pl->wc, pl->wv, pl->wc_lo, pl->wv_lo);
      break;
  }
  return cudaGetLastError();
}
