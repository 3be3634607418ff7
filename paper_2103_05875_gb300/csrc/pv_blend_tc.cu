// K1 (tensor-core form): the probe blend of Section 3.2 of arXiv 2103.05875 as
// a tcgen05 contraction with a fused epilogue, for sm_103a.
//
// The blend is a dense contraction because every probe of a volume shares the
// frame's ray directions: for a probe row x (one colour channel, d or d^2 of
// one probe) and a texel t, acc[x, t] = sum_r x[r] W[t, r]. Probe rows form
// the MMA's M dimension, so one tensor-memory lane holds one probe row and one
// epilogue thread owns it; texels form N, rays K:
//
//   A (probe rows, K-major): lane quarter q holds one channel of the work
//     item's probes (lane 32q + j = probe j of the item, np <= 32):
//       visibility phase: q0 = d, q1 = d^2
//       colour phase:     q1 = R, q2 = G, q3 = B
//     FP32 form: the rays arrive by TMA in shared memory and converter warps
//     split them into TF32 hi + lo parts held in tensor memory (A from TMEM,
//     so the MMAs read only the weights from shared memory). 16-bit forms:
//     A is the TMA tile itself in shared memory; d^2 = hi + lo is formed on
//     chip, the lo part in a second A tile whose d lanes are zero.
//   B (texels, K-major): the weights kernel writes each K chunk as the exact
//     swizzled shared-memory image of [visibility texels | colour texels],
//     each block padded to 16 rows, so a chunk's block arrives with one bulk
//     copy per plane.
//   D (tensor memory, FP32): visibility accumulators in columns [0, NVP),
//     colour from the next multiple of 32 on (NCP columns); one per texel, in
//     interior order. The FP32 form's A ring follows them.
//
// Each work item runs a visibility phase (all ray chunks), then a colour
// phase. The visibility epilogue runs while the colour phase's loads and MMAs
// are in flight, and the colour epilogue while the next item's visibility
// phase is, so the tensor pipe and the epilogue overlap even with one item
// per CTA.
//
// Operand forms (pv_desc.operand_fmt):
//   F32  kind::tf32; x = x_hi + x_lo and W = W_hi + W_lo with TF32 parts,
//        three MMAs (hi*hi + hi*lo + lo*hi) recover float32 accuracy.
//   F16  kind::f16, binary16; visibility weights scaled by 2^15 and d^2 by
//        2^-4 (both undone exactly) to stay in range; d^2 as hi + lo.
//   BF16 kind::f16 with bfloat16; W = W_hi + W_lo, d^2 as hi + lo.
//
// Epilogue (one thread per probe row, two warps per lane quarter): a thread
// updates its probe's tile two interior rows at a time, row i with its
// mirror row n-1-i, because each one's guard-band texels are copies of the
// other's first and last texels (the octahedral rule of Section 3.4; the
// pair of row 0 also makes the top and bottom guard rows). Per texel: weight-
// sum normalisation and hysteresis (Section 3.2), rounding to the state
// format, the transmitted code (Section 3.3) and its comparison with the last
// transmitted code (Section 3.4). Tile rows move through shared memory as
// 16-byte vectors (rows padded so that the 32 lanes of a warp hit distinct
// banks); each thread moves its own probe row between global and shared
// memory with bulk copies, and streams in its next item's old texels and
// codes as soon as this item's are written back.
//
// Warp roles (512 threads, one CTA per SM, persistent over work items):
//   warp 0      ray producer (TMA), running ahead from the kernel's start
//   warp 1      TMEM allocation
//   warp 2      weight producer (bulk copies of the weight tile images)
//   warp 3      the single MMA-issuing thread
//   warps 4-7   converters (lane quarter = warp % 4): TF32 split into TMEM
//               (F32), d^2 hi + lo into shared memory (16-bit forms)
//   warps 8-15  epilogue, two per lane quarter
// Programmatic dependent launch: the kernel lets its successor launch at its
// start and runs its set-up (barriers, TMEM, tensor-map prefetch) before
// waiting for its predecessor; each role waits only before its first read of
// memory a predecessor wrote. Every mbarrier wait is bounded in time; on
// expiry the kernel raises the volume's error word and every role finishes
// its loop without further work, so no wait can hang the GPU.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "pv_codes.cuh"
#include "pv_internal.h"

namespace {

enum Form { kF16 = 0, kBF16 = 1, kF32 = 2 };

constexpr int NT = 512;
constexpr int ROWB = 64;                 // bytes per K-chunk row (SWIZZLE_64B): 16 FP32 or 32 16-bit rays
constexpr int QROWS = 32;                // probe rows per lane quarter
constexpr int A_BYTES = 128 * ROWB;      // one 128-row A tile of a stage
constexpr int EPI_THREADS = 256;         // warps 8..15
// exchange of the visibility accumulators' second parts between lane
// quarters: per lane two interior rows of up to 16 texels (4-byte floats,
// a row of 8 16-byte units: distinct bank groups for 8 consecutive lanes),
// two buffers per warp pair
constexpr uint32_t XROW_BYTES = 2 * 14 * 4;
constexpr uint32_t XBUF_BYTES = 32 * XROW_BYTES;
// Bound of every mbarrier wait, in SM clock cycles: 4e9 is 2 s at 2 GHz
// (1.9 s at the 2.07 GHz maximum, longer at lower clocks).
constexpr long long kWaitCycles = 4000000000ll;
// Chunk rings: per K chunk n (counted over the CTA's run) one "ready" barrier
// (operands in place) and one "done" barrier (the chunk's MMAs completed), in
// rings of kRing; slot n % kRing, phase parity (n / kRing) % 2.
constexpr int kRing = 16;
// binary16 operand form: d^2 enters the MMA scaled by 2^-4 (exact), which
// keeps the high part of d^2 for hit distances up to 2^10 in binary16 range
constexpr float kD2ScaleF16 = 0.0625f;

__host__ __device__ constexpr int round_up_c(int x, int a) { return (x + a - 1) / a * a; }

// Interior sizes the kernel is compiled for, with their derived shapes.
template <int NC, int NV>
struct Shape {
  static constexpr int TC = NC * NC, TV = NV * NV;
  static constexpr int NCP = round_up_c(TC, 16), NVP = round_up_c(TV, 16);   // MMA N of each phase
  static constexpr int WROWS = NCP > NVP ? NCP : NVP;
  static constexpr int CBASE = round_up_c(NVP, 32);                          // TMEM column of the colour accumulators
  static constexpr int RPC = round_up_c(NC, 4), RPV = round_up_c(NV, 4);     // table row pitch (floats)
};

struct TcParams {
  pv_dev k;                              // shapes and formats shared by the volumes of the launch
  int np, items, kc;                     // probes per item, items, rays per chunk
  int xs, ws, as_;                       // ring depths: ray tiles, weight tiles, F32 TMEM A tiles
  int xstage, wstage;                    // bytes per ray stage (A tile [+ lo A tile]) and weight stage
  int off_xr, off_wr;                    // the two rings
  int off_tv, off_lv, off_tc, off_lc;    // epilogue regions: visibility tiles / codes, colour tiles / codes
  int boxb;                              // bytes reserved per tile box (np rows of 128 bytes, 1024-aligned)
  int lreg_v, lreg_c;                    // bytes reserved per channel of code rows (np dense rows)
  int off_cf, off_km, off_xb, off_bar;   // tables, exchange buffers, barriers
  uint32_t tx_xv, tx_xc, tx_wv, tx_wc;   // bytes per ray / weight stage, visibility / colour phase
  uint32_t idesc_v, idesc_c, idesc_c2;   // instruction descriptors (N = NVP, NCP, 2 NCP)
  int abase;                             // F32: first TMEM column of the A ring (32 columns per stage)
};

// One volume of a launch: its tensor maps, its buffers and its work items.
// The epilogue moves texels and codes with 3-D maps [channel][probe][row]:
// texels in boxes of 128-byte column strips of np probe rows (SWIZZLE_128B),
// codes in one box of np whole rows.
struct BlendVol {
  CUtensorMap rad, dist;                 // this frame's rays
  CUtensorMap st_v, st_c;                // state tiles (read and written)
  CUtensorMap last_v, last_c;            // last-transmitted codes (read)
  CUtensorMap cur_v, cur_c;              // current codes (written)
  pv_dev k;
  int item0;                             // first work item of the volume in the launch
  int nchunks;                           // ray chunks of kc rays
};

template <int MAXV>
struct BlendArgs {
  TcParams tp;
  int nvol;
  BlendVol v[MAXV];
};

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
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false if it expired or
// another role already gave up. A phase that has completed already is seen
// by a non-blocking test, without the cost of a potentially suspending wait.
__device__ __noinline__ bool mbar_wait_slow(uint64_t* b, uint32_t parity, int* err);
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err) {
  return mbar_test(b, parity) || mbar_wait_slow(b, parity, err);
}
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* b, uint32_t parity, int* err) {
  // the common case (phase already complete) through a non-blocking test and a
  // vote, so that the branch around the bounded wait is warp-uniform
  if (__all_sync(0xffffffffu, mbar_test(b, parity))) return true;
  return __all_sync(0xffffffffu, mbar_wait_slow(b, parity, err));
}
// The MMAs of chunk m are complete (always true for m < 0). A role refilling a
// stage last read by chunk m waits here; a later phase of the same slot cannot
// mislead the parity test, since chunk m + kRing needs the stage refilled first.
__device__ __forceinline__ bool wait_done_warp(uint64_t* done, int m, int* err) {
  return m < 0 || mbar_wait_warp(&done[m & (kRing - 1)], (uint32_t)((m / kRing) & 1), err);
}
__device__ __noinline__ bool mbar_wait_slow(uint64_t* b, uint32_t parity, int* err) {
  // The deadline is kept with the SM's cycle counter: reading the global
  // timer costs hundreds of cycles, which every wait that blocks would pay
  // before it could see its phase complete.
  if (mbar_try(b, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 64; ++i)
      if (mbar_try(b, parity)) return true;
    if (*(volatile int*)err) return false;
    if (clock64() - t0 > kWaitCycles) {
      atomicExch(err, 1);
      return false;
    }
  }
}
// One lane of the (converged) warp; the issuing roles run their loops with the
// whole warp, so that addresses and descriptors stay warp-uniform, and let the
// elected lane issue the asynchronous instructions.
__device__ __forceinline__ bool elect_one() {
  uint32_t p;
  asm volatile(
      "{\n .reg .b32 r;\n .reg .pred e;\n elect.sync r|e, 0xffffffff;\n selp.u32 %0, 1, 0, e;\n}\n"
      : "=r"(p));
  return p != 0;
}
// Bounded wait by every lane of a warp; the result is the same in all lanes.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* b, uint32_t parity, int* err);
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void named_bar(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
// Named barrier that also returns the AND of every participant's flag, so
// that the threads meeting there take the same branch afterwards.
__device__ __forceinline__ bool named_bar_and(int id, int threads, bool flag) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.b32 a, %1, 0;\n bar.red.and.pred b, %2, %3, a;\n selp.u32 %0, 1, 0, b;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)flag), "r"(id), "r"(threads)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map),
               "r"(x), "r"(y), "r"(z), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D (+)= A * B with A and B in shared memory.
template <int FORM>
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
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
// D (+)= A * B with A in tensor memory (TF32), B in shared memory.
__device__ __forceinline__ void mma_ts_tf32(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// Two accumulator columns of this thread's TMEM lane (issued; completed by tmem_wait_ld).
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float& x, float& y) {
  uint32_t r0, r1;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr));
  x = __uint_as_float(r0);
  y = __uint_as_float(r1);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major rows of 64 bytes with SWIZZLE_64B,
// 8-row groups 512 bytes apart (SBO); LBO unused for this layout; version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t a) {
  uint64_t d = 0;
  d |= (uint64_t)((a & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Byte offset of 16-byte unit u of row r in a SWIZZLE_64B tile (512-byte aligned).
__device__ __forceinline__ uint32_t swz64(int r, int u) { return (uint32_t)(r * 64 + ((u ^ ((r >> 1) & 3)) << 4)); }

__device__ __forceinline__ void lds128(uint32_t a, uint32_t& x, uint32_t& y, uint32_t& z, uint32_t& w) {
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(x), "=r"(y), "=r"(z), "=r"(w) : "r"(a));
}
__device__ __forceinline__ void lds128f(uint32_t a, float& x, float& y, float& z, float& w) {
  asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(x), "=f"(y), "=f"(z), "=f"(w) : "r"(a));
}
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
// Stores only where `on` is set (predicate inside the instruction).
__device__ __forceinline__ void sts128_if(bool on, uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %5, 0;\n @q st.shared.v4.u32 [%0], {%1,%2,%3,%4};\n}\n" ::"r"(a),
               "r"(x), "r"(y), "r"(z), "r"(w), "r"((uint32_t)on)
               : "memory");
}
__device__ __forceinline__ void sts32_if(bool on, uint32_t a, uint32_t v) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q st.shared.u32 [%0], %1;\n}\n" ::"r"(a), "r"(v),
               "r"((uint32_t)on)
               : "memory");
}

// ------------------------------------------------------------------ epilogue
// One probe row's bytes in a set of 128-byte boxes (SWIZZLE_128B, 1024-byte
// aligned): byte o of the row sits in box o / 128, at row r of that box, in
// 16-byte unit ((o / 16) % 8) XOR (r % 8). Eight consecutive rows therefore
// put the same unit in eight different bank groups.
struct BoxRow {
  uint32_t base, boxb, roff, rx;
};
__device__ __forceinline__ BoxRow box_row(uint32_t base, uint32_t boxb, int r) {
  return BoxRow{base, boxb, (uint32_t)r * 128u, (uint32_t)(r & 7)};
}
__device__ __forceinline__ uint32_t at(const BoxRow& b, uint32_t o) {
  return b.base + (o >> 7) * b.boxb + b.roff + ((((o >> 4) & 7u) ^ b.rx) << 4) + (o & 15u);
}

// Stored texels: SB = 2 (binary16) or 4 (binary32) bytes.
template <int SB>
__device__ __forceinline__ float state_value(uint32_t b) {
  if constexpr (SB == 2) return __half2float(__ushort_as_half((unsigned short)b));
  else return __uint_as_float(b);
}
template <int SB>
__device__ __forceinline__ uint32_t state_bits(float v) {
  if constexpr (SB == 2) return (uint32_t)__half_as_ushort(__float2half_rn(v));
  else return __float_as_uint(v);
}
// Element e of a tile row held as 32-bit words.
template <int SB, int RW>
__device__ __forceinline__ uint32_t row_el(const uint32_t (&w)[RW], int e) {
  if constexpr (SB == 4) return w[e];
  else return (e & 1) ? (w[e >> 1] >> 16) : (w[e >> 1] & 0xFFFFu);
}
// Transmitted code of a stored texel (Sections 3.3-3.4): visibility as
// binary16 bits, colour as UF10 or UNORM10.
template <int SB, int KIND, bool VIS>
__device__ __forceinline__ uint32_t texel_code(uint32_t b) {
  if constexpr (VIS) {
    if constexpr (SB == 2) return b;
    else return (uint32_t)__half_as_ushort(__float2half_rn(__uint_as_float(b)));
  } else if constexpr (KIND == PV_CODE_UNORM10) {
    return pv::unorm10_from_float(state_value<SB>(b));
  } else {
    if constexpr (SB == 2) return pv::uf10_from_half_bits(b);
    else return pv::uf10_from_float_bits(b);
  }
}

// Loads of interior row i of this thread's probe row, issued without waiting:
// its accumulators (TMEM; with tsplit > 0 also the second column block this
// far apart, the weights' lo part, which is added) and its old tile row i + 1.
template <int N, int SB>
struct RowIn {
  float acc[N], lo[N];
  uint32_t w[(N + 2) * SB / 4];
};
template <int N, int SB>
__device__ __forceinline__ void load_row(uint32_t tm, uint32_t tsplit, const BoxRow& tb, int ti, RowIn<N, SB>& r) {
  constexpr int RW = (N + 2) * SB / 4;
#pragma unroll
  for (int m = 0; m < N / 2; ++m) tmem_ld2(tm + 2u * m, r.acc[2 * m], r.acc[2 * m + 1]);
  if (tsplit) {
#pragma unroll
    for (int m = 0; m < N / 2; ++m) tmem_ld2(tm + tsplit + 2u * m, r.lo[2 * m], r.lo[2 * m + 1]);
  }
#pragma unroll
  for (int c = 0; c < RW / 4; ++c)
    lds128(at(tb, (uint32_t)ti * (RW * 4) + 16u * c), r.w[4 * c], r.w[4 * c + 1], r.w[4 * c + 2], r.w[4 * c + 3]);
}

// Interior row i once its loads completed: new stored bits nb[j] and the
// transmitted codes in pairs cw[m] = code(2m) | code(2m+1) << 16.
//   s_cf    shared address of the row's factors (1 - h) * scale / S per texel
//   km      texels of the row whose weight sum is 0 (bit j): they keep their value
template <int N, int SB, int KIND, bool VIS>
__device__ __forceinline__ void finish_row(RowIn<N, SB>& r, bool split, uint32_t s_cf, uint32_t km, float h,
                                           uint32_t (&nb)[N], uint32_t (&cw)[N / 2]) {
  constexpr int RW = (N + 2) * SB / 4;
  constexpr int RP = round_up_c(N, 4);
  float cf[RP];
#pragma unroll
  for (int c = 0; c < RP / 4; ++c) lds128f(s_cf + 16u * c, cf[4 * c], cf[4 * c + 1], cf[4 * c + 2], cf[4 * c + 3]);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const float acc = split ? r.acc[j] + r.lo[j] : r.acc[j];
    const float of = state_value<SB>(row_el<SB, RW>(r.w, j + 1));
    nb[j] = state_bits<SB>(fmaf(h, of, acc * cf[j]));
  }
  if (km) {                                          // rare: texels without any weight
#pragma unroll
    for (int j = 0; j < N; ++j)
      if ((km >> j) & 1u) nb[j] = row_el<SB, RW>(r.w, j + 1);
  }
#pragma unroll
  for (int m = 0; m < N / 2; ++m)
    cw[m] = texel_code<SB, KIND, VIS>(nb[2 * m]) | (texel_code<SB, KIND, VIS>(nb[2 * m + 1]) << 16);
}

// Tile row ti: guard texel L, interior v[0..N-1], guard texel R.
template <int N, int SB>
__device__ __forceinline__ void store_row(bool on, const BoxRow& tb, int ti, uint32_t L, const uint32_t (&v)[N],
                                          uint32_t R) {
  constexpr int RW = (N + 2) * SB / 4;
  uint32_t w[RW];
#pragma unroll
  for (int k = 0; k < RW; ++k) {
    if constexpr (SB == 4) {
      w[k] = k == 0 ? L : (k == N + 1 ? R : v[k - 1 < N ? (k - 1 < 0 ? 0 : k - 1) : N - 1]);
    } else {
      const int e0 = 2 * k, e1 = 2 * k + 1;
      const uint32_t a = e0 == 0 ? L : v[e0 - 1 < N ? e0 - 1 : N - 1];
      const uint32_t b = e1 == N + 1 ? R : v[e1 - 1 < N ? e1 - 1 : N - 1];
      w[k] = a | (b << 16);
    }
  }
#pragma unroll
  for (int c = 0; c < RW / 4; ++c)
    sts128_if(on, at(tb, (uint32_t)ti * (RW * 4) + 16u * c), w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
}

// Interior rows i and N-1-i of this thread's tile with the guard texels they
// determine (Section 3.4's octahedral guard band): the left / right guard
// texel of tile row r copies interior texel (N-r, 0) / (N-r, N-1), i.e. the
// first / last texel of the mirror row; the top guard row is interior row 0
// reversed, the bottom one interior row N-1 reversed, the corners the
// diagonally opposite interior corners. Writes the tile rows and the codes,
// and returns whether any code differs from the last transmitted one.
template <int N, int SB, int KIND, bool VIS>
//   xb      != 0: the rows' second parts come from the partner warp through
//           this exchange buffer (lane-major, rows i then N-1-i), after the
//           rendezvous at named barrier xbar
__device__ __forceinline__ bool update_pair(bool on, int i, uint32_t tm0, uint32_t tsplit, const BoxRow& tb,
                                            uint32_t cb, uint32_t s_cf, uint32_t s_km, float h, uint32_t xb,
                                            int xbar) {
  constexpr int RP = round_up_c(N, 4);
  const int i2 = N - 1 - i;
  const uint32_t qa = 2u * N * i, qb = 2u * N * i2;  // code row offsets of the two rows
  // every load of both rows first (one TMEM wait for the pair), then the arithmetic
  RowIn<N, SB> ra, rb;
  load_row<N, SB>(tm0 + (uint32_t)(N * i), tsplit, tb, i + 1, ra);
  load_row<N, SB>(tm0 + (uint32_t)(N * i2), tsplit, tb, i2 + 1, rb);
  uint32_t la[N / 2], lb[N / 2];
#pragma unroll
  for (int m = 0; m < N / 2; ++m) {
    la[m] = lds32(cb + qa + 4u * m);
    lb[m] = lds32(cb + qb + 4u * m);
  }
  const uint32_t kma = lds32(s_km + 4u * i), kmb = lds32(s_km + 4u * i2);
  if (xb) named_bar(xbar, 64);                       // the partner wrote this pair's second parts
  tmem_wait_ld();
  if (xb) {
#pragma unroll
    for (int c = 0; c < N / 2; ++c) {
      float v[4];
      lds128f(xb + 16u * c, v[0], v[1], v[2], v[3]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int t = 4 * c + e;
        if (t < N) ra.acc[t] += v[e];
        else if (t < 2 * N) rb.acc[t - N] += v[e];
      }
    }
  }
  uint32_t a[N], b[N], ca[N / 2], cc[N / 2];
  finish_row<N, SB, KIND, VIS>(ra, tsplit != 0, s_cf + 4u * RP * i, kma, h, a, ca);
  finish_row<N, SB, KIND, VIS>(rb, tsplit != 0, s_cf + 4u * RP * i2, kmb, h, b, cc);
  // codes of both rows against the last transmitted ones; the code row then
  // holds the current codes (which select/pack sends)
  uint32_t diff = 0;
#pragma unroll
  for (int m = 0; m < N / 2; ++m) diff |= (la[m] ^ ca[m]) | (lb[m] ^ cc[m]);
#pragma unroll
  for (int m = 0; m < N / 2; ++m) {
    sts32_if(on, cb + qa + 4u * m, ca[m]);
    sts32_if(on, cb + qb + 4u * m, cc[m]);
  }
  store_row<N, SB>(on, tb, i + 1, b[0], a, b[N - 1]);
  store_row<N, SB>(on, tb, i2 + 1, a[0], b, a[N - 1]);
  if (i == 0) {                                      // i2 = N - 1: the top and bottom guard rows
    uint32_t ra[N], rb[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
      ra[c] = a[N - 1 - c];
      rb[c] = b[N - 1 - c];
    }
    store_row<N, SB>(on, tb, 0, b[N - 1], ra, b[0]);
    store_row<N, SB>(on, tb, N + 1, a[N - 1], rb, a[0]);
  }
  return diff != 0;
}

// This thread's share of one texture's epilogue: the interior-row pairs p of
// its slot (p % 2 == slot). Returns whether any code of the row changed.
template <int N, int SB, int KIND, bool VIS>
__device__ __forceinline__ bool epi_rows(bool on, int slot, uint32_t tm0, uint32_t tsplit, const BoxRow& tb,
                                         uint32_t cb, uint32_t s_cf, uint32_t s_km, float h, uint32_t xbuf,
                                         int xbar, int lane) {
  bool ch = false;
  int k = 0;
#pragma unroll 1
  for (int p = slot; p < N / 2; p += 2, ++k) {
    const uint32_t xb = xbuf ? xbuf + (uint32_t)(k & 1) * XBUF_BYTES + (uint32_t)lane * XROW_BYTES : 0u;
    ch |= update_pair<N, SB, KIND, VIS>(on, p, tm0, tsplit, tb, cb, s_cf, s_km, h, xb, xbar);
  }
  return ch;
}

// The partner side of the exchange: this warp's lanes hold the second parts
// of the partner warp's rows (the same probes, lo halves of the operands);
// per row pair it moves them from TMEM into the exchange buffer (double
// buffered by pair parity) and meets the partner at named barrier xbar.
template <int N>
__device__ __forceinline__ void provide_rows(int slot, uint32_t tm0, uint32_t xbuf, int xbar, int lane) {
  int k = 0;
#pragma unroll 1
  for (int p = slot; p < N / 2; p += 2, ++k) {
    const int i = p, i2 = N - 1 - p;
    float v[2 * N + 2];
#pragma unroll
    for (int m = 0; m < N / 2; ++m) {
      tmem_ld2(tm0 + (uint32_t)(N * i) + 2u * m, v[2 * m], v[2 * m + 1]);
      tmem_ld2(tm0 + (uint32_t)(N * i2) + 2u * m, v[N + 2 * m], v[N + 2 * m + 1]);
    }
    tmem_wait_ld();
    const uint32_t xb = xbuf + (uint32_t)(k & 1) * XBUF_BYTES + (uint32_t)lane * XROW_BYTES;
#pragma unroll
    for (int c = 0; c < N / 2; ++c)
      asm volatile("st.shared.v4.f32 [%0], {%1,%2,%3,%4};" ::"r"(xb + 16u * c), "f"(v[4 * c]), "f"(v[4 * c + 1]),
                   "f"(v[4 * c + 2]), "f"(v[4 * c + 3])
                   : "memory");
    named_bar(xbar, 64);
  }
}

// ------------------------------------------------------------------ kernel
template <int FORM, int SB, int NC, int NV, int MAXV>
__global__ void __launch_bounds__(NT, 1) k_blend_tc(const __grid_constant__ BlendArgs<MAXV> a) {
  using S = Shape<NC, NV>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  pv_grid_launch_dependents();
  const TcParams& tp = a.tp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool kSplitW = FORM != kF16;
  constexpr bool kTmemA = FORM == kF32;
  static_assert(2 * NV * 4 <= (int)XROW_BYTES, "exchange rows hold two visibility interior rows");
  constexpr uint32_t TBV = (uint32_t)((NV + 2) * (NV + 2) * SB), TBC = (uint32_t)((NC + 2) * (NC + 2) * SB);
  constexpr uint32_t WLO_V = (uint32_t)S::NVP * ROWB;              // visibility lo plane offset in a weight stage

  uint64_t* xfull = (uint64_t*)(smem + tp.off_bar);  // [xs] ray tiles landed (for the converters)
  uint64_t* xempty = xfull + tp.xs;                  // [xs] F32: ray stage converted, free
  uint64_t* ready = xempty + tp.xs;                  // [kRing] chunk's operands in place
  uint64_t* done = ready + kRing;                    // [kRing] chunk's MMAs completed
  uint64_t* tfull = done + kRing;                    // [2] visibility, colour accumulators ready
  uint64_t* tempty = tfull + 2;                      // [2] accumulators drained
  uint64_t* efull = tempty + 2;                      // [2] an item's old texels and codes arrived
  uint32_t* tmem_holder = (uint32_t*)(efull + 2);

  if (threadIdx.x == 0) {
    for (int i = 0; i < tp.xs; ++i) {
      mbar_init(&xfull[i], 1);
      mbar_init(&xempty[i], 4);                      // the four converter warps (F32)
    }
    // ready: the weight producer's expect-tx arrival plus four more, from the
    // converters (F32 chunks, 16-bit visibility chunks) or from the ray
    // producer (16-bit colour chunks, whose tiles land on this barrier)
    for (int i = 0; i < kRing; ++i) {
      mbar_init(&ready[i], 5);
      mbar_init(&done[i], 1);                        // the MMA thread's commit
    }
    for (int b = 0; b < 2; ++b) mbar_init(&tfull[b], 1);
    mbar_init(&tempty[0], kTmemA ? 8 : 6);           // visibility epilogue warps and their partners
    mbar_init(&tempty[1], 6);                        // colour epilogue warps (quarters 1, 2, 3)
    mbar_init(&efull[0], 2);                         // one loading thread per visibility channel
    mbar_init(&efull[1], 3);                         // and per colour channel
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // every tensor map of the launch toward the TMA unit, while warp 1
    // allocates tensor memory
    for (int v = 0; v < a.nvol; ++v) {
      const CUtensorMap* m[8] = {&a.v[v].dist, &a.v[v].rad, &a.v[v].st_v, &a.v[v].st_c,
                                 &a.v[v].last_v, &a.v[v].last_c, &a.v[v].cur_v, &a.v[v].cur_c};
      for (int i = 0; i < 8; ++i) asm volatile("prefetch.tensormap [%0];" ::"l"(m[i]) : "memory");
    }
    // The first item's first ray tiles (all stages are free) go out now, while
    // warp 1 allocates tensor memory; the ray producer continues after them.
    if (tp.items > (int)blockIdx.x) {
      const BlendVol& bv = a.v[vol_of(a, blockIdx.x)];
      const int p0 = ((int)blockIdx.x - bv.item0) * tp.np;
      const int pre = min(tp.xs, bv.nchunks);
      for (int kc = 0; kc < pre; ++kc) {
        mbar_expect_tx(&xfull[kc], tp.tx_xv);
        tma_load_2d(smem + tp.off_xr + (size_t)kc * tp.xstage, &bv.dist, kc * tp.kc, p0, &xfull[kc]);
      }
    }
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
  int* err = tp.k.err;
  const int np = tp.np;
  const int rounds = tp.items > (int)blockIdx.x ? (tp.items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  uint8_t* xring = smem + tp.off_xr;
  uint8_t* wring = smem + tp.off_wr;

  if (warp == 0) {
    // ------------------------------------------------------------ ray producer
    // The rays are this frame's inputs, complete before the weights kernel
    // started, so their tiles stream in from the kernel's start, as far
    // ahead of the MMAs as the ray ring allows (no wait for the previous
    // kernel). Visibility chunk: d rows into lane quarter 0; colour chunk:
    // R, G, B rows into quarters 1..3.
    // A stage is free once the converters hold its rays (F32: in TMEM) or
    // once the MMAs that read it completed (16-bit). Tiles land on xfull for
    // the converters, except 16-bit colour tiles, which the MMAs read as they
    // are: those land on the chunk's ready barrier, and this thread adds the
    // four arrivals the converters would have made.
    // the prologue issued the first item's first `pre` visibility tiles
    const int pre = rounds > 0 ? min(tp.xs, a.v[vol_of(a, blockIdx.x)].nchunks) : 0;
    int x = pre == tp.xs ? 0 : pre, n = pre;
    uint32_t ph = pre == tp.xs ? 1u : 0u;
    bool ok = true;
    for (int it = 0; it < rounds && ok; ++it) {
      const int item = blockIdx.x + it * gridDim.x;
      const BlendVol& bv = a.v[vol_of(a, item)];
      const int p0 = (item - bv.item0) * np;
      for (int phase = 0; phase < 2 && ok; ++phase) {
        for (int kc = (it == 0 && phase == 0) ? pre : 0; kc < bv.nchunks; ++kc, ++n) {
          if (kTmemA) ok = mbar_wait_warp(&xempty[x], ph ^ 1, err);
          else ok = wait_done_warp(done, n - tp.xs, err);
          if (!ok) break;
          uint8_t* st = xring + (size_t)x * tp.xstage;
          const int xr = kc * tp.kc;
          if (elect_one()) {
            if (phase == 0) {
              mbar_expect_tx(&xfull[x], tp.tx_xv);
              tma_load_2d(st, &bv.dist, xr, p0, &xfull[x]);
            } else {
              uint64_t* b = kTmemA ? &xfull[x] : &ready[n & (kRing - 1)];
              mbar_expect_tx(b, tp.tx_xc);
              if (!kTmemA)
                for (int i = 0; i < 3; ++i) mbar_arrive(b);
              for (int c = 0; c < 3; ++c)
                tma_load_2d(st + (c + 1) * QROWS * ROWB, &bv.rad, xr, c * bv.k.P + p0, b);
            }
          }
          __syncwarp();
          if (++x == tp.xs) {
            x = 0;
            ph ^= 1;
          }
        }
      }
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------ weight producer
    // The weight tile images (written by the weights kernel): visibility
    // chunk hi rows then lo rows; colour chunk hi then lo rows adjacent, so
    // that one MMA of N = 2 NCP takes both parts.
    // Everything the loop reads of the launch parameters for the first item
    // is fetched before the grid wait: those first reads miss the constant
    // cache, and after the wait they would delay the first weight tile (and so
    // the first MMA) by their latency. The empty asm keeps each value in a
    // register from before the wait.
    const uint32_t wvb = (uint32_t)S::NVP * ROWB, wcb = (uint32_t)S::NCP * ROWB;
    const int ws_n = tp.ws;
    const uint32_t wstage = (uint32_t)tp.wstage, tx_wv = tp.tx_wv, tx_wc = tp.tx_wc;
    auto vol_params = [&](int item, const uint8_t*& w_op, size_t& chunk_b, size_t& plane_b, int& nch) {
      const BlendVol& bv = a.v[vol_of(a, item)];
      w_op = (const uint8_t*)bv.k.w_op;
      chunk_b = (size_t)bv.k.w_rows * ROWB;
      plane_b = (size_t)bv.k.w_chunks * chunk_b;
      nch = bv.nchunks;
    };
    const uint8_t* w_op0 = nullptr;
    size_t chunk_b0 = 0, plane_b0 = 0;
    int nch0 = 0;
    if (rounds > 0) vol_params(blockIdx.x, w_op0, chunk_b0, plane_b0, nch0);
    asm volatile("" : "+l"(w_op0), "+l"(chunk_b0), "+l"(plane_b0), "+r"(nch0));
    asm volatile("" ::"r"(ws_n), "r"(wstage), "r"(tx_wv), "r"(tx_wc));
    pv_grid_wait();
    // Tiles land on the chunk's ready barrier; a stage is refilled once the
    // MMAs of the chunk that last read it completed.
    int w = 0, n = 0;
    bool ok = true;
    for (int it = 0; it < rounds && ok; ++it) {
      const uint8_t* w_op = w_op0;
      size_t chunk_b = chunk_b0, plane_b = plane_b0;
      int nchunks = nch0;
      if (it > 0) vol_params(blockIdx.x + it * gridDim.x, w_op, chunk_b, plane_b, nchunks);
      for (int phase = 0; phase < 2 && ok; ++phase) {
        for (int kc = 0; kc < nchunks; ++kc, ++n) {
          ok = wait_done_warp(done, n - ws_n, err);
          if (!ok) break;
          const uint32_t st = smem_u32(wring) + (uint32_t)w * wstage;
          const uint8_t* src = w_op + (size_t)kc * chunk_b + (phase == 0 ? 0 : wvb);
          const uint32_t wb = phase == 0 ? wvb : wcb;
          if (elect_one()) {
            uint64_t* b = &ready[n & (kRing - 1)];
            mbar_expect_tx(b, phase == 0 ? tx_wv : tx_wc);
            bulk_g2s(st, src, wb, b);
            if (kSplitW) bulk_g2s(st + wb, src + plane_b, wb, b);
          }
          __syncwarp();
          if (++w == ws_n) w = 0;
        }
      }
    }
  } else if (warp == 3) {
    // ------------------------------------------------------------ MMA issuer
    // (on the fourth SMSP, which the visibility epilogue does not use). The
    // whole warp runs the loop; one elected lane issues the MMAs and their
    // commits (a commit tracks the MMAs of its own thread: the same lane).
    // One wait per chunk (its ready barrier) and one commit (its done
    // barrier, which frees its ray, TMEM and weight stages together).
    // Descriptors advance by stage offsets: a shared-memory descriptor holds
    // address / 16 in its low bits, and every address stays below 2^18.
    int x = 0, w = 0, sa = 0, n = 0;
    uint32_t tph[2] = {0u, 0u};
    const uint64_t wdesc0 = sdesc(smem_u32(wring)), xdesc0 = sdesc(smem_u32(xring));
    const uint32_t wst16 = (uint32_t)tp.wstage >> 4, xst16 = (uint32_t)tp.xstage >> 4;
    const uint32_t abase = tmem + (uint32_t)tp.abase;
    bool ok = true;
    for (int it = 0; it < rounds && ok; ++it) {
      const int item = blockIdx.x + it * gridDim.x;
      const int nchunks = a.v[vol_of(a, item)].nchunks;
      for (int phase = 0; phase < 2 && ok; ++phase) {
        ok = mbar_wait_warp(&tempty[phase], tph[phase] ^ 1, err);
        if (!ok) break;
        tc_fence_after();
        const uint32_t d = tmem + (phase == 0 ? 0u : (uint32_t)S::CBASE);
        const uint32_t idesc = phase == 0 ? tp.idesc_v : tp.idesc_c;
        for (int kc = 0; kc < nchunks; ++kc, ++n) {
          ok = mbar_wait_warp(&ready[n & (kRing - 1)], (uint32_t)((n / kRing) & 1), err);
          if (!ok) break;
          tc_fence_after();
          const uint64_t bw0 = wdesc0 + (uint64_t)(w * wst16);
          const uint64_t ax0 = xdesc0 + (uint64_t)(x * xst16);
          if (elect_one()) {
#pragma unroll
            for (int ks = 0; ks < ROWB / 32; ++ks) {          // one MMA K step per 32 bytes of row
              const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
              const uint64_t bw = bw0 + 2u * ks;                // + 32 bytes
              if constexpr (kTmemA) {
                const uint32_t ah = abase + 32u * sa + 8u * ks;
                if (phase == 0) {                                            // lanes hold hi and lo parts
                  mma_ts_tf32(d, ah, bw, idesc, acc);                        // [d, d^2] (hi | lo) * W hi
                  mma_ts_tf32(d, ah, bw + (WLO_V >> 4), idesc, 1u);          // ... * W lo
                } else {
                  mma_ts_tf32(d, ah, bw, tp.idesc_c2, acc);                  // x hi * [W hi | W lo]
                  mma_ts_tf32(d, ah + 16u, bw, idesc, 1u);                   // x lo * W hi
                }
              } else {
                const uint64_t ax = ax0 + 2u * ks;
                if (kSplitW && phase == 1) {
                  mma_ss<FORM>(d, ax, bw, tp.idesc_c2, acc);                 // x * [W hi | W lo]
                } else {
                  mma_ss<FORM>(d, ax, bw, idesc, acc);                       // visibility: d, d^2 hi, d^2 lo
                  if (kSplitW) mma_ss<FORM>(d, ax, bw + (WLO_V >> 4), idesc, 1u);
                }
              }
            }
            mma_commit(&done[n & (kRing - 1)]);                 // the chunk's stages free once these finish
          }
          __syncwarp();
          if (++x == tp.xs) x = 0;
          if (++w == tp.ws) w = 0;
          if (kTmemA && ++sa == tp.as_) sa = 0;
        }
        if (!ok) break;
        if (elect_one()) mma_commit(&tfull[phase]);              // accumulators ready for the epilogue
        __syncwarp();
        tph[phase] ^= 1;
      }
    }
  } else if (warp >= 4 && warp < 8) {
    // ------------------------------------------------------------ converters
    // Each converter warp arrives once on the chunk's ready barrier when its
    // part is written (16-bit colour chunks need no conversion: the ray
    // producer arrives for them).
    const int q = warp & 3;
    int x = 0, sa = 0, n = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int it = 0; it < rounds && ok; ++it) {
      const int item = blockIdx.x + it * gridDim.x;
      const int nchunks = a.v[vol_of(a, item)].nchunks;
      for (int phase = 0; phase < 2 && ok; ++phase) {
        if (!kTmemA && phase == 1) {
          n += nchunks;
          x += nchunks;
          while (x >= tp.xs) {
            x -= tp.xs;
            ph ^= 1;
          }
          continue;
        }
        for (int kc = 0; kc < nchunks; ++kc, ++n) {
          ok = mbar_wait_warp(&xfull[x], ph, err);
          if (!ok) break;
          const uint32_t sx = smem_u32(xring + (size_t)x * tp.xstage);
          if constexpr (kTmemA) {
            // my lane quarter's rows, split into TF32 hi + lo parts in TMEM.
            // Visibility: q0 = d hi, q1 = d^2 hi, q2 = d lo, q3 = d^2 lo (all
            // from the d rows), in the stage's first 16 columns, so that each
            // MMA takes both parts and the epilogue adds quarter 2 to 0 and 3
            // to 1. Colour: q1..q3 = R, G, B, hi in the first 16 columns and
            // lo in the next 16.
            ok = wait_done_warp(done, n - tp.as_, err);      // the MMAs that read this TMEM stage
            if (!ok) break;
            tc_fence_after();
            if (phase == 0 || q >= 1) {
              const int row = phase == 0 ? lane : 32 * q + lane;
              const bool sq = phase == 0 && (q & 1);
              uint32_t hi[16], lo[16];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                uint32_t x0, x1, x2, x3;
                lds128(sx + swz64(row, u), x0, x1, x2, x3);
                const uint32_t xs[4] = {x0, x1, x2, x3};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  float v = __uint_as_float(xs[e]);
                  if (sq) v = v * v;
                  const uint32_t vb = __float_as_uint(v);
                  const uint32_t h = vb & 0xFFFFE000u;
                  hi[4 * u + e] = h;
                  lo[4 * u + e] = __float_as_uint(v - __uint_as_float(h));
                }
              }
              const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)tp.abase + 32u * sa;
              if (phase == 0) {
                tmem_st16(ta, q < 2 ? hi : lo);
              } else {
                tmem_st16(ta, hi);
                tmem_st16(ta + 16u, lo);
              }
              tmem_wait_st();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              mbar_arrive(&xempty[x]);
              mbar_arrive(&ready[n & (kRing - 1)]);
            }
            if (++sa == tp.as_) sa = 0;
          } else {
            // d^2 = hi + lo in the operand format (binary16 scaled by 2^-4):
            // the hi part into lane quarter 1 of the A tile, the lo part into
            // lane quarter 2 (the epilogue adds quarter 2's accumulators to
            // quarter 1's); converter warp q takes 16-byte unit q of every d
            // row (8 rays), so the four share each chunk
            if (phase == 0) {
              const int u = q;
              uint32_t r[4];
              lds128(sx + swz64(lane, u), r[0], r[1], r[2], r[3]);
              uint32_t oh[4], ol[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                if constexpr (FORM == kF16) {
                  const __half2 h2 = *reinterpret_cast<const __half2*>(&r[e]);
                  const float d0 = __low2float(h2), d1 = __high2float(h2);
                  const float q0 = d0 * d0 * kD2ScaleF16, q1 = d1 * d1 * kD2ScaleF16;
                  const __half h0 = __float2half_rn(q0), h1 = __float2half_rn(q1);
                  const __half l0 = __float2half_rn(q0 - __half2float(h0));
                  const __half l1 = __float2half_rn(q1 - __half2float(h1));
                  oh[e] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
                  ol[e] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
                } else {
                  const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&r[e]);
                  const float d0 = __low2float(h2), d1 = __high2float(h2);
                  const float q0 = d0 * d0, q1 = d1 * d1;
                  const __nv_bfloat16 h0 = __float2bfloat16_rn(q0), h1 = __float2bfloat16_rn(q1);
                  const __nv_bfloat16 l0 = __float2bfloat16_rn(q0 - __bfloat162float(h0));
                  const __nv_bfloat16 l1 = __float2bfloat16_rn(q1 - __bfloat162float(h1));
                  oh[e] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                  ol[e] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                }
              }
              asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(sx + swz64(QROWS + lane, u)), "r"(oh[0]),
                           "r"(oh[1]), "r"(oh[2]), "r"(oh[3])
                           : "memory");
              asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(sx + swz64(2 * QROWS + lane, u)), "r"(ol[0]),
                           "r"(ol[1]), "r"(ol[2]), "r"(ol[3])
                           : "memory");
              fence_proxy_async();
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ready[n & (kRing - 1)]);
          }
          if (++x == tp.xs) {
            x = 0;
            ph ^= 1;
          }
        }
      }
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                         // TMEM lane quarter
    const int slot = (warp >> 2) - 2;               // 0 or 1 within the quarter
    const int e = threadIdx.x - 256;                // 0..255
    const bool do_v = q <= 1, do_c = q >= 1;
    const int chv = q, chc = q - 1;                 // channel of this quarter per texture
    const int kind = tp.k.color_code;
    float* cf_v = (float*)(smem + tp.off_cf);                   // [2][NV][RPV]
    float* cf_c = cf_v + 2 * NV * S::RPV;                       // [NC][RPC]
    uint32_t* km_v = (uint32_t*)(smem + tp.off_km);             // [NV]
    uint32_t* km_c = km_v + NV;                                 // [NC]
    const uint32_t boxb = (uint32_t)tp.boxb;
    // boxes per probe row: tiles (128 bytes of texels each), codes (64 codes each)
    constexpr int BTV = (int)(TBV / 128), BTC = (int)(TBC / 128);
    const uint32_t lsv = (uint32_t)tp.k.lv_stride * 2, lsc = (uint32_t)tp.k.lc_stride * 2;   // code row bytes
    // this quarter's channel regions
    const uint32_t s_tv = smem_u32(smem + tp.off_tv) + (uint32_t)(chv * BTV) * boxb;
    const uint32_t s_lv = smem_u32(smem + tp.off_lv) + (uint32_t)(chv * tp.lreg_v);
    const uint32_t s_tc = smem_u32(smem + tp.off_tc) + (uint32_t)(chc * BTC) * boxb;
    const uint32_t s_lc = smem_u32(smem + tp.off_lc) + (uint32_t)(chc * tp.lreg_c);
    const bool io = slot == 0 && lane == 0;         // this channel's loading / storing thread
    // visibility exchange: F32 lanes of quarters 2 / 3 hold the lo parts of
    // quarters 0 / 1 (d, d^2); 16-bit lanes of quarter 2 hold d^2's lo part
    // (quarter 1). A target warp meets its provider (same slot) at its own
    // named barrier and reads the provider's values from a double buffer.
    const bool x_target = kTmemA ? q <= 1 : q == 1;
    const bool x_provider = kTmemA ? q >= 2 : q == 2;
    const int x_t = kTmemA ? (q & 1) : 0;           // partnership index of this quarter's target
    const int xbar = 6 + 2 * x_t + slot;
    const uint32_t xbuf = smem_u32(smem + tp.off_xb) + (uint32_t)((2 * x_t + slot) * 2) * XBUF_BYTES;
    // the item's old texels and last-transmitted codes of this quarter's channel
    auto issue_prefetch = [&](int item, bool vis) {
      const BlendVol& bv = a.v[vol_of(a, item)];
      const int p0 = (item - bv.item0) * np;
      if (vis) {
        mbar_expect_tx(&efull[0], (uint32_t)(BTV * np * 128) + (uint32_t)np * lsv);
        for (int b = 0; b < BTV; ++b) tma_load_3d(s_tv + (uint32_t)b * boxb, &bv.st_v, b * (128 / SB), p0, chv, &efull[0]);
        tma_load_3d(s_lv, &bv.last_v, 0, p0, chv, &efull[0]);
      } else {
        mbar_expect_tx(&efull[1], (uint32_t)(BTC * np * 128) + (uint32_t)np * lsc);
        for (int b = 0; b < BTC; ++b) tma_load_3d(s_tc + (uint32_t)b * boxb, &bv.st_c, b * (128 / SB), p0, chc, &efull[1]);
        tma_load_3d(s_lc, &bv.last_c, 0, p0, chc, &efull[1]);
      }
    };
    pv_grid_wait();
    if (rounds > 0 && io) {
      if (do_v) issue_prefetch(blockIdx.x, true);
      if (do_c) issue_prefetch(blockIdx.x, false);
    }
    int cur = -1;
    float h = 0.0f;
    uint32_t eph = 0;
    bool ok = true;
    for (int it = 0; it < rounds; ++it) {
      const int item = blockIdx.x + it * gridDim.x;
      const int vi = vol_of(a, item);
      const BlendVol& bv = a.v[vi];
      const pv_dev& kv = bv.k;
      const int p0 = (item - bv.item0) * np, npi = min(np, kv.P - p0);
      const bool on = lane < npi;
      const int jr = on ? lane : 0;                 // box row read by lanes without a probe
      named_bar(1, EPI_THREADS);                    // the previous item's epilogue is done everywhere
      if (vi != cur) {                              // this volume's factors: (1 - h) * scale / S per texel
        h = *(volatile float*)kv.hy;
        const float omh = 1.0f - h;
        for (int t = e; t < NV * NV + NC * NC; t += EPI_THREADS) {
          const bool vis = t < NV * NV;
          const int tt = vis ? t : t - NV * NV;
          const int n = vis ? NV : NC;
          const float Sm = kv.sums[vis ? NC * NC + tt : tt];
          const float rS = Sm > 0.0f ? 1.0f / Sm : 0.0f;
          if (vis) {
            cf_v[(tt / n) * S::RPV + tt % n] = omh * rS;
            cf_v[NV * S::RPV + (tt / n) * S::RPV + tt % n] = omh * (rS * (FORM == kF16 ? 1.0f / kD2ScaleF16 : 1.0f));
          } else {
            cf_c[(tt / n) * S::RPC + tt % n] = omh * rS;
          }
        }
        named_bar(1, EPI_THREADS);
        // texels without any weight (factor 0), per interior row, from the table
        for (int r = e; r < NV + NC; r += EPI_THREADS) {
          const bool vis = r < NV;
          const int n = vis ? NV : NC, i = vis ? r : r - NV;
          const float* row = vis ? cf_v + i * S::RPV : cf_c + i * S::RPC;
          uint32_t m = 0;
          for (int j = 0; j < n; ++j)
            if (!(row[j] > 0.0f)) m |= 1u << j;
          (vis ? km_v : km_c)[i] = m;
        }
        cur = vi;
        named_bar(1, EPI_THREADS);
      }
      const int next = item + gridDim.x;
      // ---- visibility
      if (x_provider) {                             // the lo parts of a partner quarter's rows
        if (ok) ok = mbar_wait(&tfull[0], eph, err);
        tc_fence_after();
        ok = named_bar_and(xbar, 64, ok);
        if (ok) provide_rows<NV>(slot, tmem + ((uint32_t)(32 * q) << 16), xbuf, xbar, lane);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[0]);
      }
      if (do_v) {
        if (ok) ok = mbar_wait(&efull[0], eph, err);
        if (ok) ok = mbar_wait(&tfull[0], eph, err);
        tc_fence_after();
        if (x_target) ok = named_bar_and(xbar, 64, ok);
        bool chg = false;
        if (ok) {
          const uint32_t tm0 = tmem + ((uint32_t)(32 * q) << 16);
          chg = epi_rows<NV, SB, 0, true>(on, slot, tm0, 0u, box_row(s_tv, boxb, jr), s_lv + (uint32_t)jr * lsv,
                                          smem_u32(cf_v + chv * NV * S::RPV), smem_u32(km_v), h,
                                          x_target ? xbuf : 0u, xbar, lane);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[0]);
        const uint32_t m = __ballot_sync(0xffffffffu, chg && on);
        if (lane == 0 && m && ok) {
          uint32_t* w = &kv.chg[kv.chg_words + (p0 >> 5)];
          const int sh = p0 & 31;
          atomicOr(w, m << sh);
          if (sh && (m >> (32 - sh))) atomicOr(w + 1, m >> (32 - sh));
        }
        fence_proxy_async();
        named_bar(2 + q, 64);                       // both warps of the quarter wrote their rows
        if (io) {
          if (ok) {
            for (int b = 0; b < BTV; ++b) tma_store_3d(&bv.st_v, b * (128 / SB), p0, chv, s_tv + (uint32_t)b * boxb);
            if (kv.cur_v) tma_store_3d(&bv.cur_v, 0, p0, chv, s_lv);
            bulk_commit();
          }
          if (next < tp.items && ok) {              // the boxes are refilled once the stores read them
            bulk_wait_read();
            issue_prefetch(next, true);
          }
        }
      }
      // ---- colour
      if (do_c) {
        if (ok) ok = mbar_wait(&efull[1], eph, err);
        if (ok) ok = mbar_wait(&tfull[1], eph, err);
        tc_fence_after();
        bool chg = false;
        if (ok) {
          const uint32_t tm0 = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)S::CBASE;
          const BoxRow tb = box_row(s_tc, boxb, jr);
          const uint32_t cb = s_lc + (uint32_t)jr * lsc;
          const uint32_t tsplit = kSplitW ? (uint32_t)S::NCP : 0u;   // colour: hi and lo weight columns
          if (kind == PV_CODE_UNORM10)
            chg = epi_rows<NC, SB, PV_CODE_UNORM10, false>(on, slot, tm0, tsplit, tb, cb, smem_u32(cf_c),
                                                           smem_u32(km_c), h, 0u, 0, lane);
          else
            chg = epi_rows<NC, SB, PV_CODE_UF10, false>(on, slot, tm0, tsplit, tb, cb, smem_u32(cf_c), smem_u32(km_c),
                                                        h, 0u, 0, lane);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[1]);
        const uint32_t m = __ballot_sync(0xffffffffu, chg && on);
        if (lane == 0 && m && ok) {
          uint32_t* w = &kv.chg[p0 >> 5];
          const int sh = p0 & 31;
          atomicOr(w, m << sh);
          if (sh && (m >> (32 - sh))) atomicOr(w + 1, m >> (32 - sh));
        }
        fence_proxy_async();
        named_bar(2 + q, 64);
        if (io) {
          if (ok) {
            for (int b = 0; b < BTC; ++b) tma_store_3d(&bv.st_c, b * (128 / SB), p0, chc, s_tc + (uint32_t)b * boxb);
            if (kv.cur_c) tma_store_3d(&bv.cur_c, 0, p0, chc, s_lc);
            bulk_commit();
          }
          if (next < tp.items && ok) {
            bulk_wait_read();
            issue_prefetch(next, false);
          }
        }
      }
      eph ^= 1;
    }
    bulk_wait_all();
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

// Rays of rows [rows] x [inner] elements, boxes of box_inner (64 bytes) x
// box_rows, SWIZZLE_64B; rays past `inner` and rows past `rows` read zero.
cudaError_t encode_2d(CUtensorMap* m, int fmt, const void* base, uint64_t inner, uint64_t rows, uint64_t row_bytes,
                      uint32_t box_inner, uint32_t box_rows) {
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(m, dtype_of(fmt), 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
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

// The compiled interior sizes (colour, visibility).
constexpr int kNC = 6, kNV = 14;
using Shp = Shape<kNC, kNV>;

template <int MAXV>
const void* kernel_of(int form, int sb) {
  if (form == kF16)
    return sb == 2 ? (const void*)k_blend_tc<kF16, 2, kNC, kNV, MAXV> : (const void*)k_blend_tc<kF16, 4, kNC, kNV, MAXV>;
  if (form == kBF16)
    return sb == 2 ? (const void*)k_blend_tc<kBF16, 2, kNC, kNV, MAXV> : (const void*)k_blend_tc<kBF16, 4, kNC, kNV, MAXV>;
  return sb == 2 ? (const void*)k_blend_tc<kF32, 2, kNC, kNV, MAXV> : (const void*)k_blend_tc<kF32, 4, kNC, kNV, MAXV>;
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

// Shared-memory layout for volumes shaped like k, with work items of at most
// np_want probes (fewer when shared memory demands). Fills every field of tp
// except items.
// lim: optional upper bounds of the ray, weight and TMEM A ring depths (0: none).
cudaError_t make_layout(const pv_dev& k, int form, int np_want, int smem_max, TcParams& tp, size_t* smem,
                        const pv_tc_opts* lim = nullptr) {
  const int sb = k.state_fmt == PV_FMT_F16 ? 2 : 4;
  if (k.nc != kNC || k.nv != kNV) return cudaErrorInvalidValue;
  if (k.w_rb != ROWB || k.w_vb != Shp::NVP || k.w_rows != Shp::NVP + Shp::NCP) return cudaErrorInvalidValue;
  tp.k = k;
  tp.kc = k.w_kc;
  const int planes = form == kF16 ? 1 : 2;
  // ray stage: the 128-row A tile (TMA rows at the lane quarters); weight
  // stage: the visibility block (the larger one) in every plane
  tp.xstage = A_BYTES;
  tp.wstage = (int)align1k((size_t)planes * Shp::WROWS * ROWB);
  // epilogue: tile boxes (128-byte column strips of np rows, 1024-byte
  // aligned for SWIZZLE_128B) and dense code rows per channel
  const int btv = (kNV + 2) * (kNV + 2) * sb / 128, btc = (kNC + 2) * (kNC + 2) * sb / 128;
  const size_t xbytes = (size_t)(form == kF32 ? 4 : 2) * 2 * XBUF_BYTES;   // visibility exchange buffers
  const size_t tables = align1k((size_t)(2 * kNV * Shp::RPV + kNC * Shp::RPC) * 4) + align1k((size_t)(kNV + kNC) * 4) +
                        align1k(xbytes);
  const size_t bars = 1024;
  int np = np_want;
  size_t epi = 0, rings = 0;
  for (; np >= 1; --np) {
    tp.boxb = (int)align1k((size_t)np * 128);
    tp.lreg_v = (int)align1k((size_t)np * k.lv_stride * 2);
    tp.lreg_c = (int)align1k((size_t)np * k.lc_stride * 2);
    epi = (size_t)(2 * btv + 3 * btc) * tp.boxb + 2 * (size_t)tp.lreg_v + 3 * (size_t)tp.lreg_c;
    const size_t need = 1024 + epi + tables + bars;
    rings = need < (size_t)smem_max ? (size_t)smem_max - need : 0;
    if (rings >= (size_t)(3 * tp.xstage + 2 * tp.wstage)) break;
  }
  if (np < 1) return cudaErrorInvalidConfiguration;
  // The weight tiles come from L2 and need a shallow ring (3 stages of the
  // split forms' 26 KB, 4 of 13 KB); the ray tiles come from HBM, so the ray
  // ring takes the rest (up to 16 stages) to keep enough bytes in flight.
  int ws = tp.wstage > 16384 ? 3 : 4;
  if (lim && lim->weight_stages > 0) ws = lim->weight_stages;
  while (ws > 2 && (size_t)ws * tp.wstage + (size_t)3 * tp.xstage > rings) --ws;
  int xs = (int)((rings - (size_t)ws * tp.wstage) / tp.xstage);
  if (xs > 16) xs = 16;
  if (lim && lim->ray_stages > 0 && xs > lim->ray_stages) xs = lim->ray_stages;
  if (xs < 2) return cudaErrorInvalidConfiguration;
  tp.abase = round_up_c(Shp::CBASE + 2 * Shp::NCP, 32);
  tp.as_ = form == kF32 ? (512 - tp.abase) / 32 : 1;
  if (tp.as_ > 6) tp.as_ = 6;
  if (form == kF32 && lim && lim->tmem_stages > 0 && tp.as_ > lim->tmem_stages) tp.as_ = lim->tmem_stages;
  if (form == kF32 && tp.as_ < 2) return cudaErrorInvalidConfiguration;
  tp.np = np;
  tp.xs = xs;
  tp.ws = ws;
  tp.tx_xv = (uint32_t)(np * ROWB);
  tp.tx_xc = (uint32_t)(3 * np * ROWB);
  tp.tx_wv = (uint32_t)(planes * Shp::NVP * ROWB);
  tp.tx_wc = (uint32_t)(planes * Shp::NCP * ROWB);
  tp.idesc_v = make_idesc(form, 128, Shp::NVP);
  tp.idesc_c = make_idesc(form, 128, Shp::NCP);
  tp.idesc_c2 = make_idesc(form, 128, 2 * Shp::NCP);
  size_t off = 0;
  tp.off_xr = (int)off;
  off += (size_t)xs * tp.xstage;
  tp.off_wr = (int)off;
  off += (size_t)ws * tp.wstage;
  tp.off_tv = (int)off;
  off += (size_t)2 * btv * tp.boxb;
  tp.off_lv = (int)off;
  off += (size_t)2 * tp.lreg_v;
  tp.off_tc = (int)off;
  off += (size_t)3 * btc * tp.boxb;
  tp.off_lc = (int)off;
  off += (size_t)3 * tp.lreg_c;
  tp.off_cf = (int)off;
  off += align1k((size_t)(2 * kNV * Shp::RPV + kNC * Shp::RPC) * 4);
  tp.off_km = (int)off;
  off += align1k((size_t)(kNV + kNC) * 4);
  tp.off_xb = (int)off;
  off += align1k(xbytes);
  tp.off_bar = (int)off;
  off += bars;
  *smem = off + 1024;                          // slack for aligning the dynamic base
  return (*smem <= (size_t)smem_max) ? cudaSuccess : cudaErrorInvalidConfiguration;
}

// [channels][rows][inner] elements of esize bytes. Tiles (dense = false):
// boxes of 128 bytes x box_rows x 1 with SWIZZLE_128B; codes (dense = true):
// boxes of whole rows x box_rows x 1, unswizzled. Out-of-range rows read zero
// and are not written.
cudaError_t encode_3d(CUtensorMap* m, CUtensorMapDataType dt, int esize, const void* base, uint64_t inner,
                      uint64_t rows, uint64_t nch, uint32_t box_rows, bool dense) {
  cuuint64_t dims[3] = {inner, rows, nch};
  cuuint64_t strides[2] = {inner * esize, rows * inner * esize};
  cuuint32_t box[3] = {dense ? (cuuint32_t)inner : (cuuint32_t)(128 / esize), box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_encode(m, dt, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        dense ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor maps of a volume's state tiles and codes, for the epilogue.
cudaError_t encode_epi_maps(const pv_dev& k, int np, BlendVol& bv) {
  const int sb = k.state_fmt == PV_FMT_F16 ? 2 : 4;
  const CUtensorMapDataType st = sb == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
  const CUtensorMapDataType cd = CU_TENSOR_MAP_DATA_TYPE_UINT16;
  cudaError_t e = encode_3d(&bv.st_v, st, sb, k.state_v, k.sv_stride, k.P, 2, np, false);
  if (e == cudaSuccess) e = encode_3d(&bv.st_c, st, sb, k.state_c, k.sc_stride, k.P, 3, np, false);
  if (e == cudaSuccess) e = encode_3d(&bv.last_v, cd, 2, k.last_v, k.lv_stride, k.P, 2, np, true);
  if (e == cudaSuccess) e = encode_3d(&bv.last_c, cd, 2, k.last_c, k.lc_stride, k.P, 3, np, true);
  if (e == cudaSuccess && k.cur_v) e = encode_3d(&bv.cur_v, cd, 2, k.cur_v, k.lv_stride, k.P, 2, np, true);
  if (e == cudaSuccess && k.cur_c) e = encode_3d(&bv.cur_c, cd, 2, k.cur_c, k.lc_stride, k.P, 3, np, true);
  return e;
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
cudaError_t launch_blend(const BlendArgs<MAXV>& a, int form, int sb, int grid, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0] = pv_pdl_attr();
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void (*fn)(BlendArgs<MAXV>) = (void (*)(BlendArgs<MAXV>))kernel_of<MAXV>(form, sb);
  cudaError_t e = cudaLaunchKernelEx(&cfg, fn, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int MAXV>
cudaError_t set_smem_attr(int form, int sb, int bytes) {
  return cudaFuncSetAttribute(kernel_of<MAXV>(form, sb), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

struct TcPlan {
  BlendArgs<1> args;
  size_t smem;
  int grid;
  int form, sb;
};

}  // namespace

// Batch plan (opaque to the API layer).
struct pv_tc_batch {
  BlendArgs<kMaxBatch> args;
  size_t smem;
  int grid;
  int form, sb;
  int n;
  pv_volume* vols[kMaxBatch];
};

bool pv_tc_supported(const pv_desc* d, const char** why) {
  const int ob = d->operand_fmt == PV_FMT_F32 ? 4 : 2;
  if (d->color_interior != kNC || d->vis_interior != kNV) {
    if (why) *why = "the tensor-core blend is compiled for 6x6 colour and 14x14 visibility interiors";
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
  const int sb = v->state_bytes;
  e = set_smem_attr<1>(form, sb, di.smem_max);
  if (e != cudaSuccess) return e;
  // one item per SM where possible
  const int resident = di.sms;
  int np = (k.P + resident - 1) / resident;
  np = np < 1 ? 1 : (np > QROWS ? QROWS : np);
  TcPlan* pl = new TcPlan();
  memset(pl, 0, sizeof(TcPlan));
  TcParams& tp = pl->args.tp;
  e = make_layout(k, form, np, di.smem_max, tp, &pl->smem);
  if (e == cudaSuccess) {
    tp.items = (k.P + tp.np - 1) / tp.np;
    pl->grid = tp.items < resident ? tp.items : resident;
    pl->form = form;
    pl->sb = sb;
    pl->args.nvol = 1;
    BlendVol& bv = pl->args.v[0];
    bv.k = k;
    bv.item0 = 0;
    bv.nchunks = k.w_chunks;
    e = encode_epi_maps(k, tp.np, bv);
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
  return launch_blend(a, pl->form, pl->sb, pl->grid, pl->smem, st);
}

cudaError_t pv_tc_batch_create(pv_volume* const* vols, int n, int np_want, pv_tc_batch** out) {
  pv_tc_opts o = {};
  o.probes_per_item = np_want;
  return pv_tc_batch_create_opts(vols, n, &o, out);
}

cudaError_t pv_tc_batch_create_opts(pv_volume* const* vols, int n, const pv_tc_opts* opts, pv_tc_batch** out) {
  if (n < 1 || n > kMaxBatch || !opts) return cudaErrorInvalidValue;
  const int np_want = opts->probes_per_item;
  cudaError_t e = get_encoder();
  DevInfo di;
  if (e == cudaSuccess) e = dev_info(&di);
  if (e != cudaSuccess) return e;
  const pv_dev& k0 = vols[0]->k;
  const int form = form_of(k0.operand_fmt);
  const int sb = vols[0]->state_bytes;
  e = set_smem_attr<kMaxBatch>(form, sb, di.smem_max);
  if (e != cudaSuccess) return e;
  int total = 0;
  for (int i = 0; i < n; ++i) total += vols[i]->k.P;
  int np = np_want > 0 ? np_want : (total + di.sms - 1) / di.sms;
  np = np < 1 ? 1 : (np > QROWS ? QROWS : np);
  pv_tc_batch* b = new pv_tc_batch();
  memset(b, 0, sizeof(pv_tc_batch));
  TcParams& tp = b->args.tp;
  e = make_layout(k0, form, np, di.smem_max, tp, &b->smem, opts);
  if (e == cudaSuccess) {
    int items = 0;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
      const pv_dev& k = vols[i]->k;
      BlendVol& bv = b->args.v[i];
      bv.k = k;
      bv.item0 = items;
      bv.nchunks = k.w_chunks;
      e = encode_epi_maps(k, tp.np, bv);
      items += (k.P + tp.np - 1) / tp.np;
      b->vols[i] = vols[i];
    }
    tp.items = items;
    b->grid = items < di.sms ? items : di.sms;
    if (opts->ctas > 0 && opts->ctas < b->grid) b->grid = opts->ctas;
    b->args.nvol = n;
    b->form = form;
    b->sb = sb;
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

void pv_tc_batch_config(const pv_tc_batch* b, pv_tc_opts* o) {
  o->probes_per_item = b->args.tp.np;
  o->ray_stages = b->args.tp.xs;
  o->weight_stages = b->args.tp.ws;
  o->tmem_stages = b->form == kF32 ? b->args.tp.as_ : 0;
  o->ctas = b->grid;
}

cudaError_t pv_tc_batch_launch(pv_tc_batch* b, const void* const* rad, const void* const* dist, cudaStream_t st) {
  BlendArgs<kMaxBatch>* a = new BlendArgs<kMaxBatch>(b->args);
  cudaError_t e = cudaSuccess;
  a->tp.k = b->vols[0]->k;
  for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
    a->v[i].k = b->vols[i]->k;
    e = encode_ray_maps(b->vols[i]->k, b->form, a->tp, rad[i], dist[i], a->v[i]);
  }
  if (e == cudaSuccess) e = launch_blend(*a, b->form, b->sb, b->grid, b->smem, st);
  delete a;
  return e;
}
