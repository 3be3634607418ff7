// Change selection, probe index buffers and bit packing (Sections 3.3 and
// 3.4 of arXiv 2103.05875), fused into one kernel, plus the flag
// recomputation used after a state import.
//
// Selection: the blend raises bit p of the colour (visibility) mask when a
// transmitted code of probe p differs from its last-transmitted code, and
// keeps every probe's current codes; slots are assigned in ascending probe
// id. A block owns SP_RANGE consecutive probes. It first starts asynchronous
// copies of its probes' current codes into shared memory; meanwhile its first
// warp reads both masks (P/8 bytes each) and reduces them, so the block knows
// its probes' slots, the last selected probe before its range (for the delta
// code) and the totals without any grid-wide synchronisation. After one
// barrier it writes, for its selected probes:
//   the last-transmitted codes (16-byte vectors from the staged codes);
//   the index buffer entries and deltas (d0 = id0, dk = id_k - id_(k-1));
//   colour: the 10-bit codes of the interior to planes Y=R, U=G, V=B at
//           block (k / B_w, k % B_w) as 16-bit samples (code << 6 unless
//           color_lsb);
//   visibility: per atlas row each texel's bytes (R.lo, R.hi, G.lo, G.hi)
//           continue the row's byte stream; byte s goes to plane s mod 3,
//           column s div 3 (the paper's YUVY / UVYU / VYUV pattern).
// It also clears its share of the slots that held a probe last frame but are
// empty now (slots beyond both counts are already zero). The masks count once
// per update: the kernel compares the frame counter with the frame of the
// previous select, so a second select without a new update selects nothing.
// The last block to have read the select state advances the select sequence,
// which double-buffers the previous counts; the next select sees it, since a
// kernel waits for its predecessors to complete before reading.
#include "pv_codes.cuh"
#include "pv_internal.h"

namespace {

// 256 threads and 8 probes per block keep a 16^3 volume's 512 blocks resident
// in one wave (several blocks per SM)
constexpr int SP_THREADS = 256;
constexpr int SP_RANGE = 8;              // probes per block: their codes are staged in shared memory
constexpr int SP_MAX_T = PV_MAX_INTERIOR * PV_MAX_INTERIOR;

struct SpShared {
  // current codes of the block's probes (local index), channel rows lc_stride
  // (colour) and lv_stride (visibility R then G) apart
  uint16_t cc[SP_RANGE][3 * SP_MAX_T];
  uint16_t cv[SP_RANGE][2 * SP_MAX_T];
  int slot_c[SP_RANGE], slot_v[SP_RANGE];
  uint16_t prev_c[SP_RANGE], prev_v[SP_RANGE];
  int list_c[SP_RANGE], list_v[SP_RANGE];  // the block's selected probes (local index), slot order
  int n_c, n_v, first_c, first_v;          // how many, and the slot of the first
  int tot_c, tot_v, prev_cnt_c, prev_cnt_v;
  uint32_t seq;
  uint16_t xoff[SP_RANGE * PV_MAX_INTERIOR];   // per texel column of a visibility run: its staged row 0
};

using pv::fdiv;

// ceil(2^31 / d) for run lengths d = 1..SP_RANGE
__constant__ uint32_t c_rcp_run[SP_RANGE + 1] = {0u,          0x80000000u, 0x40000000u, 0x2AAAAAABu, 0x20000000u,
                                                 0x1999999Au, 0x15555556u, 0x12492493u, 0x10000000u};

// Colour samples of slots [a, b) (all in one block row) from the staged codes
// of the block's selected probe list_c[q0 + slot - a] (zero when `clear`).
// Thread tid = (g * cnt + so) * n + j owns column j of slot so and writes it
// down rows g, g + groups, ... of the 3 * n_c rows; consecutive threads write
// consecutive 16-bit samples.
__device__ __forceinline__ void write_color_run(const pv_dev& k, const SpShared& sh, int a, int b, int q0, bool clear) {
  const int n = k.nc, cnt = b - a;
  const int by = a / k.bw, bx0 = a - by * k.bw;
  const int t2 = fdiv(threadIdx.x, k.rcp_nc), j = threadIdx.x - t2 * n;
  const int g = fdiv(t2, c_rcp_run[cnt]), so = t2 - g * cnt;
  const int groups = fdiv(fdiv(SP_THREADS, k.rcp_nc), c_rcp_run[cnt]);   // = SP_THREADS / (cnt * n)
  if (g >= groups) return;
  const int x = so * n + j;
  const uint16_t* src = sh.cc[clear ? 0 : sh.list_c[q0 + so]] + j;
  uint8_t* base = reinterpret_cast<uint8_t*>(k.planes_c) + ((size_t)by * n) * k.cpitch + ((size_t)bx0 * n + x) * 2;
  for (int row = g; row < 3 * n; row += groups) {      // row = c * n + i
    const int c = row >= 2 * n ? 2 : (row >= n ? 1 : 0), i = row - c * n;
    const uint32_t code = clear ? 0u : src[c * k.lc_stride + i * n];
    *reinterpret_cast<uint16_t*>(base + ((size_t)c * k.ch + i) * k.cpitch) = (uint16_t)(code << k.color_shift);
  }
}

// Visibility bytes of slots [a, b) (one block row) from staged codes. An
// atlas row is the byte stream of its RG16F texels, texel X at stream bytes
// 4X..4X+3 = (R.lo, R.hi, G.lo, G.hi), i.e. the little-endian bytes of
// R | G << 16; stream byte s goes to plane s % 3, column s / 3. Twelve stream
// bytes (three texels) are therefore exactly one 32-bit word of each plane, so
// a thread owns one such chunk of one atlas row and writes three aligned words,
// byte-permuted from the three texels; the run's first and last chunks share
// bytes with neighbouring slots (written by other blocks) and are written byte
// by byte, only where they belong to these slots.
__device__ __forceinline__ void write_vis_run(const pv_dev& k, SpShared& sh, int a, int b, int q0, bool clear) {
  const int n = k.nv, by = a / k.bw, bx0 = a - by * k.bw;
  // the run's texel columns -> offset of their row-0 R code in the staging area
  // (block-uniform: every thread of the block takes the same runs)
  if (!clear) {
    for (int X = threadIdx.x; X < n * (b - a); X += SP_THREADS) {
      const int so = fdiv(X, k.rcp_nv), j = X - so * n;
      sh.xoff[X] = (uint16_t)(sh.list_v[q0 + so] * (2 * SP_MAX_T) + j);
    }
    __syncthreads();
  }
  const uint16_t* cv0 = &sh.cv[0][0];
  const int s_lo = 4 * n * bx0, s_hi = 4 * n * (bx0 + (b - a));   // stream bytes [s_lo, s_hi)
  const int w_lo = s_lo / 12, w_hi = (s_hi - 1) / 12;             // chunks touched
  const int nw = w_hi - w_lo + 1;
  const uint32_t rcp_nw = (0x80000000u + (uint32_t)nw - 1u) / (uint32_t)nw;
  const size_t plane = (size_t)k.vh * k.vpitch;
  for (int q = threadIdx.x; q < n * nw; q += SP_THREADS) {
    const int i = fdiv(q, rcp_nw), w = w_lo + (q - i * nw);
    uint32_t t3[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {                                 // texels 3w, 3w+1, 3w+2 of the atlas row
      const int X = 3 * w + e - n * bx0;                          // texel column within the run
      t3[e] = 0u;
      if (!clear && X >= 0 && X < n * (b - a)) {
        const uint16_t* src = cv0 + sh.xoff[X] + i * n;
        t3[e] = (uint32_t)src[0] | (uint32_t)src[k.lv_stride] << 16;
      }
    }
    const uint32_t w0 = __byte_perm(__byte_perm(t3[0], t3[1], 0x0630), t3[2], 0x5210);
    const uint32_t w1 = __byte_perm(__byte_perm(t3[0], t3[1], 0x0741), t3[2], 0x6210);
    const uint32_t w2 = __byte_perm(__byte_perm(t3[0], t3[1], 0x0052), t3[2], 0x7410);
    uint8_t* dst = k.planes_v + ((size_t)by * n + i) * k.vpitch + 4 * (size_t)w;
    if (12 * w >= s_lo && 12 * w + 12 <= s_hi) {
      *reinterpret_cast<uint32_t*>(dst) = w0;
      *reinterpret_cast<uint32_t*>(dst + plane) = w1;
      *reinterpret_cast<uint32_t*>(dst + 2 * plane) = w2;
    } else {
      const uint32_t ws[3] = {w0, w1, w2};
#pragma unroll
      for (int pl = 0; pl < 3; ++pl)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int sb = 12 * w + 3 * e + pl;                     // stream byte of this plane byte
          if (sb >= s_lo && sb < s_hi) dst[pl * plane + e] = (uint8_t)(ws[pl] >> (8 * e));
        }
    }
  }
  if (!clear) __syncthreads();                                  // the table is rebuilt by the next run
}

// Slots [s0, s1) split into runs within one block row; each run written by
// `fn` with staged codes from index q0 (+ its offset in [s0, s1)).
template <typename F>
__device__ __forceinline__ void for_runs(const pv_dev& k, int s0, int s1, F fn) {
  for (int a = s0; a < s1;) {
    const int row_end = (a / k.bw + 1) * k.bw;
    const int b = s1 < row_end ? s1 : row_end;
    fn(a, b, a - s0);
    a = b;
  }
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}

// Block `bid` of the `nblocks` blocks that select and pack volume k; block
// bid owns probes [bid * SP_RANGE, (bid + 1) * SP_RANGE).
__device__ __forceinline__ void select_pack_block(const pv_dev& k, int bid, int nblocks) {
  __shared__ __align__(16) SpShared sh;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int pb = bid * SP_RANGE, pe = min(k.P, pb + SP_RANGE);
  const int W = k.chg_words, wb = pb >> 5;
  const int vc = k.lc_stride / 8, vv = k.lv_stride / 8;    // 16-byte vectors per channel row

  // 0. copies of the block's current codes into shared memory, in flight
  //    while the masks are read (every probe of the range: most are selected)
  for (int it = tid; it < (pe - pb) * 3 * vc; it += SP_THREADS) {
    const int t = fdiv(it, k.rcp_vc), v = it - t * vc, q = t / 3, c = t - 3 * q;
    cp_async16(&sh.cc[q][c * k.lc_stride + 8 * v], k.cur_c + ((size_t)c * k.P + pb + q) * k.lc_stride + 8 * v);
  }
  for (int it = tid; it < (pe - pb) * 2 * vv; it += SP_THREADS) {
    const int t = fdiv(it, k.rcp_vv), v = it - t * vv, q = t >> 1, c = t & 1;
    cp_async16(&sh.cv[q][c * k.lv_stride + 8 * v], k.cur_v + ((size_t)c * k.P + pb + q) * k.lv_stride + 8 * v);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");

  // 1. first warp: select state, totals, selected probes before this block's
  //    word and the last of them, then the slots of the block's probes (lane
  //    = bit of the block's word, rank from a prefix count of the word). All
  //    loads are issued before any is used.
  if (wid == 0) {
    const unsigned long long fr = *k.frame, sf = *k.sel_frame;
    const uint32_t seq = k.sel[0];
    const uint32_t cnt2 = k.sel[2], cnt3 = k.sel[3], cnt4 = k.sel[4], cnt5 = k.sel[5];
    const uint32_t own_c = k.chg[wb], own_v = k.chg[W + wb];
    int tot_c = 0, tot_v = 0, bef_c = 0, bef_v = 0, last_c = -1, last_v = -1;
#pragma unroll 4
    for (int w = lane; w < W; w += 32) {
      const uint32_t mc = k.chg[w], mv = k.chg[W + w];
      tot_c += __popc(mc);
      tot_v += __popc(mv);
      if (w < wb) {
        bef_c += __popc(mc);
        bef_v += __popc(mv);
        if (mc) last_c = max(last_c, 32 * w + 31 - __clz(mc));
        if (mv) last_v = max(last_v, 32 * w + 31 - __clz(mv));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tot_c += __shfl_xor_sync(0xffffffffu, tot_c, o);
      tot_v += __shfl_xor_sync(0xffffffffu, tot_v, o);
      bef_c += __shfl_xor_sync(0xffffffffu, bef_c, o);
      bef_v += __shfl_xor_sync(0xffffffffu, bef_v, o);
      last_c = max(last_c, __shfl_xor_sync(0xffffffffu, last_c, o));
      last_v = max(last_v, __shfl_xor_sync(0xffffffffu, last_v, o));
    }
    const bool fresh = fr != sf;                   // masks not yet consumed by a select
    if (!fresh) tot_c = tot_v = bef_c = bef_v = 0, last_c = last_v = -1;
    const uint32_t mc = (fresh && pb < pe) ? own_c : 0u, mv = (fresh && pb < pe) ? own_v : 0u;
    const uint32_t below = (1u << lane) - 1u;
    const int p = 32 * wb + lane;
    const bool in = p >= pb && p < pe;
    const bool selc = in && ((mc >> lane) & 1u), selv = in && ((mv >> lane) & 1u);
    const uint32_t bal_c = __ballot_sync(0xffffffffu, selc), bal_v = __ballot_sync(0xffffffffu, selv);
    const int rank_c = __popc(bal_c & below), rank_v = __popc(bal_v & below);
    if (selc) sh.list_c[rank_c] = p - pb;
    if (selv) sh.list_v[rank_v] = p - pb;
    if (selc && rank_c == 0) sh.first_c = bef_c + __popc(mc & below);
    if (selv && rank_v == 0) sh.first_v = bef_v + __popc(mv & below);
    if (lane == 0) {
      sh.n_c = __popc(bal_c);
      sh.n_v = __popc(bal_v);
      sh.tot_c = tot_c;
      sh.tot_v = tot_v;
      const bool odd = (seq & 1u) != 0u;           // previous counts: the other parity's pair
      sh.prev_cnt_c = (int)(odd ? cnt2 : cnt4);
      sh.prev_cnt_v = (int)(odd ? cnt3 : cnt5);
      sh.seq = seq;
    }
    if (in) {
      const uint32_t bc = mc & below, bv = mv & below;
      sh.slot_c[p - pb] = ((mc >> lane) & 1u) ? bef_c + __popc(bc) : -1;
      sh.slot_v[p - pb] = ((mv >> lane) & 1u) ? bef_v + __popc(bv) : -1;
      const int lc = bc ? 32 * wb + 31 - __clz(bc) : last_c;
      const int lv = bv ? 32 * wb + 31 - __clz(bv) : last_v;
      sh.prev_c[p - pb] = (uint16_t)(lc < 0 ? 0 : lc);
      sh.prev_v[p - pb] = (uint16_t)(lv < 0 ? 0 : lv);
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int n_c = sh.n_c, n_v = sh.n_v, first_c = sh.first_c, first_v = sh.first_v;
  const int tot_c = sh.tot_c, tot_v = sh.tot_v, prev_cnt_c = sh.prev_cnt_c, prev_cnt_v = sh.prev_cnt_v;
  const uint32_t seq = sh.seq, par = seq & 1u;
  const int* list_c = sh.list_c;
  const int* list_v = sh.list_v;
  // every thread of the block has what it needs of the select state (the
  // sequence, the previous counts, the frame of the last select): the last
  // block to get here advances it for the next select
  if (tid == 0) {
    const uint32_t ticket = atomicAdd(&k.sel[1], 1u);
    if (ticket == (uint32_t)nblocks - 1) {
      k.sel[1] = 0;
      k.sel[0] = seq + 1u;
      *k.sel_frame = *k.frame;
    }
  }

  // 2. the selected probes' codes into the last-transmitted textures
  for (int it = tid; it < n_c * 3 * vc; it += SP_THREADS) {
    const int t = fdiv(it, k.rcp_vc), v = it - t * vc, r = t / 3, c = t - 3 * r, q = list_c[r];
    reinterpret_cast<uint4*>(k.last_c + ((size_t)c * k.P + pb + q) * k.lc_stride)[v] =
        *reinterpret_cast<const uint4*>(&sh.cc[q][c * k.lc_stride + 8 * v]);
  }
  for (int it = tid; it < n_v * 2 * vv; it += SP_THREADS) {
    const int t = fdiv(it, k.rcp_vv), v = it - t * vv, r = t >> 1, c = t & 1, q = list_v[r];
    reinterpret_cast<uint4*>(k.last_v + ((size_t)c * k.P + pb + q) * k.lv_stride)[v] =
        *reinterpret_cast<const uint4*>(&sh.cv[q][c * k.lv_stride + 8 * v]);
  }
  // 3. index buffers
  if (tid < n_c) {
    const int lp = list_c[tid], sc = sh.slot_c[lp];
    k.idx_c[sc] = (uint16_t)(pb + lp);
    k.delta_c[sc] = (uint16_t)(pb + lp - sh.prev_c[lp]);
  }
  if (tid >= 32 && tid - 32 < n_v) {
    const int lp = list_v[tid - 32], sv = sh.slot_v[lp];
    k.idx_v[sv] = (uint16_t)(pb + lp);
    k.delta_v[sv] = (uint16_t)(pb + lp - sh.prev_v[lp]);
  }

  // 4. the block's slots into the planes, one block row at a time
  if (n_c > 0)
    for_runs(k, first_c, first_c + n_c, [&](int a, int b, int q0) { write_color_run(k, sh, a, b, q0, false); });
  if (n_v > 0)
    for_runs(k, first_v, first_v + n_v, [&](int a, int b, int q0) { write_vis_run(k, sh, a, b, q0, false); });
  // 5. clear slots used by the previous frame and empty now, SP_RANGE at a time
  for (int a = tot_c + bid * SP_RANGE; a < prev_cnt_c; a += nblocks * SP_RANGE)
    for_runs(k, a, min(prev_cnt_c, a + SP_RANGE), [&](int x, int y, int q0) { write_color_run(k, sh, x, y, q0, true); });
  for (int a = tot_v + bid * SP_RANGE; a < prev_cnt_v; a += nblocks * SP_RANGE)
    for_runs(k, a, min(prev_cnt_v, a + SP_RANGE), [&](int x, int y, int q0) { write_vis_run(k, sh, x, y, q0, true); });
  // 6. counts, into this select's parity slot (the previous counts, read
  //    above by every block, sit in the other one)
  if (bid == 0 && tid == 0) {
    k.counts[0] = (uint32_t)tot_c;
    k.counts[1] = (uint32_t)tot_v;
    k.sel[2 + 2 * par] = (uint32_t)tot_c;
    k.sel[3 + 2 * par] = (uint32_t)tot_v;
  }
}

__global__ void __launch_bounds__(SP_THREADS) k_select_pack(pv_dev k) {
  pv_grid_launch_dependents();
  pv_grid_wait();
  select_pack_block(k, blockIdx.x, gridDim.x);
}

// Several volumes in one launch: blockIdx.y is the volume.
struct SpBatch {
  pv_dev k[PV_MAX_BATCH];
  int nblocks[PV_MAX_BATCH];
};

__global__ void __launch_bounds__(SP_THREADS) k_select_pack_batch(const __grid_constant__ SpBatch b) {
  pv_grid_launch_dependents();
  pv_grid_wait();
  const int v = blockIdx.y;
  if ((int)blockIdx.x >= b.nblocks[v]) return;
  select_pack_block(b.k[v], blockIdx.x, b.nblocks[v]);
}


}  // namespace

cudaError_t pv_launch_select_pack(const pv_dev& k, cudaStream_t st) {
  const int blocks = (k.P + SP_RANGE - 1) / SP_RANGE;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1] = {pv_pdl_attr()};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(SP_THREADS);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_select_pack, k);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t pv_launch_select_pack_batch(const pv_dev* ks, int n, cudaStream_t st) {
  if (n < 1 || n > PV_MAX_BATCH) return cudaErrorInvalidValue;
  SpBatch* b = new SpBatch();
  int most = 0;
  for (int i = 0; i < n; ++i) {
    b->k[i] = ks[i];
    b->nblocks[i] = (ks[i].P + SP_RANGE - 1) / SP_RANGE;
    most = b->nblocks[i] > most ? b->nblocks[i] : most;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1] = {pv_pdl_attr()};
  cfg.gridDim = dim3(most, n);
  cfg.blockDim = dim3(SP_THREADS);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_select_pack_batch, *b);
  delete b;
  return e != cudaSuccess ? e : cudaGetLastError();
}

namespace {

// After a state import: recompute every (channel, probe) changed flag.
__global__ void __launch_bounds__(256) k_recompute_flags(pv_dev k) {
  const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= 5LL * k.P) return;
  const int ch5 = (int)(item / k.P), p = (int)(item % k.P);
  const bool vis = ch5 >= 3;
  const int ch = vis ? ch5 - 3 : ch5;
  const int n = vis ? k.nv : k.nc, tile = n + 2, T = n * n;
  const void* st = vis ? k.state_v : k.state_c;
  const int sstride = vis ? k.sv_stride : k.sc_stride;
  const uint16_t* last = (vis ? k.last_v : k.last_c) + ((size_t)ch * k.P + p) * (vis ? k.lv_stride : k.lc_stride);
  int f = 0;
  for (int t = 0; t < T; ++t) {
    const size_t at = ((size_t)ch * k.P + p) * sstride + (size_t)(t / n + 1) * tile + (t % n + 1);
    const uint32_t code = vis ? pv::vis_code_of(st, at, k.state_fmt)
                              : pv::color_code_of(st, at, k.state_fmt, k.color_code);
    f |= code != last[t];
    if (k.cur_c)
      (vis ? k.cur_v : k.cur_c)[((size_t)ch * k.P + p) * (vis ? k.lv_stride : k.lc_stride) + t] = (uint16_t)code;
  }
  if (f) atomicOr(&k.chg[(vis ? k.chg_words : 0) + (p >> 5)], 1u << (p & 31));
}

}  // namespace

cudaError_t pv_launch_recompute_flags(const pv_dev& k, cudaStream_t st) {
  const long long items = 5LL * k.P;
  k_recompute_flags<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(k);
  return cudaGetLastError();
}
