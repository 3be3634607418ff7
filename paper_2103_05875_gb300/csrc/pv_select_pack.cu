// Change selection, probe index buffers and bit packing (Sections 3.3 and
// 3.4 of arXiv 2103.05875), fused into one kernel, plus the flag
// recomputation used after a state import.
//
// Selection: the blend raises bit p of the colour (visibility) mask when a
// transmitted code of probe p differs from its last-transmitted code; slots
// are assigned in ascending probe id. Each block reads both masks (P/8 bytes
// each) and reduces them, so it knows its probes' slots, the last selected
// probe before its range (for the delta code) and the totals without any
// grid-wide synchronisation. It then packs its own contiguous probe range, one
// warp per probe:
//   colour: the 10-bit codes of the interior go to planes Y=R, U=G, V=B at
//           block (k / B_w, k % B_w) as 16-bit samples (code << 6 unless
//           color_lsb), and to the last-transmitted texture;
//   visibility: per atlas row each texel's bytes (R.lo, R.hi, G.lo, G.hi)
//           continue the row's byte stream; byte s goes to plane s mod 3,
//           column s div 3 (the paper's YUVY / UVYU / VYUV pattern). Byte
//           stores, because neighbouring slots share plane words.
// Each block writes its probes' index-buffer entries and deltas
// (d0 = id0, dk = id_k - id_(k-1)), and clears its share of the slots that
// held a probe last frame but are empty now (slots beyond both counts are
// already zero). The masks count once per update: the kernel compares the
// frame counter with the frame of the previous select, so a second select
// without a new update selects nothing. The last block to finish advances the
// select sequence, which double-buffers the previous counts.
#include "pv_codes.cuh"
#include "pv_internal.h"

namespace {

constexpr int SP_THREADS = 256;
constexpr int SP_WARPS = SP_THREADS / 32;
constexpr int SP_MAX_RANGE = 512;        // probes per block
constexpr int SP_MAX_TEX = 3 * PV_MAX_INTERIOR * PV_MAX_INTERIOR;

struct SpTables {
  uint32_t col[SP_MAX_TEX];   // colour (c, t): c << 24 | tile_pos << 12 | i << 6 | j
  uint32_t vis[PV_MAX_INTERIOR * PV_MAX_INTERIOR];   // visibility t: tile_pos << 12 | i << 6 | j
};

// Colour block of slot `slot` from probe p (p < 0: clear the block). Loads of
// four codes per lane are issued before any of them is used.
__device__ __forceinline__ void pack_color_probe(const pv_dev& k, const SpTables& tb, int p, int slot, int lane) {
  const int by = slot / k.bw, bx = slot % k.bw;
  const int per = 3 * k.Tc;
  uint8_t* plane0 = reinterpret_cast<uint8_t*>(k.planes_c) + (size_t)by * k.nc * k.cpitch + (size_t)bx * k.nc * 2;
  for (int q0 = 0; q0 < per; q0 += 128) {
    uint32_t bits[4], ent[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + lane + 32 * u;
      ent[u] = q < per ? tb.col[q] : 0xFFFFFFFFu;
      bits[u] = 0;
      if (q < per && p >= 0) {
        const uint32_t c = ent[u] >> 24, pos = (ent[u] >> 12) & 0xFFFu;
        bits[u] = pv::load_state_bits(k.state_c, ((size_t)c * k.P + p) * k.sc_stride + pos, k.state_fmt);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (ent[u] == 0xFFFFFFFFu) continue;
      const uint32_t c = ent[u] >> 24, i = (ent[u] >> 6) & 63u, j = ent[u] & 63u;
      uint16_t* dst = reinterpret_cast<uint16_t*>(plane0 + ((size_t)c * k.ch + i) * k.cpitch) + j;
      if (p >= 0) {
        const uint32_t code = pv::color_code_of_bits(bits[u], k.state_fmt, k.color_code);
        *dst = (uint16_t)(code << k.color_shift);
        k.last_c[((size_t)c * k.P + p) * k.lc_stride + i * k.nc + j] = (uint16_t)code;
      } else {
        *dst = 0;
      }
    }
  }
}

// Visibility block of slot `slot` from probe p (p < 0: clear the block).
__device__ __forceinline__ void pack_vis_probe(const pv_dev& k, const SpTables& tb, int p, int slot, int lane) {
  const int by = slot / k.bw, bx = slot % k.bw;
  const int n = k.nv;
  for (int q0 = 0; q0 < k.Tv; q0 += 128) {
    uint32_t b0[4], b1[4], ent[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + lane + 32 * u;
      ent[u] = q < k.Tv ? tb.vis[q] : 0xFFFFFFFFu;
      b0[u] = b1[u] = 0;
      if (q < k.Tv && p >= 0) {
        const uint32_t pos = ent[u] >> 12;
        b0[u] = pv::load_state_bits(k.state_v, (size_t)p * k.sv_stride + pos, k.state_fmt);
        b1[u] = pv::load_state_bits(k.state_v, ((size_t)k.P + p) * k.sv_stride + pos, k.state_fmt);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (ent[u] == 0xFFFFFFFFu) continue;
      const int i = (int)((ent[u] >> 6) & 63u), j = (int)(ent[u] & 63u);
      uint32_t c0 = 0, c1 = 0;
      if (p >= 0) {
        c0 = pv::vis_code_of_bits(b0[u], k.state_fmt);
        c1 = pv::vis_code_of_bits(b1[u], k.state_fmt);
        k.last_v[(size_t)p * k.lv_stride + i * n + j] = (uint16_t)c0;
        k.last_v[((size_t)k.P + p) * k.lv_stride + i * n + j] = (uint16_t)c1;
      }
      const uint32_t bytes[4] = {c0 & 0xFFu, c0 >> 8, c1 & 0xFFu, c1 >> 8};
      const size_t y = (size_t)by * n + i;
      const int s0 = 4 * (bx * n + j);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int sb = s0 + b;
        const int pl = sb % 3;
        k.planes_v[((size_t)pl * k.vh + y) * k.vpitch + (size_t)(sb / 3)] = (uint8_t)bytes[b];
      }
    }
  }
}

// Block-wide sums (and maxima) of three values over all threads.
__device__ __forceinline__ void block_reduce3(int& a, int& b, int& c, int* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
  }
  if (lane == 0) { sh[3 * wid] = a; sh[3 * wid + 1] = b; sh[3 * wid + 2] = c; }
  __syncthreads();
  a = 0; b = 0; c = -1;
  for (int w = 0; w < SP_WARPS; ++w) { a += sh[3 * w]; b += sh[3 * w + 1]; c = max(c, sh[3 * w + 2]); }
  __syncthreads();
}

// Block `bid` of the `nblocks` blocks that select and pack volume k, each
// block owning `range` consecutive probes.
__device__ __forceinline__ void select_pack_block(const pv_dev& k, int range, int bid, int nblocks) {
  __shared__ SpTables tb;
  __shared__ int red[3 * SP_WARPS];
  __shared__ int slot_c[SP_MAX_RANGE], slot_v[SP_MAX_RANGE];
  __shared__ uint16_t prev_c[SP_MAX_RANGE], prev_v[SP_MAX_RANGE];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool fresh = *k.frame != *k.sel_frame;
  const uint32_t seq = k.sel[0];
  const uint32_t par = seq & 1u;
  const int prev_cnt_c = (int)k.sel[2 + 2 * (par ^ 1u)], prev_cnt_v = (int)k.sel[3 + 2 * (par ^ 1u)];
  const int pb = bid * range, pe = min(k.P, pb + range);
  const int W = k.chg_words, wb = pb >> 5;

  for (int q = tid; q < 3 * k.Tc; q += SP_THREADS) {
    const int c = q / k.Tc, t = q % k.Tc, i = t / k.nc, j = t % k.nc;
    tb.col[q] = ((uint32_t)c << 24) | ((uint32_t)((i + 1) * k.tc + j + 1) << 12) | ((uint32_t)i << 6) | (uint32_t)j;
  }
  for (int t = tid; t < k.Tv; t += SP_THREADS) {
    const int i = t / k.nv, j = t % k.nv;
    tb.vis[t] = ((uint32_t)((i + 1) * k.tv + j + 1) << 12) | ((uint32_t)i << 6) | (uint32_t)j;
  }

  // 1. totals, selected probes before this block's first word, last of them
  int tot_c = 0, tot_v = 0, dummy = -1;
  int bef_c = 0, bef_v = 0, last_c = -1, last_v = -1;
  if (fresh) {
    for (int w = tid; w < W; w += SP_THREADS) {
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
  }
  block_reduce3(tot_c, tot_v, dummy, red);
  int zero_c = 0;
  block_reduce3(bef_c, zero_c, last_c, red);
  int zero_v = 0;
  block_reduce3(bef_v, zero_v, last_v, red);

  // 2. slots of this block's probes: walk its words in order (thread 0; at
  //    most a few words per block)
  if (tid == 0) {
    int rc = bef_c, rv = bef_v, lc = last_c, lv = last_v;
    for (int w = wb; w <= ((pe - 1) >> 5) && pb < pe; ++w) {
      const uint32_t mc = fresh ? k.chg[w] : 0u, mv = fresh ? k.chg[W + w] : 0u;
      for (int bit = 0; bit < 32; ++bit) {
        const int p = 32 * w + bit;
        if (p >= pe) break;
        if (p < pb) {                                  // selected probes of this word before the range
          if ((mc >> bit) & 1u) { ++rc; lc = p; }
          if ((mv >> bit) & 1u) { ++rv; lv = p; }
          continue;
        }
        const bool sc = (mc >> bit) & 1u, sv = (mv >> bit) & 1u;
        if (p >= pb) {
          slot_c[p - pb] = sc ? rc : -1;
          slot_v[p - pb] = sv ? rv : -1;
          prev_c[p - pb] = (uint16_t)(lc < 0 ? 0 : lc);
          prev_v[p - pb] = (uint16_t)(lv < 0 ? 0 : lv);
        }
        if (sc) { ++rc; lc = p; }
        if (sv) { ++rv; lv = p; }
      }
    }
  }
  __syncthreads();

  // 3. pack this block's selected probes, one warp per probe
  for (int p = pb + wid; p < pe; p += SP_WARPS) {
    const int sc = slot_c[p - pb], sv = slot_v[p - pb];
    if (sc >= 0) {
      pack_color_probe(k, tb, p, sc, lane);
      if (lane == 0) { k.idx_c[sc] = (uint16_t)p; k.delta_c[sc] = (uint16_t)(p - prev_c[p - pb]); }
    }
    if (sv >= 0) {
      pack_vis_probe(k, tb, p, sv, lane);
      if (lane == 0) { k.idx_v[sv] = (uint16_t)p; k.delta_v[sv] = (uint16_t)(p - prev_v[p - pb]); }
    }
  }
  // 4. clear slots used by the previous frame and empty now
  for (int s = tot_c + bid * SP_WARPS + wid; s < prev_cnt_c; s += nblocks * SP_WARPS)
    pack_color_probe(k, tb, -1, s, lane);
  for (int s = tot_v + bid * SP_WARPS + wid; s < prev_cnt_v; s += nblocks * SP_WARPS)
    pack_vis_probe(k, tb, -1, s, lane);
  // 5. counts, and the select sequence once every block is done
  if (bid == 0 && tid == 0) {
    k.counts[0] = (uint32_t)tot_c;
    k.counts[1] = (uint32_t)tot_v;
    k.sel[2 + 2 * par] = (uint32_t)tot_c;
    k.sel[3 + 2 * par] = (uint32_t)tot_v;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const uint32_t ticket = atomicAdd(&k.sel[1], 1u);
    if (ticket == (uint32_t)nblocks - 1) {
      k.sel[1] = 0;
      k.sel[0] = seq + 1u;
      *k.sel_frame = *k.frame;
      __threadfence();
    }
  }
}

__global__ void __launch_bounds__(SP_THREADS) k_select_pack(pv_dev k, int range) {
  select_pack_block(k, range, blockIdx.x, gridDim.x);
}

// Several volumes in one launch: blockIdx.y is the volume.
struct SpBatch {
  pv_dev k[PV_MAX_BATCH];
  int range[PV_MAX_BATCH];
  int nblocks[PV_MAX_BATCH];
};

__global__ void __launch_bounds__(SP_THREADS) k_select_pack_batch(const __grid_constant__ SpBatch b) {
  const int v = blockIdx.y;
  if ((int)blockIdx.x >= b.nblocks[v]) return;
  select_pack_block(b.k[v], b.range[v], blockIdx.x, b.nblocks[v]);
}

// One probe per warp keeps every probe's loads in flight at once (a warp
// waits one memory round trip per probe); larger volumes take several.
int sp_range(const pv_dev& k, int sms) {
  int range = SP_WARPS;
  while ((k.P + range - 1) / range > 16 * sms && range < SP_MAX_RANGE) range *= 2;
  return range;
}

int device_sms() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

cudaError_t pv_launch_select_pack(const pv_dev& k, cudaStream_t st) {
  const int range = sp_range(k, device_sms());
  const int blocks = (k.P + range - 1) / range;
  k_select_pack<<<blocks, SP_THREADS, 0, st>>>(k, range);
  return cudaGetLastError();
}

cudaError_t pv_launch_select_pack_batch(const pv_dev* ks, int n, cudaStream_t st) {
  if (n < 1 || n > PV_MAX_BATCH) return cudaErrorInvalidValue;
  SpBatch* b = new SpBatch();
  const int sms = device_sms();
  int most = 0;
  for (int i = 0; i < n; ++i) {
    b->k[i] = ks[i];
    b->range[i] = sp_range(ks[i], sms);
    b->nblocks[i] = (ks[i].P + b->range[i] - 1) / b->range[i];
    most = b->nblocks[i] > most ? b->nblocks[i] : most;
  }
  k_select_pack_batch<<<dim3(most, n), SP_THREADS, 0, st>>>(*b);
  delete b;
  return cudaGetLastError();
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
  }
  if (f) atomicOr(&k.chg[(vis ? k.chg_words : 0) + (p >> 5)], 1u << (p & 31));
}

}  // namespace

cudaError_t pv_launch_recompute_flags(const pv_dev& k, cudaStream_t st) {
  const long long items = 5LL * k.P;
  k_recompute_flags<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(k);
  return cudaGetLastError();
}
