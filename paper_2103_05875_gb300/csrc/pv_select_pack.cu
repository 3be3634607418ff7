// Change selection, probe index buffers and bit packing (Sections 3.3 and
// 3.4 of arXiv 2103.05875), fused into one kernel, plus the flag
// recomputation used after a state import.
//
// Selection: a probe is sent iff any of its channel flags (raised by the
// blend when a transmitted code differs from the last-transmitted one) is
// set; slots are assigned in ascending probe id. Every block scans all flags
// (a few bytes per probe, from L2), so each block knows the slot of every
// probe and the total without a grid-wide synchronisation; it then packs its
// own contiguous range of probes, one warp per probe:
//   colour: the 10-bit codes of the interior go to planes Y=R, U=G, V=B at
//           block (k / B_w, k % B_w) as 16-bit samples (code << 6 unless
//           color_lsb), and to the last-transmitted texture;
//   visibility: per atlas row each texel's bytes (R.lo, R.hi, G.lo, G.hi)
//           continue the row's byte stream; byte s goes to plane s mod 3,
//           column s div 3 (the paper's YUVY / UVYU / VYUV pattern). Byte
//           stores, because neighbouring slots share plane words.
// Each block writes its probes' index-buffer entries and deltas
// (d0 = id0, dk = id_k - id_(k-1)); slots that held a probe last frame but
// are empty now are cleared (slots beyond both counts are already zero).
// Flags count only once per update: the kernel compares the frame counter
// with the frame of the previous select, so a second select without a new
// update selects nothing. The last block to finish advances the select
// sequence (which double-buffers the previous counts).
#include "pv_codes.cuh"
#include "pv_internal.h"

namespace {

constexpr int SP_THREADS = 256;
constexpr int SP_MAX_RANGE = 512;        // probes per block (shared slot tables)

// All loads of a probe's interior are issued before any is used, so a warp
// waits for one memory round trip per probe rather than one per texel.
__device__ __forceinline__ void pack_color_probe(const pv_dev& k, int p, int slot, int lane) {
  constexpr int MAXQ = 3 * PV_MAX_INTERIOR * PV_MAX_INTERIOR / 32;   // 24
  const int by = slot / k.bw, bx = slot % k.bw;
  const int per = 3 * k.Tc;
  uint32_t bits[MAXQ];
#pragma unroll
  for (int m = 0; m < MAXQ; ++m) {
    const int q = lane + 32 * m;
    bits[m] = 0;
    if (q < per && p >= 0) {
      const int c = q / k.Tc, t = q % k.Tc, i = t / k.nc, j = t % k.nc;
      bits[m] = pv::load_state_bits(k.state_c, ((size_t)c * k.P + p) * k.sc_stride + (size_t)(i + 1) * k.tc + (j + 1),
                                    k.state_fmt);
    }
  }
#pragma unroll
  for (int m = 0; m < MAXQ; ++m) {
    const int q = lane + 32 * m;
    if (q < per) {
      const int c = q / k.Tc, t = q % k.Tc, i = t / k.nc, j = t % k.nc;
      uint16_t* dst = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(k.planes_c) +
                                                  ((size_t)c * k.ch + (size_t)by * k.nc + i) * k.cpitch) +
                      (size_t)bx * k.nc + j;
      if (p >= 0) {
        const uint32_t code = pv::color_code_of_bits(bits[m], k.state_fmt, k.color_code);
        *dst = (uint16_t)(code << k.color_shift);
        k.last_c[((size_t)c * k.P + p) * k.lc_stride + t] = (uint16_t)code;
      } else {
        *dst = 0;
      }
    }
  }
}

__device__ __forceinline__ void pack_vis_probe(const pv_dev& k, int p, int slot, int lane) {
  constexpr int MAXQ = PV_MAX_INTERIOR * PV_MAX_INTERIOR / 32;        // 8
  const int by = slot / k.bw, bx = slot % k.bw;
  const int n = k.nv;
  uint32_t b0[MAXQ], b1[MAXQ];
#pragma unroll
  for (int m = 0; m < MAXQ; ++m) {
    const int q = lane + 32 * m;
    b0[m] = b1[m] = 0;
    if (q < k.Tv && p >= 0) {
      const size_t off = (size_t)(q / n + 1) * k.tv + (q % n + 1);
      b0[m] = pv::load_state_bits(k.state_v, (size_t)p * k.sv_stride + off, k.state_fmt);
      b1[m] = pv::load_state_bits(k.state_v, ((size_t)k.P + p) * k.sv_stride + off, k.state_fmt);
    }
  }
#pragma unroll
  for (int m = 0; m < MAXQ; ++m) {
    const int q = lane + 32 * m;
    if (q < k.Tv) {
      const int i = q / n, j = q % n;
      uint32_t c0 = 0, c1 = 0;
      if (p >= 0) {
        c0 = pv::vis_code_of_bits(b0[m], k.state_fmt);
        c1 = pv::vis_code_of_bits(b1[m], k.state_fmt);
        k.last_v[(size_t)p * k.lv_stride + q] = (uint16_t)c0;
        k.last_v[((size_t)k.P + p) * k.lv_stride + q] = (uint16_t)c1;
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

__global__ void __launch_bounds__(SP_THREADS) k_select_pack(pv_dev k, int range) {
  __shared__ int warp_c[SP_THREADS / 32], warp_v[SP_THREADS / 32];
  __shared__ int warp_lc[SP_THREADS / 32], warp_lv[SP_THREADS / 32];
  __shared__ int slot_c[SP_MAX_RANGE], slot_v[SP_MAX_RANGE];
  __shared__ uint16_t prev_c[SP_MAX_RANGE], prev_v[SP_MAX_RANGE];
  __shared__ int tot_c, tot_v;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool fresh = *k.frame != *k.sel_frame;
  const uint32_t seq = k.sel[0];
  const uint32_t par = seq & 1u;
  const int prev_cnt_c = (int)k.sel[2 + 2 * (par ^ 1u)], prev_cnt_v = (int)k.sel[3 + 2 * (par ^ 1u)];
  const int pb = blockIdx.x * range, pe = min(k.P, pb + range);

  // 1. scan of every probe's flags
  const int per = (k.P + SP_THREADS - 1) / SP_THREADS;
  const int b = min(k.P, tid * per), e = min(k.P, b + per);
  int nc = 0, nv = 0, lastc = -1, lastv = -1;
  if (fresh) {
    for (int p0 = b; p0 < e; p0 += 8) {               // loads of 8 probes in flight at once
      uint32_t fc[8], fv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int p = p0 + u;
        fc[u] = fv[u] = 0;
        if (p < e) {
          fc[u] = k.flags[p] | k.flags[(size_t)k.P + p] | k.flags[2 * (size_t)k.P + p];
          fv[u] = k.flags[3 * (size_t)k.P + p] | k.flags[4 * (size_t)k.P + p];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (fc[u]) { ++nc; lastc = p0 + u; }
        if (fv[u]) { ++nv; lastv = p0 + u; }
      }
    }
  }
  int ic = nc, iv = nv, mc = lastc, mv = lastv;        // inclusive sums / running max
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int yc = __shfl_up_sync(0xffffffffu, ic, o), yv = __shfl_up_sync(0xffffffffu, iv, o);
    const int zc = __shfl_up_sync(0xffffffffu, mc, o), zv = __shfl_up_sync(0xffffffffu, mv, o);
    if (lane >= o) { ic += yc; iv += yv; mc = max(mc, zc); mv = max(mv, zv); }
  }
  if (lane == 31) { warp_c[wid] = ic; warp_v[wid] = iv; warp_lc[wid] = mc; warp_lv[wid] = mv; }
  __syncthreads();
  if (tid == 0) {
    int sc = 0, sv = 0, lc = -1, lv = -1;
    for (int w = 0; w < SP_THREADS / 32; ++w) {
      const int a = warp_c[w], bb = warp_v[w], x = warp_lc[w], y = warp_lv[w];
      warp_c[w] = sc; warp_v[w] = sv; warp_lc[w] = lc; warp_lv[w] = lv;
      sc += a; sv += bb; lc = max(lc, x); lv = max(lv, y);
    }
    tot_c = sc; tot_v = sv;
  }
  __syncthreads();
  // exclusive prefix and last selected probe before this thread's chunk
  int rc = warp_c[wid] + ic - nc, rv = warp_v[wid] + iv - nv;
  const int up_c = __shfl_up_sync(0xffffffffu, mc, 1), up_v = __shfl_up_sync(0xffffffffu, mv, 1);
  int lc = max(warp_lc[wid], lane > 0 ? up_c : -1);
  int lv = max(warp_lv[wid], lane > 0 ? up_v : -1);
  // 2. slots of this block's probes
  if (fresh) {
    for (int p = b; p < e; ++p) {
      const int fc = k.flags[p] | k.flags[(size_t)k.P + p] | k.flags[2 * (size_t)k.P + p];
      const int fv = k.flags[3 * (size_t)k.P + p] | k.flags[4 * (size_t)k.P + p];
      if (p >= pb && p < pe) {
        slot_c[p - pb] = fc ? rc : -1;
        slot_v[p - pb] = fv ? rv : -1;
        prev_c[p - pb] = (uint16_t)(lc < 0 ? 0 : lc);
        prev_v[p - pb] = (uint16_t)(lv < 0 ? 0 : lv);
      }
      if (fc) { ++rc; lc = p; }
      if (fv) { ++rv; lv = p; }
    }
  } else {
    for (int p = max(b, pb); p < min(e, pe); ++p) { slot_c[p - pb] = -1; slot_v[p - pb] = -1; }
  }
  __syncthreads();
  const int cnt_c = tot_c, cnt_v = tot_v;
  // 3. pack this block's selected probes, one warp per probe
  for (int p = pb + wid; p < pe; p += SP_THREADS / 32) {
    const int sc = slot_c[p - pb], sv = slot_v[p - pb];
    if (sc >= 0) {
      pack_color_probe(k, p, sc, lane);
      if (lane == 0) { k.idx_c[sc] = (uint16_t)p; k.delta_c[sc] = (uint16_t)(p - prev_c[p - pb]); }
    }
    if (sv >= 0) {
      pack_vis_probe(k, p, sv, lane);
      if (lane == 0) { k.idx_v[sv] = (uint16_t)p; k.delta_v[sv] = (uint16_t)(p - prev_v[p - pb]); }
    }
  }
  // 4. clear slots used by the previous frame and empty now
  for (int s = cnt_c + blockIdx.x * (SP_THREADS / 32) + wid; s < prev_cnt_c; s += gridDim.x * (SP_THREADS / 32))
    pack_color_probe(k, -1, s, lane);
  for (int s = cnt_v + blockIdx.x * (SP_THREADS / 32) + wid; s < prev_cnt_v; s += gridDim.x * (SP_THREADS / 32))
    pack_vis_probe(k, -1, s, lane);
  // 5. counts, and the select sequence once every block is done
  if (blockIdx.x == 0 && tid == 0) {
    k.counts[0] = (uint32_t)cnt_c;
    k.counts[1] = (uint32_t)cnt_v;
    k.sel[2 + 2 * par] = (uint32_t)cnt_c;
    k.sel[3 + 2 * par] = (uint32_t)cnt_v;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const uint32_t ticket = atomicAdd(&k.sel[1], 1u);
    if (ticket == gridDim.x - 1) {
      k.sel[1] = 0;
      k.sel[0] = seq + 1u;
      *k.sel_frame = *k.frame;
      __threadfence();
    }
  }
}

}  // namespace

cudaError_t pv_launch_select_pack(const pv_dev& k, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int range = (k.P + 4 * sms - 1) / (4 * sms);       // about four blocks per SM
  if (range < 4) range = 4;
  if (range > SP_MAX_RANGE) range = SP_MAX_RANGE;
  const int blocks = (k.P + range - 1) / range;
  k_select_pack<<<blocks, SP_THREADS, 0, st>>>(k, range);
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
  k.flags[(size_t)ch5 * k.P + p] = (uint8_t)f;
}

}  // namespace

cudaError_t pv_launch_recompute_flags(const pv_dev& k, cudaStream_t st) {
  const long long items = 5LL * k.P;
  k_recompute_flags<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(k);
  return cudaGetLastError();
}
