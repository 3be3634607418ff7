// K2-K4: change selection, probe index buffers and bit packing (Sections 3.3
// and 3.4 of arXiv 2103.05875), plus the flag recomputation used after a
// state import.
//
// K2 (select): one block per texture (colour, visibility). Each probe's
//   changed flag is the OR of its channel flags written by the blend
//   epilogue; a block-wide exclusive scan in ascending probe id gives each
//   selected probe its slot. Writes the uint16 index buffer, its delta
//   encoding (d0 = id0, dk = id_k - id_(k-1)) and the counts, keeping the
//   previous frame's count so the pack kernels can clear slots that were used
//   last frame and are empty now.
// K3 (colour pack): one thread per (slot, channel, interior row): the row's
//   UF10/UNORM10 codes go to plane c at block (k / B_w, k % B_w) as 16-bit
//   samples (code << 6 unless color_lsb), and to the last-transmitted texture.
// K4 (visibility pack): output-centric; one thread per (atlas row, group of
//   three RG16F texels). The twelve bytes (R.lo, R.hi, G.lo, G.hi per texel)
//   are spread over Y, U, V as YUVY / UVYU / VYUV, i.e. one aligned 32-bit
//   word per plane, so plane rows are written with coalesced word stores.
// Slots at or beyond max(count, previous count) are left untouched: they are
// already zero.
#include "pv_codes.cuh"
#include "pv_internal.h"

namespace {

constexpr int SCAN_THREADS = 1024;

__global__ void __launch_bounds__(SCAN_THREADS) k_select(pv_dev k) {
  const int which = blockIdx.x;                  // 0 colour, 1 visibility
  const int nch = which ? 2 : 3;
  uint8_t* flags = k.flags + (size_t)(which ? 3 : 0) * k.P;
  uint16_t* idx = which ? k.idx_v : k.idx_c;
  uint16_t* delta = which ? k.delta_v : k.delta_c;
  const int tid = threadIdx.x;
  const int per = (k.P + SCAN_THREADS - 1) / SCAN_THREADS;
  const int b = min(k.P, tid * per), e = min(k.P, b + per);

  int local = 0;
  for (int p = b; p < e; ++p) {
    int f = 0;
    for (int c = 0; c < nch; ++c) f |= flags[(size_t)c * k.P + p];
    local += f != 0;
  }
  // block exclusive scan of the per-thread counts
  __shared__ int warp_tot[SCAN_THREADS / 32];
  const int lane = tid & 31, wid = tid >> 5;
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int v = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    warp_tot[lane] = v;                           // inclusive over warps
  }
  __syncthreads();
  const int excl = incl - local + (wid ? warp_tot[wid - 1] : 0);
  const int total = warp_tot[SCAN_THREADS / 32 - 1];

  int slot = excl;
  for (int p = b; p < e; ++p) {
    int f = 0;
    for (int c = 0; c < nch; ++c) f |= flags[(size_t)c * k.P + p];
    if (f) idx[slot++] = (uint16_t)p;
  }
  // every changed probe is sent now, so no flag stays raised: a second
  // select without a new update selects nothing
  for (int p = b; p < e; ++p)
    for (int c = 0; c < nch; ++c) flags[(size_t)c * k.P + p] = 0;
  __syncthreads();                               // idx visible block-wide
  for (int s = excl; s < excl + local; ++s)
    delta[s] = (uint16_t)(s ? (int)idx[s] - (int)idx[s - 1] : (int)idx[s]);
  if (tid == 0) {
    k.counts[2 + which] = k.counts[which];       // previous frame's count
    k.counts[which] = (uint32_t)total;
  }
}

__global__ void __launch_bounds__(256) k_pack_color(pv_dev k) {
  const int per_slot = 3 * k.nc;
  const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int slot = (int)(item / per_slot);
  if (slot >= k.P) return;
  const int cnt = (int)k.counts[0], prev = (int)k.counts[2];
  if (slot >= max(cnt, prev)) return;
  const int rem = (int)(item % per_slot);
  const int c = rem / k.nc, i = rem % k.nc;
  const int by = slot / k.bw, bx = slot % k.bw;
  uint16_t* dst = reinterpret_cast<uint16_t*>(
      reinterpret_cast<uint8_t*>(k.planes_c) + ((size_t)c * k.ch + (size_t)by * k.nc + i) * k.cpitch) +
      (size_t)bx * k.nc;
  if (slot < cnt) {
    const int p = k.idx_c[slot];
    const size_t row0 = ((size_t)c * k.P + p) * k.sc_stride + (size_t)(i + 1) * k.tc + 1;
    uint16_t* last = k.last_c + ((size_t)c * k.P + p) * k.lc_stride + (size_t)i * k.nc;
    for (int j = 0; j < k.nc; ++j) {
      const uint32_t code = pv::color_code_of(k.state_c, row0 + j, k.state_fmt, k.color_code);
      dst[j] = (uint16_t)(code << k.color_shift);
      last[j] = (uint16_t)code;
    }
  } else {
    for (int j = 0; j < k.nc; ++j) dst[j] = 0;
  }
}

__global__ void __launch_bounds__(256) k_pack_vis(pv_dev k) {
  const int W = k.bw * k.nv;                     // atlas width in texels
  const int U = (W + 2) / 3;                     // groups of three texels per row
  const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (long long)k.vh * U) return;
  const int y = (int)(item / U), u = (int)(item % U);
  const int by = y / k.nv, i = y % k.nv;
  const int cnt = (int)k.counts[1], prev = (int)k.counts[3];
  const int lim = max(cnt, prev);
  uint32_t bytes[12];
  bool touched = false;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    uint32_t lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
    const int t = 3 * u + q;
    if (t < W) {
      const int bx = t / k.nv, j = t % k.nv;
      const int slot = by * k.bw + bx;
      if (slot < lim) touched = true;
      if (slot < cnt) {
        const int p = k.idx_v[slot];
        const size_t off = (size_t)(i + 1) * k.tv + (j + 1);
        const size_t at0 = (size_t)p * k.sv_stride + off;
        const size_t at1 = ((size_t)k.P + p) * k.sv_stride + off;
        const uint32_t c0 = pv::vis_code_of(k.state_v, at0, k.state_fmt);
        const uint32_t c1 = pv::vis_code_of(k.state_v, at1, k.state_fmt);
        k.last_v[(size_t)p * k.lv_stride + (size_t)i * k.nv + j] = (uint16_t)c0;
        k.last_v[((size_t)k.P + p) * k.lv_stride + (size_t)i * k.nv + j] = (uint16_t)c1;
        lo0 = c0 & 0xFFu; hi0 = c0 >> 8; lo1 = c1 & 0xFFu; hi1 = c1 >> 8;
      }
    }
    bytes[4 * q + 0] = lo0;
    bytes[4 * q + 1] = hi0;
    bytes[4 * q + 2] = lo1;
    bytes[4 * q + 3] = hi1;
  }
  if (!touched) return;
#pragma unroll
  for (int pl = 0; pl < 3; ++pl) {
    const uint32_t word = bytes[pl] | (bytes[pl + 3] << 8) | (bytes[pl + 6] << 16) | (bytes[pl + 9] << 24);
    uint8_t* row = k.planes_v + ((size_t)pl * k.vh + y) * k.vpitch;
    reinterpret_cast<uint32_t*>(row)[u] = word;
  }
}

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

cudaError_t pv_launch_select(const pv_dev& k, cudaStream_t st) {
  k_select<<<2, SCAN_THREADS, 0, st>>>(k);
  return cudaGetLastError();
}

cudaError_t pv_launch_pack(const pv_dev& k, cudaStream_t st) {
  const long long items_c = (long long)k.P * 3 * k.nc;
  k_pack_color<<<(unsigned)((items_c + 255) / 256), 256, 0, st>>>(k);
  const int W = k.bw * k.nv;
  const long long items_v = (long long)k.vh * ((W + 2) / 3);
  k_pack_vis<<<(unsigned)((items_v + 255) / 256), 256, 0, st>>>(k);
  return cudaGetLastError();
}

cudaError_t pv_launch_recompute_flags(const pv_dev& k, cudaStream_t st) {
  const long long items = 5LL * k.P;
  k_recompute_flags<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(k);
  return cudaGetLastError();
}
