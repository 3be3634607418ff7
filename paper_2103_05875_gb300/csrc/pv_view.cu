// Shared-volume multi-client selection (Section 3.4 of arXiv 2103.05875): the
// server keeps one last-transmitted texture pair per client, so one update of
// a volume serves many clients, each selecting and packing against what it
// has already received. A view is one client's side of a volume: its
// last-transmitted codes, change masks, select state and packed frame. Its
// select compares the volume's current codes (kept by the blend) with its own
// last codes, then runs the volume's select/pack kernel on its own buffers.
#include <string.h>

#include "pv_codes.cuh"
#include "pv_internal.h"

struct pv_view {
  pv_volume* vol;
  int device;
  char* base;                 // one allocation for the view's buffers
  pv_dev k;                   // the volume's shapes and current codes, the view's buffers
  uint32_t* host_counts;      // pinned [2]
  uint32_t* cursors;          // device [2]: round-robin cursors of the colour and visibility budgets
  pv_view_opts opts;
};

namespace {

constexpr int VF_THREADS = 256;

// Changed-probe masks of one 32-probe word for a view: a probe changed when
// any of its current codes differs from the view's last code (a never-sent
// probe holds the sentinel 0xFFFF, which no code takes). Codes are compared
// eight at a time; the row padding past the T texels is ignored.
__global__ void __launch_bounds__(VF_THREADS) k_view_flags(const pv_dev k, const uint8_t* __restrict__ active,
                                                            uint32_t th_c, uint32_t th_v) {
  __shared__ uint32_t red[2];
  const int w = blockIdx.x, p0 = 32 * w, np = min(32, k.P - p0);
  const int vc = k.lc_stride / 8, vv = k.lv_stride / 8, per = 3 * vc + 2 * vv;
  const uint32_t rcp_per = (0x80000000u + (uint32_t)per - 1u) / (uint32_t)per;
  if (threadIdx.x < 2) red[threadIdx.x] = 0u;
  __syncthreads();
  uint32_t mc = 0, mv = 0;
  for (int it = threadIdx.x; it < np * per; it += VF_THREADS) {
    const int q = pv::fdiv(it, rcp_per), r = it - q * per;
    const bool vis = r >= 3 * vc;
    const int rr = vis ? r - 3 * vc : r, nvec = vis ? vv : vc;
    const int c = rr / nvec, v = rr - c * nvec;
    const int stride = vis ? k.lv_stride : k.lc_stride, T = vis ? k.Tv : k.Tc;
    const size_t row = ((size_t)c * k.P + p0 + q) * stride;
    const uint4 x = reinterpret_cast<const uint4*>((vis ? k.cur_v : k.cur_c) + row)[v];
    const uint4 y = reinterpret_cast<const uint4*>((vis ? k.last_v : k.last_c) + row)[v];
    const uint32_t xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
    const uint32_t th = vis ? th_v : th_c;
    bool diff = false;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int cu = (int)((xs[e >> 1] >> (16 * (e & 1))) & 0xFFFFu), la = (int)((ys[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
      // moved by more than the threshold, or never sent (the sentinel no code takes)
      if (8 * v + e < T) diff |= (uint32_t)abs(cu - la) > th || la == 0xFFFF;
    }
    if (diff) {
      if (vis) mv |= 1u << q;
      else mc |= 1u << q;
    }
  }
  mc = __reduce_or_sync(0xffffffffu, mc);
  mv = __reduce_or_sync(0xffffffffu, mv);
  if ((threadIdx.x & 31) == 0) {
    if (mc) atomicOr(&red[0], mc);
    if (mv) atomicOr(&red[1], mv);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t act = 0xffffffffu;                          // probes of the word that may be sent
    if (active) act = __ballot_sync(0xffffffffu, (int)threadIdx.x < np && active[p0 + threadIdx.x] != 0);
    if (threadIdx.x == 0) {
      k.chg[w] = red[0] & act;
      k.chg[k.chg_words + w] = red[1] & act;
    }
  }
}

// Per-client probe budget: of each texture's changed probes, keep the first
// `budget` in cyclic probe order from the texture's cursor; the cursor moves
// one past the last kept probe. One block; the first two warps find the cut of
// the colour and visibility masks, then every thread clears the bits outside
// the kept cyclic range. Does nothing when the masks were already consumed
// (no update since the last select), like the select itself.
__global__ void __launch_bounds__(1024) k_view_budget(const pv_dev k, uint32_t* cursors, int budget) {
  __shared__ int cut_s[2], old_s[2];
  if (*k.frame == *k.sel_frame) return;                  // uniform
  const int W = k.chg_words, P = k.P;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 2) {
    const uint32_t* words = k.chg + warp * W;
    const int cursor = (int)cursors[warp] % P, wc = cursor >> 5, bc = cursor & 31;
    const int nvirt = W + (bc > 0 ? 1 : 0);              // word wc split in two: bits >= bc first, < bc last
    int remaining = budget, cut = -1, last = -1;
    for (int j0 = 0; j0 < nvirt && cut < 0; j0 += 32) {
      const int j = j0 + lane;
      uint32_t m = 0u;
      int w = 0;
      if (j < nvirt) {
        w = j == W ? wc : (wc + j) % W;
        const uint32_t mask = j == 0 ? (0xffffffffu << bc) : (j == W ? ((1u << bc) - 1u) : 0xffffffffu);
        m = words[w] & mask;
      }
      const int c = __popc(m);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const uint32_t hit = __ballot_sync(0xffffffffu, incl >= remaining && c > 0);
      if (hit) {
        const int L = __ffs(hit) - 1;
        if (lane == L) {
          uint32_t mm = m;
          for (int r = remaining - (incl - c) - 1; r > 0; --r) mm &= mm - 1u;   // drop the earlier kept bits
          cut = 32 * w + __ffs(mm) - 1;
        }
        cut = __shfl_sync(0xffffffffu, cut, L);
      } else {
        remaining -= __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t nz = __ballot_sync(0xffffffffu, m != 0u);          // last candidate so far
        if (nz) {
          const int L = 31 - __clz(nz);
          int lb = 32 * w + 31 - __clz(m | 1u);
          last = __shfl_sync(0xffffffffu, lb, L);
        }
      }
    }
    if (lane == 0) {
      cut_s[warp] = cut;
      old_s[warp] = cursor;
      const int next = cut >= 0 ? (cut + 1) % P : (last >= 0 ? (last + 1) % P : cursor);
      cursors[warp] = (uint32_t)next;
    }
  }
  __syncthreads();
  // keep the candidates of the cyclic range [old cursor, cut]
  for (int q = threadIdx.x; q < 2 * W; q += blockDim.x) {
    const int t = q >= W ? 1 : 0, w = q - t * W;
    const int cut = cut_s[t], lo = old_s[t];
    if (cut < 0) continue;                               // nothing past the budget
    const auto range = [&](int a, int b) -> uint32_t {   // bits of word w for ids a..b
      const int s0 = max(a, 32 * w), s1 = min(b, 32 * w + 31);
      if (s0 > s1) return 0u;
      const int n = s1 - s0 + 1;
      return (n == 32 ? 0xffffffffu : ((1u << n) - 1u)) << (s0 - 32 * w);
    };
    const uint32_t keep = lo <= cut ? range(lo, cut) : (range(lo, P - 1) | range(0, cut));
    k.chg[t * W + w] &= keep;
  }
}

size_t up256(size_t x) { return pv_host::round_up(x, 256); }

using pv_host::cuda_fail;

}  // namespace

extern "C" {

pv_status pv_view_create(pv_volume* vol, pv_view** out) {
  if (!vol || !out) return pv_set_error(PV_ERR_INVALID, "pv_view_create: NULL argument");
  *out = nullptr;
  pv_geom g;
  pv_status s = pv_frame_geometry(&vol->d, &g);
  if (s != PV_OK) return s;
  pv_host::DeviceGuard guard(vol->device);
  const pv_dev& vk = vol->k;
  const size_t b_lc = up256((size_t)3 * vk.P * vk.lc_stride * 2), b_lv = up256((size_t)2 * vk.P * vk.lv_stride * 2);
  const size_t b_chg = up256((size_t)2 * vk.chg_words * 4), b_idx = up256((size_t)vk.P * 2);
  const size_t b_sel = 256;                                 // counts [2], select state [6], frame of last select
  const size_t b_pc = up256((size_t)3 * g.cheight * g.cpitch), b_pv = up256((size_t)3 * g.vheight * g.vpitch);
  const size_t total = b_lc + b_lv + b_chg + 4 * b_idx + b_sel + b_pc + b_pv;
  pv_view* v = new pv_view();
  memset(v, 0, sizeof(pv_view));
  v->vol = vol;
  v->device = vol->device;
  cudaError_t e = cudaMalloc((void**)&v->base, total);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&v->host_counts, 2 * sizeof(uint32_t));
  if (e != cudaSuccess) {
    cudaFree(v->base);
    delete v;
    cudaGetLastError();
    return pv_set_error(PV_ERR_OOM, "pv_view_create: %zu device bytes: %s", total, cudaGetErrorString(e));
  }
  v->k = vk;
  char* b = v->base;
  v->k.last_c = (uint16_t*)b;
  b += b_lc;
  v->k.last_v = (uint16_t*)b;
  b += b_lv;
  v->k.chg = (uint32_t*)b;
  b += b_chg;
  v->k.idx_c = (uint16_t*)b;
  b += b_idx;
  v->k.idx_v = (uint16_t*)b;
  b += b_idx;
  v->k.delta_c = (uint16_t*)b;
  b += b_idx;
  v->k.delta_v = (uint16_t*)b;
  b += b_idx;
  v->k.counts = (uint32_t*)b;
  v->k.sel = (uint32_t*)(b + 32);
  v->k.sel_frame = (unsigned long long*)(b + 64);
  v->cursors = (uint32_t*)(b + 80);
  b += b_sel;
  v->k.planes_c = (uint16_t*)b;
  b += b_pc;
  v->k.planes_v = (uint8_t*)b;
  // nothing sent yet: sentinel codes, zero frame, a select state that has never selected
  e = cudaMemset(v->base, 0, total);
  if (e == cudaSuccess) e = cudaMemset(v->k.last_c, 0xFF, b_lc + b_lv);
  if (e == cudaSuccess) {
    const unsigned long long never = ~0ull;
    e = cudaMemcpy(v->k.sel_frame, &never, sizeof never, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaFreeHost(v->host_counts);
    cudaFree(v->base);
    delete v;
    return cuda_fail(e, "pv_view_create");
  }
  *out = v;
  return PV_OK;
}

pv_status pv_view_destroy(pv_view* v) {
  if (!v) return PV_OK;
  pv_host::DeviceGuard guard(v->device);
  cudaFree(v->base);
  cudaFreeHost(v->host_counts);
  delete v;
  return PV_OK;
}

pv_status pv_view_set_options(pv_view* v, const pv_view_opts* o) {
  if (!v || !o) return pv_set_error(PV_ERR_INVALID, "pv_view_set_options: NULL argument");
  if (o->budget < 0 || o->threshold_c < 0 || o->threshold_v < 0)
    return pv_set_error(PV_ERR_INVALID, "pv_view_set_options: negative budget or threshold");
  v->opts = *o;
  return PV_OK;
}

pv_status pv_view_select_and_pack(pv_view* v, pv_frame* out, int32_t want_host_counts, void* stream) {
  if (!v || !out) return pv_set_error(PV_ERR_INVALID, "pv_view_select_and_pack: NULL argument");
  pv_host::DeviceGuard guard(v->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_view_flags<<<v->k.chg_words, VF_THREADS, 0, st>>>(v->k, v->opts.active, (uint32_t)v->opts.threshold_c,
                                                     (uint32_t)v->opts.threshold_v);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && v->opts.budget > 0) {
    k_view_budget<<<1, 1024, 0, st>>>(v->k, v->cursors, v->opts.budget);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = pv_launch_select_pack(v->k, st);
  out->color_planes = v->k.planes_c;
  out->vis_planes = v->k.planes_v;
  out->index_c = v->k.idx_c;
  out->index_v = v->k.idx_v;
  out->delta_c = v->k.delta_c;
  out->delta_v = v->k.delta_v;
  out->count_c_dev = v->k.counts;
  out->count_v_dev = v->k.counts + 1;
  out->count_c = -1;
  out->count_v = -1;
  out->frame = v->vol->frame;
  if (e == cudaSuccess && want_host_counts) {
    e = cudaMemcpyAsync(v->host_counts, v->k.counts, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
      out->count_c = v->host_counts[0];
      out->count_v = v->host_counts[1];
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "view select/pack");
  return PV_OK;
}

}  // extern "C"
