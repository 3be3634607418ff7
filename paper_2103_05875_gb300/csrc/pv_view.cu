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
};

namespace {

constexpr int VF_THREADS = 256;

// Changed-probe masks of one 32-probe word for a view: a probe changed when
// any of its current codes differs from the view's last code (a never-sent
// probe holds the sentinel 0xFFFF, which no code takes). Codes are compared
// eight at a time; the row padding past the T texels is ignored.
__global__ void __launch_bounds__(VF_THREADS) k_view_flags(const pv_dev k) {
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
    const uint32_t d[4] = {x.x ^ y.x, x.y ^ y.y, x.z ^ y.z, x.w ^ y.w};
    bool diff = false;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (8 * v + e < T) diff |= ((d[e >> 1] >> (16 * (e & 1))) & 0xFFFFu) != 0u;
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
  if (threadIdx.x == 0) {
    k.chg[w] = red[0];
    k.chg[k.chg_words + w] = red[1];
  }
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

pv_status cuda_fail(cudaError_t e, const char* what) {
  return pv_set_error(PV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

extern "C" {

pv_status pv_view_create(pv_volume* vol, pv_view** out) {
  if (!vol || !out) return pv_set_error(PV_ERR_INVALID, "pv_view_create: NULL argument");
  *out = nullptr;
  pv_geom g;
  pv_status s = pv_frame_geometry(&vol->d, &g);
  if (s != PV_OK) return s;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != vol->device) cudaSetDevice(vol->device);
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
    if (prev != vol->device) cudaSetDevice(prev);
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
  if (prev != vol->device) cudaSetDevice(prev);
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
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != v->device) cudaSetDevice(v->device);
  cudaFree(v->base);
  cudaFreeHost(v->host_counts);
  if (prev != v->device) cudaSetDevice(prev);
  delete v;
  return PV_OK;
}

pv_status pv_view_select_and_pack(pv_view* v, pv_frame* out, int32_t want_host_counts, void* stream) {
  if (!v || !out) return pv_set_error(PV_ERR_INVALID, "pv_view_select_and_pack: NULL argument");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != v->device) cudaSetDevice(v->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_view_flags<<<v->k.chg_words, VF_THREADS, 0, st>>>(v->k);
  cudaError_t e = cudaGetLastError();
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
  if (prev != v->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "view select/pack");
  return PV_OK;
}

}  // extern "C"
