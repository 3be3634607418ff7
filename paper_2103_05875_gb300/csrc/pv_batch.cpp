// Batched form: several volumes with equal tile shapes and formats updated
// together -- the weights of every volume in one launch, the blend of every
// volume in one persistent launch over all of their work items, and
// select-and-pack of every volume in one launch -- plus a tuner that picks the
// work-item size (probes per item) by timing candidates on the device.
#include <string.h>

#include "pv_internal.h"

struct pv_batch {
  int n;
  int device;
  pv_volume* vols[PV_MAX_BATCH];
  pv_tc_batch* plan;
};

namespace {

using pv_host::as_stream;
using pv_host::cuda_fail;
using pv_host::DeviceGuard;

pv_status check_members(pv_volume* const* vols, int32_t n) {
  if (!vols || n < 1) return pv_set_error(PV_ERR_INVALID, "probe_batch_create: no volumes");
  if (n > PV_MAX_BATCH) return pv_set_error(PV_ERR_RANGE, "probe_batch_create: %d volumes, at most %d", n, PV_MAX_BATCH);
  for (int i = 0; i < n; ++i) {
    if (!vols[i]) return pv_set_error(PV_ERR_INVALID, "probe_batch_create: volume %d is NULL", i);
    for (int j = 0; j < i; ++j)
      if (vols[j] == vols[i]) return pv_set_error(PV_ERR_INVALID, "probe_batch_create: volume %d listed twice", i);
    const pv_desc& a = vols[0]->d;
    const pv_desc& b = vols[i]->d;
    if (vols[i]->device != vols[0]->device)
      return pv_set_error(PV_ERR_INVALID, "probe_batch_create: volumes on different devices");
    if (a.color_interior != b.color_interior || a.vis_interior != b.vis_interior || a.state_fmt != b.state_fmt ||
        a.operand_fmt != b.operand_fmt || a.color_code != b.color_code)
      return pv_set_error(PV_ERR_INVALID,
                          "probe_batch_create: volume %d differs in tile interiors, state or operand format, or "
                          "colour code",
                          i);
    if (vols[i]->kernel != PV_KERNEL_TCGEN05)
      return pv_set_error(PV_ERR_UNSUPPORTED, "probe_batch_create: volume %d does not use the tensor-core blend", i);
  }
  return PV_OK;
}

void fill_frame(pv_volume* v, pv_frame* out) {
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
  out->frame = v->frame;
}

// Device bytes a volume's blend writes besides the weights: its tiles, its
// current codes, its changed-probe bits, its frame counter and hysteresis.
struct Saved {
  size_t tc, tv, cc, cv, chg;
};

Saved saved_sizes(const pv_volume* v) {
  const pv_dev& k = v->k;
  const size_t sb = (size_t)v->state_bytes;
  return Saved{(size_t)3 * k.P * k.sc_stride * sb, (size_t)2 * k.P * k.sv_stride * sb,
               (size_t)3 * k.P * k.lc_stride * 2, (size_t)2 * k.P * k.lv_stride * 2,
               (size_t)2 * k.chg_words * sizeof(uint32_t)};
}

}  // namespace

extern "C" {

pv_status probe_batch_create(pv_volume* const* vols, int32_t n, int32_t probes_per_item, pv_batch** out) {
  if (!out) return pv_set_error(PV_ERR_INVALID, "probe_batch_create: NULL out");
  *out = nullptr;
  pv_status s = check_members(vols, n);
  if (s != PV_OK) return s;
  if (probes_per_item < 0) return pv_set_error(PV_ERR_INVALID, "probe_batch_create: negative probes_per_item");
  DeviceGuard g(vols[0]->device);
  pv_batch* b = new pv_batch();
  memset(b, 0, sizeof(pv_batch));
  b->n = n;
  b->device = vols[0]->device;
  for (int i = 0; i < n; ++i) b->vols[i] = vols[i];
  cudaError_t e = pv_tc_batch_create(b->vols, n, probes_per_item, &b->plan);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "probe_batch_create: blend plan");
  }
  *out = b;
  return PV_OK;
}

pv_status probe_batch_destroy(pv_batch* b) {
  if (!b) return PV_OK;
  pv_tc_batch_destroy(b->plan);
  delete b;
  return PV_OK;
}

pv_status probe_batch_info(const pv_batch* b, int32_t* probes_per_item) {
  if (!b || !probes_per_item) return pv_set_error(PV_ERR_INVALID, "probe_batch_info: NULL argument");
  *probes_per_item = pv_tc_batch_np(b->plan);
  return PV_OK;
}

pv_status probe_batch_update(pv_batch* b, const void* const* radiance, const void* const* dist,
                             const float* const* dirs, void* stream) {
  if (!b || !radiance || !dist || !dirs) return pv_set_error(PV_ERR_INVALID, "probe_batch_update: NULL argument");
  for (int i = 0; i < b->n; ++i)
    if (!radiance[i] || !dist[i] || !dirs[i])
      return pv_set_error(PV_ERR_INVALID, "probe_batch_update: NULL input of volume %d", i);
  DeviceGuard g(b->device);
  cudaStream_t st = as_stream(stream);
  pv_dev ks[PV_MAX_BATCH];
  for (int i = 0; i < b->n; ++i) ks[i] = b->vols[i]->k;
  cudaError_t e = pv_launch_weights_batch(ks, dirs, b->n, 0, 1, st);
  if (e != cudaSuccess) return cuda_fail(e, "batched weights kernel");
  for (int i = 0; i < b->n; ++i) b->vols[i]->frame += 1;
  e = pv_tc_batch_launch(b->plan, radiance, dist, st);
  if (e != cudaSuccess) return cuda_fail(e, "batched blend kernel");
  return PV_OK;
}

pv_status probe_batch_select_and_pack(pv_batch* b, pv_frame* out, void* stream) {
  if (!b || !out) return pv_set_error(PV_ERR_INVALID, "probe_batch_select_and_pack: NULL argument");
  DeviceGuard g(b->device);
  pv_dev ks[PV_MAX_BATCH];
  for (int i = 0; i < b->n; ++i) {
    ks[i] = b->vols[i]->k;
    pv_wait_downloads(b->vols[i], as_stream(stream));
  }
  cudaError_t e = pv_launch_select_pack_batch(ks, b->n, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "batched select/pack kernel");
  for (int i = 0; i < b->n; ++i) fill_frame(b->vols[i], &out[i]);
  return PV_OK;
}

pv_status probe_batch_tune(pv_batch* b, const void* const* radiance, const void* const* dist,
                           const float* const* dirs, int32_t reps, int32_t* out_probes_per_item, void* stream) {
  if (!b || !radiance || !dist || !dirs) return pv_set_error(PV_ERR_INVALID, "probe_batch_tune: NULL argument");
  if (reps < 1) reps = 1;
  DeviceGuard g(b->device);
  cudaStream_t st = as_stream(stream);
  // save what the trial launches overwrite
  size_t total = 0;
  Saved sz[PV_MAX_BATCH];
  for (int i = 0; i < b->n; ++i) {
    sz[i] = saved_sizes(b->vols[i]);
    total += sz[i].tc + sz[i].tv + sz[i].cc + sz[i].cv + sz[i].chg + 64;
  }
  char* save = nullptr;
  cudaError_t e = cudaMalloc(&save, total);
  if (e != cudaSuccess) return pv_set_error(PV_ERR_OOM, "probe_batch_tune: %zu scratch bytes", total);
  auto copy_all = [&](bool to_save) {
    cudaError_t r = cudaSuccess;
    char* p = save;
    for (int i = 0; i < b->n && r == cudaSuccess; ++i) {
      const pv_dev& k = b->vols[i]->k;
      void* dev[6] = {k.state_c, k.state_v, k.cur_c, k.cur_v, k.chg, k.frame};
      const size_t n[6] = {sz[i].tc, sz[i].tv, sz[i].cc, sz[i].cv, sz[i].chg, sizeof(unsigned long long)};
      for (int q = 0; q < 6 && r == cudaSuccess; ++q) {
        r = to_save ? cudaMemcpyAsync(p, dev[q], n[q], cudaMemcpyDeviceToDevice, st)
                    : cudaMemcpyAsync(dev[q], p, n[q], cudaMemcpyDeviceToDevice, st);
        p += n[q];
      }
      if (r == cudaSuccess)
        r = to_save ? cudaMemcpyAsync(p, k.hy, sizeof(float), cudaMemcpyDeviceToDevice, st)
                    : cudaMemcpyAsync(k.hy, p, sizeof(float), cudaMemcpyDeviceToDevice, st);
      p += 56;
    }
    return r;
  };
  e = copy_all(true);
  pv_dev ks[PV_MAX_BATCH];
  for (int i = 0; i < b->n; ++i) ks[i] = b->vols[i]->k;
  if (e == cudaSuccess) e = pv_launch_weights_batch(ks, dirs, b->n, 0, 1, st);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  const int np_max = b->vols[0]->state_bytes == 2 ? 32 : 16;
  static const int cand[] = {8, 10, 12, 14, 16, 20, 24, 28, 32};
  int best_np = 0;
  float best_ms = 1e30f;
  for (int c : cand) {
    if (e != cudaSuccess) break;
    if (c > np_max) continue;
    pv_tc_batch* trial = nullptr;
    if (pv_tc_batch_create(b->vols, b->n, c, &trial) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    const int np = pv_tc_batch_np(trial);
    if (np != c) {                                  // shared memory gave fewer probes: a repeat
      pv_tc_batch_destroy(trial);
      continue;
    }
    e = pv_tc_batch_launch(trial, radiance, dist, st);   // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(t0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = pv_tc_batch_launch(trial, radiance, dist, st);
    if (e == cudaSuccess) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    pv_tc_batch_destroy(trial);
    if (e == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best_np = c;
    }
  }
  if (e == cudaSuccess && best_np > 0) {
    pv_tc_batch* plan = nullptr;
    e = pv_tc_batch_create(b->vols, b->n, best_np, &plan);
    if (e == cudaSuccess) {
      pv_tc_batch_destroy(b->plan);
      b->plan = plan;
    }
  }
  const cudaError_t r = copy_all(false);
  if (e == cudaSuccess) e = r;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(save);
  if (e != cudaSuccess) return cuda_fail(e, "probe_batch_tune");
  if (out_probes_per_item) *out_probes_per_item = pv_tc_batch_np(b->plan);
  return PV_OK;
}

}  // extern "C"
