// Batched form: several volumes with equal tile shapes and formats updated
// together -- the weights of every volume in one launch, the blend of every
// volume in one persistent launch over all of their work items, and
// select-and-pack of every volume in one launch -- plus a tuner that picks the
// work-item size (probes per item) by timing candidates on the device.
#include <dlfcn.h>
#include <stdio.h>
#include <string.h>
#include <sys/stat.h>

#include <string>

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

// What trial launches of the blend overwrite, copied aside on the device and
// put back afterwards (the tuners leave every volume as they found it).
struct Snapshot {
  char* buf = nullptr;
  Saved sz[PV_MAX_BATCH];
  size_t total = 0;
  cudaError_t alloc(const pv_batch* b) {
    for (int i = 0; i < b->n; ++i) {
      sz[i] = saved_sizes(b->vols[i]);
      total += sz[i].tc + sz[i].tv + sz[i].cc + sz[i].cv + sz[i].chg + 64;
    }
    return cudaMalloc(&buf, total);
  }
  cudaError_t copy(const pv_batch* b, bool to_save, cudaStream_t st) {
    cudaError_t r = cudaSuccess;
    char* p = buf;
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
  }
  ~Snapshot() { cudaFree(buf); }
};

// Microseconds per blend launch of a trial plan built with `o` (one warm-up
// launch, then `reps` timed ones). *skip is set when the plan cannot be built
// or repeats one already timed (`seen`, its actual configuration).
struct Trial {
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  ~Trial() {
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
  }
};
cudaError_t time_plan(pv_batch* b, const pv_tc_opts& o, const void* const* rad, const void* const* dist, int reps,
                      cudaStream_t st, Trial& tr, pv_tc_opts* seen, int* nseen, float* us, bool* skip) {
  *skip = true;
  pv_tc_batch* plan = nullptr;
  if (pv_tc_batch_create_opts(b->vols, b->n, &o, &plan) != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;
  }
  pv_tc_opts got;
  pv_tc_batch_config(plan, &got);
  for (int i = 0; i < *nseen; ++i)
    if (memcmp(&seen[i], &got, sizeof(got)) == 0) {
      pv_tc_batch_destroy(plan);
      return cudaSuccess;
    }
  seen[(*nseen)++] = got;
  cudaError_t e = pv_tc_batch_launch(plan, rad, dist, st);
  if (e == cudaSuccess) e = cudaEventRecord(tr.t0, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = pv_tc_batch_launch(plan, rad, dist, st);
  if (e == cudaSuccess) e = cudaEventRecord(tr.t1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(tr.t1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, tr.t0, tr.t1);
  pv_tc_batch_destroy(plan);
  if (e == cudaSuccess) {
    *us = ms * 1000.0f / (float)reps;
    *skip = false;
  }
  return e;
}

// Tuning cache. One text line per tuned batch shape, later lines winning:
//   <key> TAB <probes_per_item> <ray_stages> <weight_stages> <tmem_stages> <ctas> <best_us> <default_us>
// The key names the library build (size and modification time of the loaded
// library file), the device (name, SM count), the formats and interiors, and
// every volume's probe count and rays per probe.
pv_status tune_key(const pv_batch* b, std::string* key) {
  cudaDeviceProp prop;
  const cudaError_t e = cudaGetDeviceProperties(&prop, b->device);
  if (e != cudaSuccess) return cuda_fail(e, "probe_batch_autotune: device properties");
  long long lib_size = 0, lib_mtime = 0;
  Dl_info info;
  struct stat stt;
  if (dladdr((void*)&probe_batch_autotune, &info) && info.dli_fname && stat(info.dli_fname, &stt) == 0) {
    lib_size = (long long)stt.st_size;
    lib_mtime = (long long)stt.st_mtime;
  }
  char name[sizeof(prop.name) + 1];
  int j = 0;
  for (int i = 0; prop.name[i] && i < (int)sizeof(prop.name); ++i) name[j++] = prop.name[i] == ' ' ? '_' : prop.name[i];
  name[j] = 0;
  const pv_desc& d = b->vols[0]->d;
  char buf[512];
  snprintf(buf, sizeof(buf), "pvtune1 lib=%lld:%lld dev=%s sms=%d op=%d state=%d code=%d nc=%d nv=%d vols=", lib_size,
           lib_mtime, name, prop.multiProcessorCount, (int)d.operand_fmt, (int)d.state_fmt, (int)d.color_code,
           (int)d.color_interior, (int)d.vis_interior);
  *key = buf;
  for (int i = 0; i < b->n; ++i) {
    snprintf(buf, sizeof(buf), "%dx%d,", b->vols[i]->k.P, b->vols[i]->k.R);
    *key += buf;
  }
  return PV_OK;
}

bool cache_lookup(const char* path, const std::string& key, pv_tc_opts* o, float* best_us, float* default_us) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  bool found = false;
  std::string line;
  char chunk[1024];
  while (fgets(chunk, sizeof(chunk), f)) {
    line += chunk;
    if (line.empty() || line.back() != '\n') continue;    // a line longer than the buffer: read on
    const size_t tab = line.find('\t');
    if (tab != std::string::npos && line.compare(0, tab, key) == 0 && tab == key.size()) {
      pv_tc_opts t = {};
      float bu = 0.0f, du = 0.0f;
      if (sscanf(line.c_str() + tab + 1, "%d %d %d %d %d %f %f", &t.probes_per_item, &t.ray_stages,
                 &t.weight_stages, &t.tmem_stages, &t.ctas, &bu, &du) == 7) {
        *o = t;
        *best_us = bu;
        *default_us = du;
        found = true;
      }
    }
    line.clear();
  }
  fclose(f);
  return found;
}

pv_status cache_store(const char* path, const std::string& key, const pv_tc_opts& o, float best_us,
                      float default_us) {
  FILE* f = fopen(path, "a");
  if (!f) return pv_set_error(PV_ERR_INVALID, "probe_batch_autotune: cannot append to the cache file %s", path);
  const int n = fprintf(f, "%s\t%d %d %d %d %d %.3f %.3f\n", key.c_str(), o.probes_per_item, o.ray_stages,
                        o.weight_stages, o.tmem_stages, o.ctas, best_us, default_us);
  const int c = fclose(f);
  if (n < 0 || c != 0) return pv_set_error(PV_ERR_INVALID, "probe_batch_autotune: writing %s failed", path);
  return PV_OK;
}

void fill_result(const pv_tc_opts& got, pv_tune_result* r) {
  r->probes_per_item = got.probes_per_item;
  r->ray_stages = got.ray_stages;
  r->weight_stages = got.weight_stages;
  r->tmem_stages = got.tmem_stages;
  r->ctas = got.ctas;
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
  Snapshot snap;
  if (snap.alloc(b) != cudaSuccess) return pv_set_error(PV_ERR_OOM, "probe_batch_tune: %zu scratch bytes", snap.total);
  cudaError_t e = snap.copy(b, true, st);
  pv_dev ks[PV_MAX_BATCH];
  for (int i = 0; i < b->n; ++i) ks[i] = b->vols[i]->k;
  if (e == cudaSuccess) e = pv_launch_weights_batch(ks, dirs, b->n, 0, 1, st);
  Trial tr;
  if (e == cudaSuccess) e = cudaEventCreate(&tr.t0);
  if (e == cudaSuccess) e = cudaEventCreate(&tr.t1);
  const int np_max = b->vols[0]->state_bytes == 2 ? 32 : 16;
  static const int cand[] = {8, 10, 12, 14, 16, 20, 24, 28, 32};
  pv_tc_opts seen[16];
  int nseen = 0, best_np = 0;
  float best = 1e30f;
  for (int c : cand) {
    if (e != cudaSuccess) break;
    if (c > np_max) continue;
    pv_tc_opts o = {};
    o.probes_per_item = c;
    float us = 0.0f;
    bool skip = true;
    e = time_plan(b, o, radiance, dist, reps, st, tr, seen, &nseen, &us, &skip);
    if (e == cudaSuccess && !skip && seen[nseen - 1].probes_per_item == c && us < best) {
      best = us;
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
  const cudaError_t r = snap.copy(b, false, st);
  if (e == cudaSuccess) e = r;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "probe_batch_tune");
  if (out_probes_per_item) *out_probes_per_item = pv_tc_batch_np(b->plan);
  return PV_OK;
}

pv_status probe_batch_autotune(pv_batch* b, const void* const* radiance, const void* const* dist,
                               const float* const* dirs, int32_t reps, const char* cache_path, pv_tune_result* out,
                               void* stream) {
  if (!b || !radiance || !dist || !dirs) return pv_set_error(PV_ERR_INVALID, "probe_batch_autotune: NULL argument");
  if (reps < 1) reps = 1;
  DeviceGuard g(b->device);
  cudaStream_t st = as_stream(stream);
  pv_tune_result res;
  memset(&res, 0, sizeof(res));
  std::string key;
  pv_status ks_status = tune_key(b, &key);
  if (ks_status != PV_OK) return ks_status;
  pv_tc_opts best = {};
  if (cache_path && cache_lookup(cache_path, key, &best, &res.best_us, &res.default_us)) {
    pv_tc_batch* plan = nullptr;
    const cudaError_t e = pv_tc_batch_create_opts(b->vols, b->n, &best, &plan);
    if (e == cudaSuccess) {
      pv_tc_batch_destroy(b->plan);
      b->plan = plan;
      res.from_cache = 1;
      pv_tc_opts got;
      pv_tc_batch_config(b->plan, &got);
      fill_result(got, &res);
      if (out) *out = res;
      return PV_OK;
    }
    cudaGetLastError();                                // a stale entry: tune again
  }
  Snapshot snap;
  if (snap.alloc(b) != cudaSuccess)
    return pv_set_error(PV_ERR_OOM, "probe_batch_autotune: %zu scratch bytes", snap.total);
  cudaError_t e = snap.copy(b, true, st);
  pv_dev kd[PV_MAX_BATCH];
  for (int i = 0; i < b->n; ++i) kd[i] = b->vols[i]->k;
  if (e == cudaSuccess) e = pv_launch_weights_batch(kd, dirs, b->n, 0, 1, st);
  Trial tr;
  if (e == cudaSuccess) e = cudaEventCreate(&tr.t0);
  if (e == cudaSuccess) e = cudaEventCreate(&tr.t1);
  pv_tc_opts seen[64];
  int nseen = 0;
  float best_us = 1e30f;
  auto consider = [&](const pv_tc_opts& o) {
    if (e != cudaSuccess || nseen >= 64) return;
    float us = 0.0f;
    bool skip = true;
    e = time_plan(b, o, radiance, dist, reps, st, tr, seen, &nseen, &us, &skip);
    if (e == cudaSuccess && !skip) {
      ++res.candidates;
      if (o.probes_per_item == 0 && o.ray_stages == 0 && o.weight_stages == 0 && o.tmem_stages == 0 && o.ctas == 0)
        res.default_us = us;
      if (us < best_us) {
        best_us = us;
        best = o;
      }
    }
  };
  // coordinate search from the default plan: probes per item, then the ring
  // depths, then TMEM stages (F32), then the CTA count
  const pv_tc_opts none = {};
  consider(none);
  const int np_max = b->vols[0]->state_bytes == 2 ? 32 : 16;
  static const int np_c[] = {8, 12, 16, 20, 24, 28, 32};
  pv_tc_opts base = best;
  for (int c : np_c)
    if (c <= np_max) {
      pv_tc_opts o = base;
      o.probes_per_item = c;
      consider(o);
    }
  base = best;
  static const int xs_c[] = {3, 4, 6, 8, 12};
  static const int ws_c[] = {2, 3, 4, 6};
  for (int x : xs_c)
    for (int w : ws_c) {
      pv_tc_opts o = base;
      o.ray_stages = x;
      o.weight_stages = w;
      consider(o);
    }
  if (b->vols[0]->d.operand_fmt == PV_FMT_F32) {
    base = best;
    for (int t : {2, 3, 4}) {
      pv_tc_opts o = base;
      o.tmem_stages = t;
      consider(o);
    }
  }
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  base = best;
  for (int div : {2, 4}) {
    pv_tc_opts o = base;
    o.ctas = sms / div > 0 ? sms / div : 1;
    consider(o);
  }
  if (e == cudaSuccess && best_us < 1e29f) {
    pv_tc_batch* plan = nullptr;
    e = pv_tc_batch_create_opts(b->vols, b->n, &best, &plan);
    if (e == cudaSuccess) {
      pv_tc_batch_destroy(b->plan);
      b->plan = plan;
    }
  }
  const cudaError_t r = snap.copy(b, false, st);
  if (e == cudaSuccess) e = r;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "probe_batch_autotune");
  res.best_us = best_us;
  pv_tc_opts got;
  pv_tc_batch_config(b->plan, &got);
  fill_result(got, &res);
  if (cache_path) {
    const pv_status ws = cache_store(cache_path, key, best, res.best_us, res.default_us);
    if (ws != PV_OK) return ws;
  }
  if (out) *out = res;
  return PV_OK;
}

}  // extern "C"
