// Host side of the C ABI declared in include/probe_stream.h: descriptor
// validation, one device allocation per volume carved into its buffers, and
// the launch sequences of probe_update (K0 weights, K1 blend) and
// probe_select_and_pack (K2 select, K3/K4 pack).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>

#include "pv_internal.h"

namespace {

thread_local std::string g_last_error;

using pv_host::as_stream;
using pv_host::cuda_fail;
using pv_host::DeviceGuard;
using pv_host::round_up;

// Buffer sizes of a volume, computed from its descriptor alone.
struct Layout {
  int P, R, nc, nv, tc, tv, Tc, Tv, bw, bh;
  int cwidth, cheight, cpitch, vwidth, vheight, vpitch;
  int w_rows, w_rb, w_kc, w_vb, w_chunks;
  int sb, ob;
  int sc_stride, sv_stride, lc_stride, lv_stride;
  size_t off_state_c, off_state_v, off_last_c, off_last_v, off_cur_c, off_cur_v, off_flags, off_wrt, off_sums, off_wop,
      off_hy, off_frame, off_idx_c, off_idx_v, off_delta_c, off_delta_v, off_counts, off_planes_c,
      off_planes_v, off_err, off_sel, total;
};

pv_status validate(const pv_desc* d) {
  if (!d) return pv_set_error(PV_ERR_INVALID, "descriptor is NULL");
  if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0)
    return pv_set_error(PV_ERR_INVALID, "probe grid %dx%dx%d must be positive", d->nx, d->ny, d->nz);
  const long long P = (long long)d->nx * d->ny * d->nz;
  if (P > PV_MAX_PROBES)
    return pv_set_error(PV_ERR_RANGE, "%lld probes exceed the 2-byte index buffer limit %d", P,
                        PV_MAX_PROBES);
  if (d->rays_per_probe <= 0 || d->rays_per_probe > PV_MAX_RAYS)
    return pv_set_error(PV_ERR_RANGE, "rays_per_probe %d outside 1..%d", d->rays_per_probe,
                        PV_MAX_RAYS);
  if (d->color_interior <= 0 || d->color_interior > PV_MAX_INTERIOR || d->vis_interior <= 0 ||
      d->vis_interior > PV_MAX_INTERIOR)
    return pv_set_error(PV_ERR_RANGE, "tile interiors %d/%d outside 1..%d", d->color_interior,
                        d->vis_interior, PV_MAX_INTERIOR);
  if (!(d->hysteresis >= 0.0f && d->hysteresis < 1.0f))
    return pv_set_error(PV_ERR_INVALID, "hysteresis %g outside [0, 1)", (double)d->hysteresis);
  if (!(d->sharpness > 0.0f && d->sharpness < 1e4f))
    return pv_set_error(PV_ERR_INVALID, "sharpness %g must be positive", (double)d->sharpness);
  if (d->state_fmt != PV_FMT_F32 && d->state_fmt != PV_FMT_F16)
    return pv_set_error(PV_ERR_INVALID, "state_fmt must be PV_FMT_F32 or PV_FMT_F16");
  if (d->operand_fmt != PV_FMT_F32 && d->operand_fmt != PV_FMT_F16 && d->operand_fmt != PV_FMT_BF16)
    return pv_set_error(PV_ERR_INVALID, "operand_fmt must be F32, F16 or BF16");
  if (d->color_code != PV_CODE_UF10 && d->color_code != PV_CODE_UNORM10)
    return pv_set_error(PV_ERR_INVALID, "color_code must be UF10 or UNORM10");
  if (d->kernel != PV_KERNEL_AUTO && d->kernel != PV_KERNEL_SIMT && d->kernel != PV_KERNEL_TCGEN05)
    return pv_set_error(PV_ERR_INVALID, "kernel must be AUTO, SIMT or TCGEN05");
  return PV_OK;
}

Layout layout_of(const pv_desc* d) {
  Layout L{};
  L.P = d->nx * d->ny * d->nz;
  L.R = d->rays_per_probe;
  L.nc = d->color_interior;
  L.nv = d->vis_interior;
  L.tc = L.nc + 2;
  L.tv = L.nv + 2;
  L.Tc = L.nc * L.nc;
  L.Tv = L.nv * L.nv;
  L.bw = d->nx * d->ny;
  L.bh = d->nz;
  L.cwidth = L.bw * L.nc;
  L.cheight = L.bh * L.nc;
  L.cpitch = (int)round_up((size_t)L.cwidth * 2, 16);
  const int W = L.bw * L.nv;
  L.vwidth = (4 * W + 2) / 3;
  L.vheight = L.bh * L.nv;
  L.vpitch = (int)round_up((size_t)4 * ((W + 2) / 3), 16);
  // tensor-core weight images: 64-byte rows (16 FP32 or 32 16-bit weights
  // per chunk); visibility texels in rows 0..Tv-1, colour texels from the
  // next multiple of 16 (each block is one MMA's N, a multiple of 16)
  {
    const int eb = d->operand_fmt == PV_FMT_F32 ? 4 : 2;
    L.w_rb = 64;
    L.w_kc = L.w_rb / eb;
    L.w_vb = (int)round_up((size_t)L.Tv, 16);
    L.w_rows = L.w_vb + (int)round_up((size_t)L.Tc, 16);
    L.w_chunks = (L.R + L.w_kc - 1) / L.w_kc;
  }
  L.sb = d->state_fmt == PV_FMT_F16 ? 2 : 4;
  L.ob = d->operand_fmt == PV_FMT_F32 ? 4 : 2;
  // per-probe strides padded to 16 bytes so each probe's tile and code row can
  // be moved by bulk copies
  L.sc_stride = (int)round_up((size_t)L.tc * L.tc, 16 / L.sb);
  L.sv_stride = (int)round_up((size_t)L.tv * L.tv, 16 / L.sb);
  L.lc_stride = (int)round_up((size_t)L.Tc, 8);
  L.lv_stride = (int)round_up((size_t)L.Tv, 8);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = round_up(off + bytes, 256);
    return at;
  };
  L.off_state_c = take((size_t)3 * L.P * L.sc_stride * L.sb);
  L.off_state_v = take((size_t)2 * L.P * L.sv_stride * L.sb);
  L.off_last_c = take((size_t)3 * L.P * L.lc_stride * 2);
  L.off_last_v = take((size_t)2 * L.P * L.lv_stride * 2);
  L.off_cur_c = take((size_t)3 * L.P * L.lc_stride * 2);
  L.off_cur_v = take((size_t)2 * L.P * L.lv_stride * 2);
  L.off_flags = take((size_t)2 * ((L.P + 31) / 32) * 4);
  L.off_wrt = take((size_t)L.R * (L.Tc + L.Tv) * 4);
  L.off_sums = take((size_t)(L.Tc + L.Tv) * 4);
  // operand weights: F16 one binary16 plane, BF16 hi + lo bfloat16 planes, F32 hi + lo float planes
  const size_t w_planes = d->operand_fmt == PV_FMT_F16 ? 1 : 2;
  L.off_wop = take(w_planes * L.w_chunks * L.w_rows * L.w_rb);
  L.off_hy = take(16);
  L.off_frame = take(16);
  L.off_idx_c = take((size_t)L.P * 2);
  L.off_idx_v = take((size_t)L.P * 2);
  L.off_delta_c = take((size_t)L.P * 2);
  L.off_delta_v = take((size_t)L.P * 2);
  L.off_counts = take(16);
  L.off_sel = take(64);
  L.off_planes_c = take((size_t)3 * L.cheight * L.cpitch);
  L.off_planes_v = take((size_t)3 * L.vheight * L.vpitch);
  L.off_err = take(16);
  L.total = off;
  return L;
}

}  // namespace

pv_status pv_set_error(pv_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

namespace {

// Streams, events and the two staging halves of the host-buffer path, made
// on first use.
void release_host_path(pv_volume* v) {
  if (v->s_in) cudaStreamSynchronize(v->s_in);
  if (v->s_out) cudaStreamSynchronize(v->s_out);
  for (int i = 0; i < 2; ++i) {
    if (v->ev_in_done[i]) cudaEventDestroy(v->ev_in_done[i]);
    if (v->ev_in_free[i]) cudaEventDestroy(v->ev_in_free[i]);
  }
  if (v->ev_packed) cudaEventDestroy(v->ev_packed);
  for (int i = 0; i < PV_DL_RING; ++i)
    if (v->ev_out[i]) cudaEventDestroy(v->ev_out[i]);
  if (v->s_in) cudaStreamDestroy(v->s_in);
  if (v->s_out) cudaStreamDestroy(v->s_out);
  cudaFree(v->stage);
  v->stage = nullptr;
  v->s_in = v->s_out = nullptr;
  v->ev_packed = nullptr;
  for (int i = 0; i < 2; ++i) v->ev_in_done[i] = v->ev_in_free[i] = nullptr;
  for (int i = 0; i < PV_DL_RING; ++i) v->ev_out[i] = nullptr;
}

pv_status ensure_host_path(pv_volume* v) {
  if (v->s_out) return PV_OK;
  const size_t nr = (size_t)3 * v->k.P * v->k.R * v->op_bytes;
  const size_t nd = (size_t)v->k.P * v->k.R * v->op_bytes;
  const size_t nq = (size_t)3 * v->k.R * sizeof(float);
  v->stage_off_dist = round_up(nr, 256);
  v->stage_off_dirs = v->stage_off_dist + round_up(nd, 256);
  v->stage_half = v->stage_off_dirs + round_up(nq, 256);
  cudaError_t e = cudaMalloc((void**)&v->stage, 2 * v->stage_half);
  if (e != cudaSuccess) {
    v->stage = nullptr;
    cudaGetLastError();
    return pv_set_error(PV_ERR_OOM, "staging allocation of %zu bytes failed", 2 * v->stage_half);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&v->s_in, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&v->ev_in_done[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->ev_in_free[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->ev_packed, cudaEventDisableTiming);
  for (int i = 0; i < PV_DL_RING && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&v->ev_out[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&v->s_out, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    release_host_path(v);
    return cuda_fail(e, "host-buffer path setup");
  }
  return PV_OK;
}

bool is_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

}  // namespace

// Makes `st` wait for the volume's last queued frame download, which reads
// the planes and index buffers the next select rewrites.
void pv_wait_downloads(pv_volume* v, cudaStream_t st) {
  if (v->dl_seq > 0) cudaStreamWaitEvent(st, v->ev_out[(v->dl_seq - 1) % PV_DL_RING], 0);
}

pv_status pv_frame_geometry(const pv_desc* d, pv_geom* g) {
  const pv_status s = validate(d);
  if (s != PV_OK) return s;
  const Layout L = layout_of(d);
  g->P = L.P;
  g->nc = L.nc;
  g->nv = L.nv;
  g->tc = L.tc;
  g->tv = L.tv;
  g->bw = L.bw;
  g->bh = L.bh;
  g->cheight = L.cheight;
  g->cpitch = L.cpitch;
  g->vheight = L.vheight;
  g->vpitch = L.vpitch;
  g->vwidth = L.vwidth;
  return PV_OK;
}

extern "C" {

const char* pv_status_string(pv_status s) {
  switch (s) {
    case PV_OK: return "PV_OK";
    case PV_PENDING: return "PV_PENDING";
    case PV_ERR_INVALID: return "PV_ERR_INVALID";
    case PV_ERR_OOM: return "PV_ERR_OOM";
    case PV_ERR_CUDA: return "PV_ERR_CUDA";
    case PV_ERR_BUSY: return "PV_ERR_BUSY";
    case PV_ERR_TIMEOUT: return "PV_ERR_TIMEOUT";
    case PV_ERR_RANGE: return "PV_ERR_RANGE";
    case PV_ERR_UNSUPPORTED: return "PV_ERR_UNSUPPORTED";
  }
  return "PV_UNKNOWN";
}

const char* pv_last_error(void) { return g_last_error.c_str(); }

const char* pv_version(void) { return "probe-stream-gb300 0.1 (sm_103a)"; }

pv_status probe_volume_bytes(const pv_desc* d, uint64_t* out) {
  pv_status s = validate(d);
  if (s != PV_OK) return s;
  if (!out) return pv_set_error(PV_ERR_INVALID, "out is NULL");
  *out = layout_of(d).total;
  return PV_OK;
}

pv_status probe_volume_create(const pv_desc* d, pv_volume** out) {
  if (!out) return pv_set_error(PV_ERR_INVALID, "out is NULL");
  *out = nullptr;
  pv_status s = validate(d);
  if (s != PV_OK) return s;
  const char* why = nullptr;
  const bool tc_ok = pv_tc_supported(d, &why);
  int kernel = d->kernel;
  if (kernel == PV_KERNEL_TCGEN05 && !tc_ok)
    return pv_set_error(PV_ERR_UNSUPPORTED, "tcgen05 blend unavailable: %s", why ? why : "?");
  if (kernel == PV_KERNEL_AUTO) kernel = tc_ok ? PV_KERNEL_TCGEN05 : PV_KERNEL_SIMT;

  const Layout L = layout_of(d);
  pv_volume* v = (pv_volume*)calloc(1, sizeof(pv_volume));
  if (!v) return pv_set_error(PV_ERR_OOM, "host allocation failed");
  v->d = *d;
  v->kernel = kernel;
  cudaGetDevice(&v->device);
  cudaError_t e = cudaMalloc((void**)&v->base, L.total);
  if (e != cudaSuccess) {
    free(v);
    cudaGetLastError();
    return pv_set_error(PV_ERR_OOM, "cudaMalloc(%zu) failed: %s", L.total, cudaGetErrorString(e));
  }
  v->bytes = L.total;
  e = cudaMallocHost((void**)&v->host_counts, 4 * sizeof(uint32_t));
  if (e != cudaSuccess) {
    cudaFree(v->base);
    free(v);
    return pv_set_error(PV_ERR_OOM, "cudaMallocHost failed: %s", cudaGetErrorString(e));
  }
  v->state_bytes = L.sb;
  v->op_bytes = L.ob;
  v->cwidth = L.cwidth;
  pv_dev& k = v->k;
  k.P = L.P; k.R = L.R; k.nc = L.nc; k.nv = L.nv; k.tc = L.tc; k.tv = L.tv; k.Tc = L.Tc; k.Tv = L.Tv;
  k.bw = L.bw; k.bh = L.bh;
  k.cpitch = L.cpitch; k.ch = L.cheight;
  k.vpitch = L.vpitch; k.vh = L.vheight; k.vwidth = L.vwidth;
  k.state_fmt = d->state_fmt; k.operand_fmt = d->operand_fmt; k.color_code = d->color_code;
  k.color_shift = d->color_lsb ? 0 : 6;
  k.h = d->hysteresis; k.sharpness = d->sharpness;
  k.first_frame_no_hysteresis = d->first_frame_no_hysteresis ? 1 : 0;
  char* b = v->base;
  k.state_c = b + L.off_state_c;
  k.state_v = b + L.off_state_v;
  k.last_c = (uint16_t*)(b + L.off_last_c);
  k.last_v = (uint16_t*)(b + L.off_last_v);
  k.cur_c = (uint16_t*)(b + L.off_cur_c);
  k.cur_v = (uint16_t*)(b + L.off_cur_v);
  k.chg = (uint32_t*)(b + L.off_flags);
  k.chg_words = (L.P + 31) / 32;
  k.w_rt = (float*)(b + L.off_wrt);
  k.sums = (float*)(b + L.off_sums);
  k.w_op = b + L.off_wop;
  k.hy = (float*)(b + L.off_hy);
  k.frame = (unsigned long long*)(b + L.off_frame);
  k.idx_c = (uint16_t*)(b + L.off_idx_c);
  k.idx_v = (uint16_t*)(b + L.off_idx_v);
  k.delta_c = (uint16_t*)(b + L.off_delta_c);
  k.delta_v = (uint16_t*)(b + L.off_delta_v);
  k.counts = (uint32_t*)(b + L.off_counts);
  k.sel = (uint32_t*)(b + L.off_sel);
  k.sel_frame = (unsigned long long*)(b + L.off_sel + 32);
  k.planes_c = (uint16_t*)(b + L.off_planes_c);
  k.planes_v = (uint8_t*)(b + L.off_planes_v);
  k.w_rows = L.w_rows; k.w_rb = L.w_rb; k.w_kc = L.w_kc; k.w_vb = L.w_vb; k.w_chunks = L.w_chunks;
  k.sc_stride = L.sc_stride; k.sv_stride = L.sv_stride;
  k.lc_stride = L.lc_stride; k.lv_stride = L.lv_stride;
  k.rcp_nc = pv_rcp31((uint32_t)L.nc); k.rcp_nv = pv_rcp31((uint32_t)L.nv);
  k.rcp_vc = pv_rcp31((uint32_t)L.lc_stride / 8); k.rcp_vv = pv_rcp31((uint32_t)L.lv_stride / 8);
  k.err = (int*)(b + L.off_err);

  // zero everything, then mark every probe "never sent"
  e = cudaMemset(v->base, 0, L.total);
  if (e == cudaSuccess) e = cudaMemset(k.last_c, 0xFF, (size_t)3 * L.P * L.lc_stride * 2);
  if (e == cudaSuccess) e = cudaMemset(k.last_v, 0xFF, (size_t)2 * L.P * L.lv_stride * 2);
  if (e == cudaSuccess) e = cudaMemset(k.cur_c, 0xFF, (size_t)3 * L.P * L.lc_stride * 2);
  if (e == cudaSuccess) e = cudaMemset(k.cur_v, 0xFF, (size_t)2 * L.P * L.lv_stride * 2);
  if (e == cudaSuccess) {
    const unsigned long long never = ~0ull;           // no select yet: flags are fresh
    e = cudaMemcpy(k.sel_frame, &never, sizeof never, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = pv_simt_prepare();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess && kernel == PV_KERNEL_TCGEN05) e = pv_tc_plan_create(v);
  if (e != cudaSuccess) {
    pv_tc_plan_destroy(v);
    cudaFreeHost(v->host_counts);
    cudaFree(v->base);
    free(v);
    return cuda_fail(e, "probe_volume_create");
  }
  *out = v;
  return PV_OK;
}

pv_status probe_volume_destroy(pv_volume* v) {
  if (!v) return PV_OK;
  DeviceGuard g(v->device);
  pv_tc_plan_destroy(v);
  release_host_path(v);
  cudaFreeHost(v->host_counts);
  cudaFree(v->base);
  free(v);
  return PV_OK;
}

pv_status probe_volume_info(const pv_volume* v, pv_volume_info* o) {
  if (!v || !o) return pv_set_error(PV_ERR_INVALID, "NULL argument");
  const Layout L = layout_of(&v->d);
  o->probes = L.P;
  o->rays = L.R;
  o->color_tile = L.tc;
  o->vis_tile = L.tv;
  o->blocks_w = L.bw;
  o->blocks_h = L.bh;
  o->color_width = L.cwidth;
  o->color_height = L.cheight;
  o->color_pitch_bytes = L.cpitch;
  o->vis_width = L.vwidth;
  o->vis_height = L.vheight;
  o->vis_pitch_bytes = L.vpitch;
  o->kernel = v->kernel;
  o->state_bytes_per_texel = L.sb;
  o->device_bytes = v->bytes;
  o->error_word = v->k.err;
  return PV_OK;
}

pv_status probe_update_weights(pv_volume* v, const float* dirs, void* stream) {
  if (!v || !dirs) return pv_set_error(PV_ERR_INVALID, "probe_update_weights: NULL argument");
  DeviceGuard g(v->device);
  const bool tc = v->kernel == PV_KERNEL_TCGEN05;
  cudaError_t e = pv_launch_weights(v->k, dirs, tc ? 0 : 1, tc ? 1 : 0, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "weights kernel");
  v->frame += 1;
  return PV_OK;
}

pv_status probe_update_blend(pv_volume* v, const void* rad, const void* dist, void* stream) {
  if (!v || !rad || !dist) return pv_set_error(PV_ERR_INVALID, "probe_update_blend: NULL argument");
  DeviceGuard g(v->device);
  cudaStream_t st = as_stream(stream);
  cudaError_t e = v->kernel == PV_KERNEL_TCGEN05 ? pv_launch_blend_tc(v, rad, dist, st)
                                                  : pv_launch_blend_simt(v->k, rad, dist, st);
  if (e != cudaSuccess) return cuda_fail(e, "blend kernel");
  return PV_OK;
}

pv_status probe_update(pv_volume* v, const void* rad, const void* dist, const float* dirs,
                       void* stream) {
  if (!v || !rad || !dist || !dirs)
    return pv_set_error(PV_ERR_INVALID, "probe_update: NULL argument");
  pv_status s = probe_update_weights(v, dirs, stream);
  if (s != PV_OK) return s;
  return probe_update_blend(v, rad, dist, stream);
}

pv_status probe_select_and_pack(pv_volume* v, pv_frame* out, int32_t want_host_counts, void* stream) {
  if (!v || !out) return pv_set_error(PV_ERR_INVALID, "probe_select_and_pack: NULL argument");
  DeviceGuard g(v->device);
  cudaStream_t st = as_stream(stream);
  pv_wait_downloads(v, st);
  cudaError_t e = pv_launch_select_pack(v->k, st);
  if (e != cudaSuccess) return cuda_fail(e, "select/pack kernel");
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
  if (want_host_counts) {
    e = cudaMemcpyAsync(v->host_counts, v->k.counts, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(v->host_counts + 2, v->k.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "count readback");
    out->count_c = v->host_counts[0];
    out->count_v = v->host_counts[1];
    if (v->host_counts[2]) {
      // reported once: clear the word so that the next frames run normally
      e = cudaMemsetAsync(v->k.err, 0, sizeof(int), st);
      if (e != cudaSuccess) return cuda_fail(e, "error word reset");
      return pv_set_error(PV_ERR_TIMEOUT, "a bounded wait in the blend kernel expired (frame %llu)",
                          (unsigned long long)v->frame);
    }
  }
  return PV_OK;
}

pv_status probe_update_host(pv_volume* v, const void* rad, const void* dist, const float* dirs,
                            void* stream) {
  if (!v || !rad || !dist || !dirs)
    return pv_set_error(PV_ERR_INVALID, "probe_update_host: NULL argument");
  DeviceGuard g(v->device);
  pv_status s = ensure_host_path(v);
  if (s != PV_OK) return s;
  const size_t nr = (size_t)3 * v->k.P * v->k.R * v->op_bytes;
  const size_t nd = (size_t)v->k.P * v->k.R * v->op_bytes;
  const size_t nq = (size_t)3 * v->k.R * sizeof(float);
  cudaStream_t st = as_stream(stream);
  // inside a capture the copies join the captured stream itself
  const bool cap = is_capturing(st);
  const int half = v->stage_next;
  v->stage_next ^= 1;
  char* sr = v->stage + (size_t)half * v->stage_half;
  char* sd = sr + v->stage_off_dist;
  float* sq = (float*)(sr + v->stage_off_dirs);
  cudaStream_t cs = cap ? st : v->s_in;
  cudaError_t e = cap ? cudaSuccess : cudaStreamWaitEvent(cs, v->ev_in_free[half], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sr, rad, nr, cudaMemcpyDefault, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sd, dist, nd, cudaMemcpyDefault, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sq, dirs, nq, cudaMemcpyDefault, cs);
  if (e == cudaSuccess && !cap) e = cudaEventRecord(v->ev_in_done[half], cs);
  if (e == cudaSuccess && !cap) e = cudaStreamWaitEvent(st, v->ev_in_done[half], 0);
  if (e != cudaSuccess) return cuda_fail(e, "input upload");
  s = probe_update(v, sr, sd, sq, stream);
  if (s != PV_OK) return s;
  if (!cap) {
    e = cudaEventRecord(v->ev_in_free[half], st);      // this half may be refilled after the blend
    if (e != cudaSuccess) return cuda_fail(e, "input upload");
  }
  return PV_OK;
}

pv_status probe_frame_download(pv_volume* v, uint16_t* color, uint8_t* vis, uint16_t* delta_c,
                               uint16_t* delta_v, uint32_t* counts, void* stream) {
  if (!v) return pv_set_error(PV_ERR_INVALID, "probe_frame_download: NULL volume");
  DeviceGuard g(v->device);
  cudaStream_t st = as_stream(stream);
  const pv_dev& k = v->k;
  cudaError_t e = cudaMemcpyAsync(v->host_counts, k.counts, 2 * sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && color)
    e = cudaMemcpy2DAsync(color, (size_t)v->cwidth * 2, k.planes_c, k.cpitch, (size_t)v->cwidth * 2,
                          (size_t)3 * k.ch, cudaMemcpyDefault, st);
  if (e == cudaSuccess && vis)
    e = cudaMemcpy2DAsync(vis, (size_t)k.vwidth, k.planes_v, k.vpitch, (size_t)k.vwidth,
                          (size_t)3 * k.vh, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "frame download");
  const uint32_t nc = v->host_counts[0], nv = v->host_counts[1];
  if (delta_c && nc) e = cudaMemcpyAsync(delta_c, k.delta_c, (size_t)nc * 2, cudaMemcpyDefault, st);
  if (e == cudaSuccess && delta_v && nv)
    e = cudaMemcpyAsync(delta_v, k.delta_v, (size_t)nv * 2, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "index download");
  if (counts) {
    counts[0] = nc;
    counts[1] = nv;
  }
  return PV_OK;
}

pv_status probe_frame_download_async(pv_volume* v, uint16_t* color, uint8_t* vis, uint16_t* delta_c,
                                     uint16_t* delta_v, uint32_t* counts, uint64_t* ticket, void* stream) {
  if (!v || !ticket) return pv_set_error(PV_ERR_INVALID, "probe_frame_download_async: NULL argument");
  *ticket = 0;
  DeviceGuard g(v->device);
  cudaStream_t st = as_stream(stream);
  if (is_capturing(st))
    return pv_set_error(PV_ERR_UNSUPPORTED, "probe_frame_download_async: the stream is being captured");
  pv_status s = ensure_host_path(v);
  if (s != PV_OK) return s;
  const pv_dev& k = v->k;
  cudaStream_t so = v->s_out;
  cudaError_t e = cudaEventRecord(v->ev_packed, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(so, v->ev_packed, 0);
  if (e == cudaSuccess && counts) e = cudaMemcpyAsync(counts, k.counts, 2 * sizeof(uint32_t), cudaMemcpyDefault, so);
  if (e == cudaSuccess && color)
    e = cudaMemcpy2DAsync(color, (size_t)v->cwidth * 2, k.planes_c, k.cpitch, (size_t)v->cwidth * 2,
                          (size_t)3 * k.ch, cudaMemcpyDefault, so);
  if (e == cudaSuccess && vis)
    e = cudaMemcpy2DAsync(vis, (size_t)k.vwidth, k.planes_v, k.vpitch, (size_t)k.vwidth, (size_t)3 * k.vh,
                          cudaMemcpyDefault, so);
  if (e == cudaSuccess && delta_c) e = cudaMemcpyAsync(delta_c, k.delta_c, (size_t)k.P * 2, cudaMemcpyDefault, so);
  if (e == cudaSuccess && delta_v) e = cudaMemcpyAsync(delta_v, k.delta_v, (size_t)k.P * 2, cudaMemcpyDefault, so);
  if (e == cudaSuccess) e = cudaEventRecord(v->ev_out[v->dl_seq % PV_DL_RING], so);
  if (e != cudaSuccess) return cuda_fail(e, "frame download");
  *ticket = ++v->dl_seq;
  return PV_OK;
}

pv_status probe_frame_wait(pv_volume* v, uint64_t ticket) {
  if (!v) return pv_set_error(PV_ERR_INVALID, "probe_frame_wait: NULL volume");
  if (ticket == 0 || ticket > v->dl_seq)
    return pv_set_error(PV_ERR_INVALID, "probe_frame_wait: ticket %llu was not issued", (unsigned long long)ticket);
  DeviceGuard g(v->device);
  // a reused event stands for a later download on the same stream, which
  // lands after this one
  const cudaError_t e = cudaEventSynchronize(v->ev_out[(ticket - 1) % PV_DL_RING]);
  if (e != cudaSuccess) return cuda_fail(e, "probe_frame_wait");
  return PV_OK;
}

pv_status probe_volume_export_state(pv_volume* v, void* tiles_c, void* tiles_v, uint16_t* last_c,
                                    uint16_t* last_v, uint64_t* frame, void* stream) {
  if (!v) return pv_set_error(PV_ERR_INVALID, "export: NULL volume");
  DeviceGuard g(v->device);
  cudaStream_t st = as_stream(stream);
  const pv_dev& k = v->k;
  const size_t sb = v->state_bytes;
  const size_t tcc = (size_t)k.tc * k.tc, tvv = (size_t)k.tv * k.tv;
  cudaError_t e = cudaSuccess;
  if (tiles_c)
    e = cudaMemcpy2DAsync(tiles_c, tcc * sb, k.state_c, (size_t)k.sc_stride * sb, tcc * sb,
                          (size_t)3 * k.P, cudaMemcpyDefault, st);
  if (e == cudaSuccess && tiles_v)
    e = cudaMemcpy2DAsync(tiles_v, tvv * sb, k.state_v, (size_t)k.sv_stride * sb, tvv * sb,
                          (size_t)2 * k.P, cudaMemcpyDefault, st);
  if (e == cudaSuccess && last_c)
    e = cudaMemcpy2DAsync(last_c, (size_t)k.Tc * 2, k.last_c, (size_t)k.lc_stride * 2,
                          (size_t)k.Tc * 2, (size_t)3 * k.P, cudaMemcpyDefault, st);
  if (e == cudaSuccess && last_v)
    e = cudaMemcpy2DAsync(last_v, (size_t)k.Tv * 2, k.last_v, (size_t)k.lv_stride * 2,
                          (size_t)k.Tv * 2, (size_t)2 * k.P, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "export");
  if (frame) *frame = v->frame;
  return PV_OK;
}

pv_status probe_volume_import_state(pv_volume* v, const void* tiles_c, const void* tiles_v,
                                    const uint16_t* last_c, const uint16_t* last_v, uint64_t frame,
                                    void* stream) {
  if (!v || !tiles_c || !tiles_v || !last_c || !last_v)
    return pv_set_error(PV_ERR_INVALID, "import: NULL argument");
  DeviceGuard g(v->device);
  cudaStream_t st = as_stream(stream);
  const pv_dev& k = v->k;
  unsigned long long f = frame;
  const size_t sb = v->state_bytes;
  const size_t tcc = (size_t)k.tc * k.tc, tvv = (size_t)k.tv * k.tv;
  cudaError_t e = cudaMemcpy2DAsync(k.state_c, (size_t)k.sc_stride * sb, tiles_c, tcc * sb, tcc * sb,
                                    (size_t)3 * k.P, cudaMemcpyDefault, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(k.state_v, (size_t)k.sv_stride * sb, tiles_v, tvv * sb, tvv * sb,
                          (size_t)2 * k.P, cudaMemcpyDefault, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(k.last_c, (size_t)k.lc_stride * 2, last_c, (size_t)k.Tc * 2,
                          (size_t)k.Tc * 2, (size_t)3 * k.P, cudaMemcpyDefault, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(k.last_v, (size_t)k.lv_stride * 2, last_v, (size_t)k.Tv * 2,
                          (size_t)k.Tv * 2, (size_t)2 * k.P, cudaMemcpyDefault, st);
  static const unsigned long long never = ~0ull;      // imported flags count as fresh
  if (e == cudaSuccess) e = cudaMemcpyAsync(k.frame, &f, sizeof f, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(k.sel_frame, &never, sizeof never, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(k.chg, 0, (size_t)2 * k.chg_words * 4, st);
  if (e == cudaSuccess) e = pv_launch_recompute_flags(k, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "import");
  v->frame = frame;
  return PV_OK;
}

}  // extern "C"
