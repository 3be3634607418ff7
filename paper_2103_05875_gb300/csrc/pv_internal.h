// Internal definitions shared by the host API and the kernels of the probe
// streaming library. Not part of the public ABI (see include/probe_stream.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/probe_stream.h"

#define PV_SENTINEL 0xFFFFu   // last-transmitted code of a probe never sent

// Everything a kernel needs to know about a volume, passed by value.
struct pv_dev {
  int P, R, nc, nv, tc, tv, Tc, Tv;     // probes, rays, interiors, tiles, texels per tile
  int bw, bh;                           // update-texture block grid
  int cpitch, ch;                       // colour plane pitch (bytes) and height
  int vpitch, vh, vwidth;               // visibility plane pitch (bytes), height, width x'
  int state_fmt, operand_fmt, color_code, color_shift;
  float h, sharpness;
  int first_frame_no_hysteresis;
  void* state_c;                        // [3][P][sc_stride], tile tc x tc at the start of each stride
  void* state_v;                        // [2][P][sv_stride]
  uint16_t* last_c;                     // [3][P][lc_stride], first Tc codes used
  uint16_t* last_v;                     // [2][P][lv_stride]
  uint16_t* cur_c;                      // [3][P][lc_stride]: transmitted codes of the current texels
  uint16_t* cur_v;                      // [2][P][lv_stride] (written by the blend; NULL: not kept)
  uint32_t* chg;                        // [2][chg_words]: changed-probe bits, colour then
                                        // visibility, bit p%32 of word p/32
  int chg_words;                        // words per texture: ceil(P / 32)
  float* w_rt;                          // [R][Tc + Tv] weights, ray-major (SIMT blend)
  float* sums;                          // [Tc + Tv] weight sums
  void* w_op;                           // weights in the operand format for the tensor-core blend, as
                                        // shared-memory tile images: [planes][w_chunks][w_rows x w_rb
                                        // bytes] (F16 one plane; BF16 and F32 hi and lo planes); see
                                        // pv_w_image_offset
  float* hy;                            // [1] hysteresis of the frame being blended
  unsigned long long* frame;            // [1] device frame counter
  uint16_t* idx_c;                      // [P]
  uint16_t* idx_v;
  uint16_t* delta_c;
  uint16_t* delta_v;
  uint32_t* counts;                     // [2]: count_c, count_v of the last packed frame
  uint32_t* sel;                        // [8]: select sequence, finished-CTA ticket, counts
                                        // history by sequence parity ([2 + 2*par] c, [3 + 2*par] v)
  unsigned long long* sel_frame;        // [1]: frame counter value at the last select
  uint16_t* planes_c;                   // 3 planes of ch rows x cpitch bytes
  uint8_t* planes_v;                    // 3 planes of vh rows x vpitch bytes
  int w_rows, w_rb, w_kc, w_vb, w_chunks;   // w_op images: rows (visibility texels from row 0,
                                        // colour texels from row w_vb), bytes per row, rays per chunk,
                                        // chunks per plane
  int sc_stride, sv_stride;             // elements per probe tile in state memory (16-byte multiple)
  int lc_stride, lv_stride;             // codes per probe in the last-transmitted arrays (multiple of 8)
  // ceil(2^31 / d) for d = n_c, n_v, lc_stride / 8, lv_stride / 8: the
  // select kernel divides small indices by them with one multiply (pv_rcp31)
  uint32_t rcp_nc, rcp_nv, rcp_vc, rcp_vv;
  int* err;                             // [1] device error word (non-zero: a bounded wait gave up)
};

constexpr int PV_DL_RING = 8;          // download events kept per volume

struct pv_volume {
  pv_desc d;
  pv_dev k;
  int device;
  int kernel;
  int state_bytes, op_bytes;
  int cwidth;                           // colour plane width in samples
  char* base;                           // single device allocation
  size_t bytes;
  // host-buffer path: two halves of input staging, each filled on s_in while
  // the other feeds the blend, and frame downloads on s_out
  char* stage;                          // 2 x (radiance | dist | dirs)
  size_t stage_half, stage_off_dist, stage_off_dirs;
  int stage_next;
  cudaStream_t s_in, s_out;
  cudaEvent_t ev_in_done[2], ev_in_free[2], ev_packed;
  cudaEvent_t ev_out[PV_DL_RING];       // download tickets, reused round robin
  unsigned long long dl_seq;            // downloads queued so far
  uint32_t* host_counts;                // pinned [4]
  unsigned long long frame;             // host mirror of the frame counter
  void* tc_plan;                        // tensor-core kernel plan (tensor maps), or NULL
};

// Frame geometry of a volume description (the same for the server volume and
// for a client that decodes its frames): PV_OK, or the validation error.
struct pv_geom {
  int P, nc, nv, tc, tv, bw, bh;
  int cheight, cpitch;                  // colour plane rows, row bytes
  int vheight, vpitch, vwidth;          // visibility plane rows, row bytes, stream bytes per row
};
pv_status pv_frame_geometry(const pv_desc* d, pv_geom* g);

// ceil(2^31 / d); x / d == umulhi(2x, ceil(2^31 / d)) for 0 <= x < 2^16 and
// 1 <= d <= 2^15 (the rounding excess x * (m - 2^31 / d) / 2^31 stays below 1/d).
inline uint32_t pv_rcp31(uint32_t d) { return (uint32_t)(((1ull << 31) + d - 1) / d); }

// Makes `st` wait for the volume's last queued frame download (the next
// select rewrites what it reads).
void pv_wait_downloads(pv_volume* v, cudaStream_t st);

// Byte offset of ray r of image row `row` in one plane of w_op. Each chunk of
// w_kc rays is a w_rows x w_rb tile with the 16-byte units of a row XORed by
// address bits 7.. (the SWIZZLE_32B / SWIZZLE_64B shared-memory layouts the
// tensor-core blend's MMA descriptors read), so a chunk moves into shared
// memory with one bulk copy.
__host__ __device__ inline size_t pv_w_image_offset(const pv_dev& k, int row, int r, int elem_bytes) {
  const int chunk = r / k.w_kc, kk = r - chunk * k.w_kc;
  const uint32_t o = (uint32_t)(row * k.w_rb + kk * elem_bytes);
  const uint32_t m = (uint32_t)(k.w_rb / 16 - 1);
  return (size_t)chunk * k.w_rows * k.w_rb + (o ^ (((o >> 7) & m) << 4));
}

// Programmatic dependent launch: a kernel launched with
// pv_pdl_attr may start while its predecessor in the stream is still running;
// it lets its own successor start early (pv_grid_launch_dependents) and must
// call pv_grid_wait before it reads anything the predecessor (or anything
// before it) wrote. Both are no-ops for a kernel launched without the attribute.
#ifdef __CUDACC__
__device__ __forceinline__ void pv_grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pv_grid_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif
inline cudaLaunchAttribute pv_pdl_attr() {
  cudaLaunchAttribute a;
  a.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  a.val.programmaticStreamSerializationAllowed = 1;
  return a;
}

// ---------------------------------------------------------------- launchers
cudaError_t pv_launch_weights(const pv_dev& k, const float* dirs, int want_rt, int want_op,
                              cudaStream_t s);
cudaError_t pv_simt_prepare();
cudaError_t pv_launch_blend_simt(const pv_dev& k, const void* rad, const void* dist,
                                 cudaStream_t s);
cudaError_t pv_launch_select_pack(const pv_dev& k, cudaStream_t s);
// batched forms (blockIdx.y = volume; n <= PV_MAX_BATCH)
cudaError_t pv_launch_weights_batch(const pv_dev* ks, const float* const* dirs, int n, int want_rt, int want_op,
                                    cudaStream_t s);
cudaError_t pv_launch_select_pack_batch(const pv_dev* ks, int n, cudaStream_t s);
cudaError_t pv_launch_recompute_flags(const pv_dev& k, cudaStream_t s);

// tensor-core blend (pv_blend_tc.cu)
bool pv_tc_supported(const pv_desc* d, const char** why);
cudaError_t pv_tc_plan_create(pv_volume* v);
void pv_tc_plan_destroy(pv_volume* v);
cudaError_t pv_launch_blend_tc(pv_volume* v, const void* rad, const void* dist, cudaStream_t s);
// one persistent launch over the work items of several volumes of equal shapes
struct pv_tc_batch;
// Plan knobs of the batched tensor-core blend (0 = the default choice):
// probes per work item, ray / weight ring depths (upper bounds; shared
// memory may give fewer), F32 TMEM A stages, CTAs (at most one per SM).
struct pv_tc_opts {
  int probes_per_item, ray_stages, weight_stages, tmem_stages, ctas;
};
cudaError_t pv_tc_batch_create(pv_volume* const* vols, int n, int np_want, pv_tc_batch** out);
cudaError_t pv_tc_batch_create_opts(pv_volume* const* vols, int n, const pv_tc_opts* opts, pv_tc_batch** out);
void pv_tc_batch_config(const pv_tc_batch* b, pv_tc_opts* out);
void pv_tc_batch_destroy(pv_tc_batch* b);
int pv_tc_batch_np(const pv_tc_batch* b);
cudaError_t pv_tc_batch_launch(pv_tc_batch* b, const void* const* rad, const void* const* dist, cudaStream_t s);

// error reporting (pv_api.cpp)
pv_status pv_set_error(pv_status s, const char* fmt, ...);

// Host helpers shared by the API files.
namespace pv_host {
// Makes `dev` current for the guard's lifetime, then restores the caller's device.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};
// PV_ERR_CUDA with the message "what: CUDA error string".
inline pv_status cuda_fail(cudaError_t e, const char* what) {
  return pv_set_error(PV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}
inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }
inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
}  // namespace pv_host
