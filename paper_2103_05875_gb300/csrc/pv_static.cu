// probe_update_static: the per-frame weights and blend (the SIMT blend
// kernel) for callers that cannot allocate device memory, for example code
// that runs where cudaMalloc is unavailable or forbidden (inside a stream
// callback or a graph host node, a plugin that must stay within memory its
// host application owns, or a process whose device memory is managed entirely
// by another allocator). Nothing is allocated: the caller passes every input
// and output buffer, and the only scratch -- this frame's blend weights, their
// sums, the hysteresis and frame words -- lives in the file-scope array below.
//
// The array belongs to the library for the life of the process on every GPU
// that loads it (PV_STATIC_SCRATCH_BYTES of device memory each). All calls on a
// device share it and it keeps the last call's contents, so calls whose work
// overlaps on the GPU (different streams, or several host threads) race and
// must be serialised by the caller. The changed-probe bits are cleared by the
// weights kernel of each call; the frame word is written by each call.
//
// In host code `g_static_scratch` is only a host-side stand-in for the device
// array: its device address is obtained once per device with
// cudaGetSymbolAddress (the first call on a device does this set-up, so that
// first call should come before any stream capture). The address is kept for
// the life of the process, so a device reset (cudaDeviceReset) after the first
// call on that device is not supported.
#include <mutex>

#include "pv_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[PV_STATIC_SCRATCH_BYTES];

__global__ void k_set_frame(unsigned long long* frame, unsigned long long value) { *frame = value; }

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on first use).
pv_status scratch_for_device(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return pv_set_error(PV_ERR_RANGE, "device index %d too large", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess)
      return pv_set_error(PV_ERR_CUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
    e = pv_simt_prepare();
    if (e != cudaSuccess) return pv_set_error(PV_ERR_CUDA, "blend kernel set-up: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = (unsigned char*)ptr;
  }
  *out = g_scratch_ptr[dev];
  return PV_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" pv_status probe_update_static(const pv_desc* d, uint64_t frame, const void* radiance,
                                         const void* dist, const float* dirs, void* tiles_c, void* tiles_v,
                                         const uint16_t* last_c, const uint16_t* last_v,
                                         uint32_t* changed_bits, void* stream) {
  if (!d || !radiance || !dist || !dirs || !tiles_c || !tiles_v || !last_c || !last_v || !changed_bits)
    return pv_set_error(PV_ERR_INVALID, "probe_update_static: NULL argument");
  uint64_t bytes = 0;
  pv_status s = probe_volume_bytes(d, &bytes);   // validates the descriptor; nothing is allocated
  if (s != PV_OK) return s;
  const int P = d->nx * d->ny * d->nz, R = d->rays_per_probe;
  const int nc = d->color_interior, nv = d->vis_interior;
  const int Tc = nc * nc, Tv = nv * nv;
  // scratch: R x T float weights, T float sums, 256 bytes of words, each
  // region rounded up to 256 bytes; the most rays that fit for these texels
  const size_t T = (size_t)(Tc + Tv);
  const size_t w_bytes = align256((size_t)R * T * sizeof(float));
  const size_t room = PV_STATIC_SCRATCH_BYTES - 256 - align256(T * sizeof(float));   // a multiple of 256
  const size_t max_rays = room / (T * sizeof(float));
  if ((size_t)R > max_rays)
    return pv_set_error(PV_ERR_RANGE,
                        "probe_update_static: %d rays per probe exceed %zu, the most the %u-byte scratch array "
                        "holds for %zu texels (n_c^2 + n_v^2)",
                        R, max_rays, (unsigned)PV_STATIC_SCRATCH_BYTES, T);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pv_set_error(PV_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  unsigned char* scratch = nullptr;
  s = scratch_for_device(dev, &scratch);
  if (s != PV_OK) return s;

  pv_dev k{};
  k.P = P; k.R = R; k.nc = nc; k.nv = nv; k.tc = nc + 2; k.tv = nv + 2; k.Tc = Tc; k.Tv = Tv;
  k.bw = d->nx * d->ny; k.bh = d->nz;
  k.state_fmt = d->state_fmt; k.operand_fmt = d->operand_fmt; k.color_code = d->color_code;
  k.color_shift = d->color_lsb ? 0 : 6;
  k.h = d->hysteresis; k.sharpness = d->sharpness;
  k.first_frame_no_hysteresis = d->first_frame_no_hysteresis ? 1 : 0;
  // caller buffers, in the public (unpadded) layouts of include/probe_stream.h
  k.state_c = tiles_c;
  k.state_v = tiles_v;
  k.last_c = const_cast<uint16_t*>(last_c);
  k.last_v = const_cast<uint16_t*>(last_v);
  k.sc_stride = k.tc * k.tc;
  k.sv_stride = k.tv * k.tv;
  k.lc_stride = Tc;
  k.lv_stride = Tv;
  k.chg = changed_bits;
  k.chg_words = (P + 31) / 32;
  // scratch
  k.w_rt = (float*)scratch;
  k.sums = (float*)(scratch + w_bytes);
  k.hy = (float*)(scratch + w_bytes + align256((size_t)(Tc + Tv) * sizeof(float)));
  k.frame = (unsigned long long*)(k.hy + 2);
  k.err = (int*)(k.hy + 4);

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_set_frame<<<1, 1, 0, st>>>(k.frame, (unsigned long long)frame);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = pv_launch_weights(k, dirs, 1, 0, st);
  if (e == cudaSuccess) e = pv_launch_blend_simt(k, radiance, dist, st);
  if (e != cudaSuccess) return pv_set_error(PV_ERR_CUDA, "probe_update_static: %s", cudaGetErrorString(e));
  return PV_OK;
}
