// Client side of Sections 3.3-3.4 of arXiv 2103.05875: a client keeps
// permanent probe textures and applies each packed update to them. Per frame
// it decodes the delta-coded index buffers, unpacks the colour codes from the
// 16-bit Y/U/V planes and the RG16F visibility texels from the three 8-bit
// planes (byte s of an atlas row's stream at plane s mod 3, column s div 3),
// writes each selected probe's interior and rebuilds its octahedral guard band
// (the reflection rule the server applies). Colour values are the exact values
// of the codes (UF10 or UNORM10) in binary32; visibility texels are the
// transmitted binary16 bits.
//
// One kernel: a block owns SLOTS consecutive slots of both textures. It sums
// the deltas before its slots itself (no grid-wide scan), unpacks its slots'
// interiors into shared memory, then writes their whole tiles with coalesced
// stores. Probe ids at or past P and counts past P are ignored, so a damaged
// frame cannot make the kernel write outside the textures.
#include <string.h>

#include "pv_codes.cuh"
#include "pv_internal.h"

struct pv_client {
  pv_desc d;
  pv_geom g;
  int device;
  float* tex_c;      // [3][P][tc*tc] colour values
  uint16_t* tex_v;   // [2][P][tv*tv] visibility texels (binary16 bits)
};

namespace {

constexpr int CA_THREADS = 256;
constexpr int CA_SLOTS = 8;                             // slots per block
constexpr int CA_MAX_T = PV_MAX_INTERIOR * PV_MAX_INTERIOR;

struct CaArgs {
  int P, nc, nv, tc, tv, bw, cheight, cpitch, vheight, vpitch;
  int kind, lsb;
  uint32_t rcp_nc, rcp_nv, rcp_tc, rcp_tv, rcp_tc2, rcp_tv2;
  const uint16_t* planes_c;
  const uint8_t* planes_v;
  const uint16_t* delta_c;
  const uint16_t* delta_v;
  const uint32_t* count_c;
  const uint32_t* count_v;
  float* tex_c;
  uint16_t* tex_v;
};

struct CaShared {
  float vc[CA_SLOTS][3 * CA_MAX_T];      // decoded colour interiors of the block's slots
  uint32_t vv[CA_SLOTS][CA_MAX_T];       // visibility interiors: R | G << 16
  int id_c[CA_SLOTS], id_v[CA_SLOTS];    // probe of each slot, -1 for none
  int bx[CA_SLOTS], by[CA_SLOTS];        // block of each slot in the update texture
  uint32_t red[2 * CA_THREADS / 32];
  uint32_t base_c, base_v;
};

// Sum of delta[0..n) (n a multiple of 8, 16-byte aligned buffer), block-wide.
__device__ __forceinline__ void sum_two(const uint16_t* da, int na, const uint16_t* db, int nb, CaShared& sh) {
  uint32_t sa = 0, sb = 0;
  for (int q = threadIdx.x; q < na / 8; q += CA_THREADS) {
    const uint4 v = reinterpret_cast<const uint4*>(da)[q];
    sa += (v.x & 0xFFFFu) + (v.x >> 16) + (v.y & 0xFFFFu) + (v.y >> 16) + (v.z & 0xFFFFu) + (v.z >> 16) +
          (v.w & 0xFFFFu) + (v.w >> 16);
  }
  for (int q = threadIdx.x; q < nb / 8; q += CA_THREADS) {
    const uint4 v = reinterpret_cast<const uint4*>(db)[q];
    sb += (v.x & 0xFFFFu) + (v.x >> 16) + (v.y & 0xFFFFu) + (v.y >> 16) + (v.z & 0xFFFFu) + (v.z >> 16) +
          (v.w & 0xFFFFu) + (v.w >> 16);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh.red[2 * wid] = sa;
    sh.red[2 * wid + 1] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0, b = 0;
    for (int w = 0; w < CA_THREADS / 32; ++w) {
      a += sh.red[2 * w];
      b += sh.red[2 * w + 1];
    }
    sh.base_c = a;
    sh.base_v = b;
  }
}

__device__ __forceinline__ float color_value(uint32_t code, int kind) {
  if (kind == PV_CODE_UNORM10) return (float)code / 1023.0f;     // correctly rounded
  return __half2float(__ushort_as_half((unsigned short)(code << 5)));   // UF10 is binary16's top bits
}

__global__ void __launch_bounds__(CA_THREADS) k_client_apply(const CaArgs a) {
  __shared__ __align__(16) CaShared sh;
  const int tid = threadIdx.x;
  const int k0 = blockIdx.x * CA_SLOTS;
  const int cnt_c = (int)min(*a.count_c, (uint32_t)a.P), cnt_v = (int)min(*a.count_v, (uint32_t)a.P);
  const int ns_c = max(0, min(CA_SLOTS, cnt_c - k0)), ns_v = max(0, min(CA_SLOTS, cnt_v - k0));
  if (ns_c == 0 && ns_v == 0) return;                   // uniform: the block has no slot
  // probe ids of the block's slots: the deltas before them, then a running sum
  sum_two(a.delta_c, ns_c ? k0 : 0, a.delta_v, ns_v ? k0 : 0, sh);
  if (tid == 0) {
    uint32_t ic = sh.base_c, iv = sh.base_v;
    for (int s = 0; s < CA_SLOTS; ++s) {
      int pc = -1, pv = -1;
      if (s < ns_c) {
        ic += a.delta_c[k0 + s];
        const int id = (int)(ic & 0xFFFFu);
        pc = id < a.P ? id : -1;
      }
      if (s < ns_v) {
        iv += a.delta_v[k0 + s];
        const int id = (int)(iv & 0xFFFFu);
        pv = id < a.P ? id : -1;
      }
      sh.id_c[s] = pc;
      sh.id_v[s] = pv;
      sh.by[s] = (k0 + s) / a.bw;
      sh.bx[s] = (k0 + s) - sh.by[s] * a.bw;
    }
  }
  __syncthreads();

  // colour interiors: items (c, i, slot, j), j fastest, so that a warp reads
  // runs of consecutive samples across neighbouring slots
  {
    const int n = a.nc, T = n * n;
    const uint32_t rcp_ns = ns_c ? (0x80000000u + (uint32_t)ns_c - 1u) / (uint32_t)ns_c : 0u;
    const size_t plane = (size_t)a.cheight * (a.cpitch / 2);
    for (int it = tid; it < ns_c * 3 * T; it += CA_THREADS) {
      const int t = pv::fdiv(it, a.rcp_nc), j = it - t * n;
      const int u = pv::fdiv(t, rcp_ns), s = t - u * ns_c;
      const int c = pv::fdiv(u, a.rcp_nc), i = u - c * n;
      const uint32_t sample =
          a.planes_c[(size_t)c * plane + (size_t)(sh.by[s] * n + i) * (a.cpitch / 2) + sh.bx[s] * n + j];
      const uint32_t code = a.lsb ? (sample & 0x3FFu) : (sample >> 6);
      sh.vc[s][c * T + i * n + j] = color_value(code, a.kind);
    }
  }
  // visibility interiors: texel (slot, i, j) takes stream bytes 4X..4X+3 of
  // its atlas row, X = bx * n + j, byte b from plane b mod 3, column b div 3
  {
    const int n = a.nv, T = n * n;
    const size_t plane = (size_t)a.vheight * a.vpitch;
    for (int it = tid; it < ns_v * T; it += CA_THREADS) {
      const int s = it / T, e = it - s * T;
      const int i = pv::fdiv(e, a.rcp_nv), j = e - i * n;
      const uint8_t* row = a.planes_v + (size_t)(sh.by[s] * n + i) * a.vpitch;
      const int b0 = 4 * (sh.bx[s] * n + j);
      uint32_t v = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int b = b0 + q;
        v |= (uint32_t)row[(size_t)(b % 3) * plane + b / 3] << (8 * q);
      }
      sh.vv[s][e] = v;
    }
  }
  __syncthreads();

  // whole tiles: interior and guard band, consecutive threads on consecutive
  // texels of a tile
  {
    const int n = a.nc, tc = a.tc, tt = tc * tc, T = n * n;
    for (int it = tid; it < ns_c * 3 * tt; it += CA_THREADS) {
      const int t = pv::fdiv(it, a.rcp_tc2), e = it - t * tt;
      const int s = t / 3, c = t - 3 * s;
      const int p = sh.id_c[s];
      if (p < 0) continue;
      const int r = pv::fdiv(e, a.rcp_tc), cc = e - r * tc;
      int sr, sc;
      pv::border_source(r, cc, n, &sr, &sc);
      a.tex_c[((size_t)c * a.P + p) * tt + e] = sh.vc[s][c * T + (sr - 1) * n + (sc - 1)];
    }
  }
  {
    const int n = a.nv, tv = a.tv, tt = tv * tv;
    for (int it = tid; it < ns_v * 2 * tt; it += CA_THREADS) {
      const int t = pv::fdiv(it, a.rcp_tv2), e = it - t * tt;
      const int s = t >> 1, c = t & 1;
      const int p = sh.id_v[s];
      if (p < 0) continue;
      const int r = pv::fdiv(e, a.rcp_tv), cc = e - r * tv;
      int sr, sc;
      pv::border_source(r, cc, n, &sr, &sc);
      const uint32_t v = sh.vv[s][(sr - 1) * n + (sc - 1)];
      a.tex_v[((size_t)c * a.P + p) * tt + e] = (uint16_t)(c ? v >> 16 : v & 0xFFFFu);
    }
  }
}

pv_status cuda_fail(cudaError_t e, const char* what) {
  return pv_set_error(PV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

extern "C" {

pv_status pv_client_create(const pv_desc* d, pv_client** out) {
  if (!out) return pv_set_error(PV_ERR_INVALID, "pv_client_create: NULL out");
  *out = nullptr;
  pv_geom g;
  const pv_status s = pv_frame_geometry(d, &g);
  if (s != PV_OK) return s;
  pv_client* c = new pv_client();
  memset(c, 0, sizeof(pv_client));
  c->d = *d;
  c->g = g;
  cudaGetDevice(&c->device);
  const size_t bc = (size_t)3 * g.P * g.tc * g.tc * sizeof(float), bv = (size_t)2 * g.P * g.tv * g.tv * 2;
  cudaError_t e = cudaMalloc((void**)&c->tex_c, bc);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->tex_v, bv);
  if (e == cudaSuccess) e = cudaMemset(c->tex_c, 0, bc);
  if (e == cudaSuccess) e = cudaMemset(c->tex_v, 0, bv);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(c->tex_c);
    cudaFree(c->tex_v);
    delete c;
    cudaGetLastError();
    return pv_set_error(PV_ERR_OOM, "pv_client_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return PV_OK;
}

pv_status pv_client_destroy(pv_client* c) {
  if (!c) return PV_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  cudaFree(c->tex_c);
  cudaFree(c->tex_v);
  cudaSetDevice(prev);
  delete c;
  return PV_OK;
}

pv_status pv_client_textures(const pv_client* c, float** color, uint16_t** vis) {
  if (!c) return pv_set_error(PV_ERR_INVALID, "pv_client_textures: NULL client");
  if (color) *color = c->tex_c;
  if (vis) *vis = c->tex_v;
  return PV_OK;
}

pv_status pv_client_apply(pv_client* c, const pv_frame* f, void* stream) {
  if (!c || !f) return pv_set_error(PV_ERR_INVALID, "pv_client_apply: NULL argument");
  if (!f->color_planes || !f->vis_planes || !f->delta_c || !f->delta_v || !f->count_c_dev || !f->count_v_dev)
    return pv_set_error(PV_ERR_INVALID, "pv_client_apply: frame lacks planes, deltas or device counts");
  if (((uintptr_t)f->delta_c | (uintptr_t)f->delta_v) & 15u)
    return pv_set_error(PV_ERR_INVALID, "pv_client_apply: delta buffers must be 16-byte aligned");
  const pv_geom& g = c->g;
  CaArgs a;
  a.P = g.P;
  a.nc = g.nc;
  a.nv = g.nv;
  a.tc = g.tc;
  a.tv = g.tv;
  a.bw = g.bw;
  a.cheight = g.cheight;
  a.cpitch = g.cpitch;
  a.vheight = g.vheight;
  a.vpitch = g.vpitch;
  a.kind = c->d.color_code;
  a.lsb = c->d.color_lsb ? 1 : 0;
  a.rcp_nc = pv_rcp31((uint32_t)g.nc);
  a.rcp_nv = pv_rcp31((uint32_t)g.nv);
  a.rcp_tc = pv_rcp31((uint32_t)g.tc);
  a.rcp_tv = pv_rcp31((uint32_t)g.tv);
  a.rcp_tc2 = pv_rcp31((uint32_t)(g.tc * g.tc));
  a.rcp_tv2 = pv_rcp31((uint32_t)(g.tv * g.tv));
  a.planes_c = f->color_planes;
  a.planes_v = f->vis_planes;
  a.delta_c = f->delta_c;
  a.delta_v = f->delta_v;
  a.count_c = f->count_c_dev;
  a.count_v = f->count_v_dev;
  a.tex_c = c->tex_c;
  a.tex_v = c->tex_v;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  const int blocks = (g.P + CA_SLOTS - 1) / CA_SLOTS;
  k_client_apply<<<blocks, CA_THREADS, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (prev != c->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "client apply kernel");
  return PV_OK;
}

}  // extern "C"
