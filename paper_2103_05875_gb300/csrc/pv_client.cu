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
constexpr int CA_SLOTS = 4;                             // slots per block (a power of two, <= 16)

struct CaArgs {
  int P, nc, nv, tc, tv, bw, cheight, cpitch, vheight, vpitch;
  int kind, lsb;
  uint32_t rcp_nc, rcp_nv;
  int vw_c, vw_v;                        // texels per vector store of a colour / visibility tile
  uint32_t rcp_cvec, rcp_vvec;           // ceil(2^31 / vectors per tile)
  const uint16_t* planes_c;
  const uint8_t* planes_v;
  const uint16_t* delta_c;
  const uint16_t* delta_v;
  const uint32_t* count_c;
  const uint32_t* count_v;
  float* tex_c;
  uint16_t* tex_v;
};

// Shared memory sized to the volume's interiors (dynamic, after this struct):
//   float    vc[CA_SLOTS][3][Tc]   decoded colour interiors of the block's slots
//   uint32_t vv[CA_SLOTS][Tv]      visibility interiors: R | G << 16
//   uint16_t src_c[tc*tc], src_v[tv*tv]   per tile position: the interior texel it holds
struct CaShared {
  int id_c[CA_SLOTS], id_v[CA_SLOTS];    // probe of each slot, -1 for none
  uint32_t red[2 * CA_THREADS / 32];
};

size_t ca_dyn_bytes(int nc, int nv) {
  return (size_t)CA_SLOTS * 3 * nc * nc * 4 + (size_t)CA_SLOTS * nv * nv * 4 + (size_t)(nc + 2) * (nc + 2) * 2 +
         (size_t)(nv + 2) * (nv + 2) * 2;
}

// Per-warp partial sums of da[0..na) and db[0..nb) (16-byte aligned buffers;
// eight at a time, then the tail) into sh.red, then a barrier.
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
  for (int q = 8 * (na / 8) + (int)threadIdx.x; q < na; q += CA_THREADS) sa += da[q];
  for (int q = 8 * (nb / 8) + (int)threadIdx.x; q < nb; q += CA_THREADS) sb += db[q];
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
}

// Whole tiles of the block's slots, VW texels per store: vector v of channel
// c of slot s holds tile texels VW*v .. VW*v+VW-1, each the interior texel
// src[e] of the slot's staged values (`get`).
template <int VW, typename V, typename T, typename G>
__device__ __forceinline__ void store_tiles(T* tex, int P, int tt, int nch, int ns, const int* ids,
                                            const uint16_t* src, uint32_t rcp_nvec, G get) {
  const int nvec = tt / VW;
  for (int it = threadIdx.x; it < ns * nch * nvec; it += CA_THREADS) {
    const int t = pv::fdiv(it, rcp_nvec), v = it - t * nvec;
    const int s = t / nch, c = t - s * nch;
    const int p = ids[s];
    if (p < 0) continue;
    union {
      V vec;
      T el[VW];
    } u;
#pragma unroll
    for (int q = 0; q < VW; ++q) u.el[q] = get(s, c, src[VW * v + q]);
    *reinterpret_cast<V*>(tex + ((size_t)c * P + p) * tt + VW * v) = u.vec;
  }
}

__device__ __forceinline__ float color_value(uint32_t code, int kind) {
  if (kind == PV_CODE_UNORM10) return (float)code / 1023.0f;     // correctly rounded
  return __half2float(__ushort_as_half((unsigned short)(code << 5)));   // UF10 is binary16's top bits
}

__global__ void __launch_bounds__(CA_THREADS) k_client_apply(const CaArgs a) {
  __shared__ __align__(16) CaShared sh;
  extern __shared__ __align__(16) uint8_t ca_dyn[];
  const int Tc = a.nc * a.nc, Tv = a.nv * a.nv;
  float* vc = reinterpret_cast<float*>(ca_dyn);
  uint32_t* vv = reinterpret_cast<uint32_t*>(vc + CA_SLOTS * 3 * Tc);
  uint16_t* src_c = reinterpret_cast<uint16_t*>(vv + CA_SLOTS * Tv);
  uint16_t* src_v = src_c + a.tc * a.tc;
  const int tid = threadIdx.x;
  const int k0 = blockIdx.x * CA_SLOTS;
  const int cnt_c = (int)min(*a.count_c, (uint32_t)a.P), cnt_v = (int)min(*a.count_v, (uint32_t)a.P);
  const int ns_c = max(0, min(CA_SLOTS, cnt_c - k0)), ns_v = max(0, min(CA_SLOTS, cnt_v - k0));
  if (ns_c == 0 && ns_v == 0) return;                   // uniform: the block has no slot
  // block of the update texture of the block's first slot; slot s follows
  const int by0 = k0 / a.bw, bx0 = k0 - by0 * a.bw;

  // Everything below up to the barrier is independent: the guard-band tables,
  // the slots' interiors from the planes, and the delta sums for the ids.
  // the guard-band rule as tables: tile position -> interior texel
  for (int e = tid; e < a.tc * a.tc + a.tv * a.tv; e += CA_THREADS) {
    const bool vis = e >= a.tc * a.tc;
    const int t = vis ? a.tv : a.tc, n = vis ? a.nv : a.nc, q = vis ? e - a.tc * a.tc : e;
    const int r = q / t, cc = q - r * t;
    int sr, sc;
    pv::border_source(r, cc, n, &sr, &sc);
    (vis ? src_v : src_c)[q] = (uint16_t)((sr - 1) * n + (sc - 1));
  }
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
      int bx = bx0 + s, by = by0;
      while (bx >= a.bw) {
        bx -= a.bw;
        ++by;
      }
      const uint32_t sample = a.planes_c[(size_t)c * plane + (size_t)(by * n + i) * (a.cpitch / 2) + bx * n + j];
      const uint32_t code = a.lsb ? (sample & 0x3FFu) : (sample >> 6);
      vc[(s * 3 + c) * T + i * n + j] = color_value(code, a.kind);
    }
  }
  // visibility interiors: an atlas row's stream bytes 12w..12w+11 (three
  // texels) are the words at column 4w of the three planes; a thread takes one
  // such chunk of one row of one run of slots within a block row, and keeps
  // the texels that belong to the block's slots
  {
    const int n = a.nv, T = n * n;
    const size_t plane = (size_t)a.vheight * a.vpitch;
    int by = by0, bxs = bx0;                            // block of slot s0
    for (int s0 = 0; s0 < ns_v;) {
      const int s1 = min(ns_v, s0 + (a.bw - bxs));      // the run s0..s1-1 shares a block row
      const int x_lo = n * bxs, x_hi = n * (bxs + (s1 - s0));   // atlas columns of the run
      const int w_lo = (4 * x_lo) / 12, w_hi = (4 * x_hi - 1) / 12;
      const int nw = w_hi - w_lo + 1;
      const uint32_t rcp_nw = (0x80000000u + (uint32_t)nw - 1u) / (uint32_t)nw;
      for (int q = tid; q < n * nw; q += CA_THREADS) {
        const int i = pv::fdiv(q, rcp_nw), w = w_lo + (q - i * nw);
        const uint8_t* row = a.planes_v + (size_t)(by * n + i) * a.vpitch + 4 * (size_t)w;
        const uint32_t p0 = *reinterpret_cast<const uint32_t*>(row);
        const uint32_t p1 = *reinterpret_cast<const uint32_t*>(row + plane);
        const uint32_t p2 = *reinterpret_cast<const uint32_t*>(row + 2 * plane);
        // stream byte 12w + b sits in plane b % 3, byte b / 3 of that word
        const uint32_t t3[3] = {__byte_perm(__byte_perm(p0, p1, 0x1040), p2, 0x3410),
                                __byte_perm(__byte_perm(p1, p2, 0x2051), p0, 0x3610),
                                __byte_perm(__byte_perm(p2, p0, 0x3072), p1, 0x3710)};
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const int X = 3 * w + e;
          if (X >= x_lo && X < x_hi) {
            const int so = pv::fdiv(X - x_lo, a.rcp_nv), j = X - x_lo - so * n;
            vv[(s0 + so) * T + i * n + j] = t3[e];
          }
        }
      }
      s0 = s1;
      bxs = 0;
      ++by;
    }
  }
  // probe ids: the deltas before the block's slots (block sum), and its own
  // slots' deltas (first warp: lanes 0..7 colour, lanes 8..15 visibility)
  uint32_t d = 0;
  if (tid < 2 * CA_SLOTS) {
    const int s = tid & (CA_SLOTS - 1);
    const bool vis = tid >= CA_SLOTS;
    if (s < (vis ? ns_v : ns_c)) d = vis ? a.delta_v[k0 + s] : a.delta_c[k0 + s];
  }
  sum_two(a.delta_c, ns_c ? k0 : 0, a.delta_v, ns_v ? k0 : 0, sh);   // ends in a barrier
  if (tid < 32) {
    const int lane = tid, s = lane & (CA_SLOTS - 1);
    const bool vis = lane >= CA_SLOTS;
    const int ns = vis ? ns_v : ns_c;
    uint32_t base_c = 0, base_v = 0;
    for (int w = 0; w < CA_THREADS / 32; ++w) {
      base_c += sh.red[2 * w];
      base_v += sh.red[2 * w + 1];
    }
#pragma unroll
    for (int o = 1; o < CA_SLOTS; o <<= 1) {            // inclusive prefix within each group of slots
      const uint32_t t = __shfl_up_sync(0xffffffffu, d, o);
      if (s >= o) d += t;
    }
    if (lane < 2 * CA_SLOTS) {
      const int id = (int)(((vis ? base_v : base_c) + d) & 0xFFFFu);
      const int p = (s < ns && id < a.P) ? id : -1;
      if (vis) sh.id_v[s] = p;
      else sh.id_c[s] = p;
    }
  }
  __syncthreads();

  // whole tiles: interior and guard band, vector stores along each tile
  {
    const int T = a.nc * a.nc;
    const auto get = [&](int s, int c, int e) { return vc[(s * 3 + c) * T + e]; };
    const int tt = a.tc * a.tc;
    if (a.vw_c == 4) store_tiles<4, float4>(a.tex_c, a.P, tt, 3, ns_c, sh.id_c, src_c, a.rcp_cvec, get);
    else if (a.vw_c == 2) store_tiles<2, float2>(a.tex_c, a.P, tt, 3, ns_c, sh.id_c, src_c, a.rcp_cvec, get);
    else store_tiles<1, float>(a.tex_c, a.P, tt, 3, ns_c, sh.id_c, src_c, a.rcp_cvec, get);
  }
  {
    const auto get = [&](int s, int c, int e) {
      const uint32_t v = vv[s * Tv + e];
      return (uint16_t)(c ? v >> 16 : v & 0xFFFFu);
    };
    const int tt = a.tv * a.tv;
    if (a.vw_v == 8) store_tiles<8, uint4>(a.tex_v, a.P, tt, 2, ns_v, sh.id_v, src_v, a.rcp_vvec, get);
    else if (a.vw_v == 4) store_tiles<4, uint2>(a.tex_v, a.P, tt, 2, ns_v, sh.id_v, src_v, a.rcp_vvec, get);
    else if (a.vw_v == 2) store_tiles<2, uint32_t>(a.tex_v, a.P, tt, 2, ns_v, sh.id_v, src_v, a.rcp_vvec, get);
    else store_tiles<1, uint16_t>(a.tex_v, a.P, tt, 2, ns_v, sh.id_v, src_v, a.rcp_vvec, get);
  }
}

using pv_host::cuda_fail;

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
  pv_host::DeviceGuard guard(c->device);
  cudaFree(c->tex_c);
  cudaFree(c->tex_v);
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
  // the kernel reads 32-bit words of the visibility rows, 16-bit colour samples and 32-bit counts
  if (((uintptr_t)f->vis_planes & 3u) || ((uintptr_t)f->color_planes & 1u) ||
      (((uintptr_t)f->count_c_dev | (uintptr_t)f->count_v_dev) & 3u))
    return pv_set_error(PV_ERR_INVALID, "pv_client_apply: misaligned planes or counts");
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
  // widest vector store that divides a tile (the textures are 16-byte aligned)
  const int ttc = g.tc * g.tc, ttv = g.tv * g.tv;
  a.vw_c = ttc % 4 == 0 ? 4 : (ttc % 2 == 0 ? 2 : 1);
  a.vw_v = ttv % 8 == 0 ? 8 : (ttv % 4 == 0 ? 4 : (ttv % 2 == 0 ? 2 : 1));
  a.rcp_cvec = pv_rcp31((uint32_t)(ttc / a.vw_c));
  a.rcp_vvec = pv_rcp31((uint32_t)(ttv / a.vw_v));
  a.planes_c = f->color_planes;
  a.planes_v = f->vis_planes;
  a.delta_c = f->delta_c;
  a.delta_v = f->delta_v;
  a.count_c = f->count_c_dev;
  a.count_v = f->count_v_dev;
  a.tex_c = c->tex_c;
  a.tex_v = c->tex_v;
  pv_host::DeviceGuard guard(c->device);
  const int blocks = (g.P + CA_SLOTS - 1) / CA_SLOTS;
  k_client_apply<<<blocks, CA_THREADS, ca_dyn_bytes(g.nc, g.nv), reinterpret_cast<cudaStream_t>(stream)>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "client apply kernel");
  return PV_OK;
}

}  // extern "C"
