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
// One kernel: a block owns SLOTS consecutive slots of both textures, one warp
// per slot. The block stages the guard-band tables (built once per client)
// and the deltas before its first slot with asynchronous copies and sums the
// deltas itself (no grid-wide scan); meanwhile each warp reads its slot's
// colour samples and visibility chunks in one batch and decodes them into its
// own shared memory. After the ids are known, each warp writes its slot's
// whole tiles with vector stores. Slots past the frame's counts are decoded
// too (they lie inside the planes) and dropped; deltas are read only below the
// counts. Probe ids at or past P and
// counts past P are ignored, so a damaged frame cannot make the kernel write
// outside the textures.
#include <string.h>

#include <vector>

#include "pv_codes.cuh"
#include "pv_internal.h"

struct pv_client {
  pv_desc d;
  pv_geom g;
  int device;
  float* tex_c;      // [3][P][tc*tc] colour values
  uint16_t* tex_v;   // [2][P][tv*tv] visibility texels (binary16 bits)
  uint16_t* src;     // guard-band tables: per colour then visibility tile position, the interior texel it holds
  int src_voff;      // the visibility table's first entry (a 16-byte boundary)
  int src_q;         // their size in 16-byte words
};

namespace {

constexpr int CA_WARPS = 8;
constexpr int CA_THREADS = 32 * CA_WARPS;
constexpr int CA_SLOTS = CA_WARPS;                      // slots per block: one per warp
constexpr int CA_BATCH = 2;                             // 16-byte delta words a thread stages
constexpr int CA_CB = 4;                                // colour samples a lane loads at once
constexpr int CA_VB = 3;                                // visibility chunks a lane loads at once

struct CaArgs {
  int P, nc, nv, tc, tv, bw, crow, vpitch;
  size_t cplane, vplane;                 // plane sizes: colour in samples, visibility in bytes
  int kind, lsb;
  uint32_t rcp_nc, rcp_Tc;
  int kv;                                // 12-byte visibility chunks a slot's row can touch
  uint32_t rcp_kv;
  int vw_c, vw_v;                        // texels per vector store of a colour / visibility tile
  uint32_t rcp_cvec;                     // ceil(2^31 / vectors per colour tile channel)
  const uint16_t* planes_c;
  const uint8_t* planes_v;
  const uint16_t* delta_c;
  const uint16_t* delta_v;
  const uint32_t* count_c;
  const uint32_t* count_v;
  const uint16_t* src;                   // guard-band tables, src_q 16-byte words, visibility from src_voff
  int src_q, src_voff;
  uint32_t off_src, off_warp, warp_bytes;   // dynamic shared memory layout (CaDyn)
  float* tex_c;
  uint16_t* tex_v;
};

// Dynamic shared memory, byte offsets of:
//   uint4    dq[CA_BATCH][2][CA_THREADS]  the first 16-byte delta words each thread sums
//   uint16_t src_c[tc*tc], src_v[tv*tv]   per tile position: the interior texel it holds
//                                         (src_v on a 16-byte boundary; copied in whole
//                                         16-byte words)
//   per warp: float vc[3][Tc], uint32_t vv[Tv]   its slot's decoded colour interior and
//                                         visibility interior (R | G << 16)
struct CaDyn {
  uint32_t src, warp, warp_bytes, bytes;
};

inline CaDyn ca_dyn_layout(int nc, int nv, int src_q) {
  const auto up16 = [](uint32_t x) { return (x + 15u) & ~15u; };
  CaDyn L;
  L.src = CA_BATCH * 2 * CA_THREADS * 16;
  L.warp = L.src + src_q * 16;
  L.warp_bytes = up16((3 * nc * nc + nv * nv) * 4);
  L.bytes = L.warp + CA_WARPS * L.warp_bytes;
  return L;
}

struct CaShared {
  int id_c[CA_SLOTS], id_v[CA_SLOTS];    // probe of each slot, -1 for none
  uint32_t red[2 * CA_WARPS];
};

// Adds the eight 16-bit deltas of a 16-byte word to acc (each dp2a adds both
// halves of a 32-bit word); ids are taken modulo 2^16, so wrap-around of acc
// is harmless.
__device__ __forceinline__ uint32_t sum16(uint32_t acc, uint4 v) {
  const uint32_t a0 = __dp2a_lo(v.x, 0x0101u, __dp2a_lo(v.y, 0x0101u, acc));
  const uint32_t a1 = __dp2a_lo(v.z, 0x0101u, __dp2a_lo(v.w, 0x0101u, 0u));
  return a0 + a1;
}

__device__ __forceinline__ float color_value(uint32_t code, int kind) {
  if (kind == PV_CODE_UNORM10) return (float)code / 1023.0f;     // correctly rounded
  return __half2float(__ushort_as_half((unsigned short)(code << 5)));   // UF10 is binary16's top bits
}

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned),
// and the wait for every copy the thread issued.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// VW consecutive table entries (VW * 2 bytes, aligned to that size).
template <int VW>
__device__ __forceinline__ void load_src(const uint16_t* src, int e, uint16_t (&out)[VW]) {
  if constexpr (VW == 8) {
    const uint4 q = *reinterpret_cast<const uint4*>(src + e);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      out[2 * k] = (uint16_t)(w[k] & 0xFFFFu);
      out[2 * k + 1] = (uint16_t)(w[k] >> 16);
    }
  } else if constexpr (VW == 4) {
    const uint2 q = *reinterpret_cast<const uint2*>(src + e);
    out[0] = (uint16_t)(q.x & 0xFFFFu);
    out[1] = (uint16_t)(q.x >> 16);
    out[2] = (uint16_t)(q.y & 0xFFFFu);
    out[3] = (uint16_t)(q.y >> 16);
  } else {
#pragma unroll
    for (int k = 0; k < VW; ++k) out[k] = src[e + k];
  }
}

// The colour tiles of probe p (three channels), VW texels per store, by the
// warp: vector v of channel c holds tile texels VW*q .. VW*q+VW-1.
template <int VW, typename V>
__device__ __forceinline__ void store_color(float* tex, int P, int p, int tt, const uint16_t* src, const float* vc,
                                            int T, uint32_t rcp_nvec, int lane) {
  const int nvec = tt / VW;
  for (int v = lane; v < 3 * nvec; v += 32) {
    const int c = pv::fdiv(v, rcp_nvec), q = v - c * nvec;
    uint16_t e[VW];
    load_src<VW>(src, VW * q, e);
    union {
      V vec;
      float el[VW];
    } u;
#pragma unroll
    for (int k = 0; k < VW; ++k) u.el[k] = vc[c * T + e[k]];
    *reinterpret_cast<V*>(tex + ((size_t)c * P + p) * tt + VW * q) = u.vec;
  }
}

// The visibility tiles of probe p (R and G from the same interior word), VW
// texels per store, by the warp.
template <int VW, typename V>
__device__ __forceinline__ void store_vis(uint16_t* tex, int P, int p, int tt, const uint16_t* src,
                                          const uint32_t* vv, int lane) {
  const int nvec = tt / VW;
  for (int v = lane; v < nvec; v += 32) {
    uint16_t e[VW];
    load_src<VW>(src, VW * v, e);
    union {
      V vec;
      uint16_t el[VW];
    } r, g;
#pragma unroll
    for (int k = 0; k < VW; ++k) {
      const uint32_t w = vv[e[k]];
      r.el[k] = (uint16_t)(w & 0xFFFFu);
      g.el[k] = (uint16_t)(w >> 16);
    }
    *reinterpret_cast<V*>(tex + (size_t)p * tt + VW * v) = r.vec;
    *reinterpret_cast<V*>(tex + ((size_t)P + p) * tt + VW * v) = g.vec;
  }
}

__global__ void __launch_bounds__(CA_THREADS) k_client_apply(const CaArgs a) {
  __shared__ __align__(16) CaShared sh;
  extern __shared__ __align__(16) uint8_t ca_dyn[];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n_c = a.nc, n_v = a.nv, Tc = n_c * n_c;
  uint4* dq = reinterpret_cast<uint4*>(ca_dyn);
  uint16_t* src_c = reinterpret_cast<uint16_t*>(ca_dyn + a.off_src);
  uint16_t* src_v = src_c + a.src_voff;
  float* vc = reinterpret_cast<float*>(ca_dyn + a.off_warp + wid * a.warp_bytes);
  uint32_t* vv = reinterpret_cast<uint32_t*>(vc + 3 * Tc);
  const int k0 = blockIdx.x * CA_SLOTS;
  const int nsl = min(CA_SLOTS, a.P - k0);             // the block's slots inside the volume
  const int slot = k0 + wid;                           // the warp's slot
  const int by = slot / a.bw, bx = slot - by * a.bw;  // its block of the update textures

  // ---- the warp's slot (inside the volume; past the frame's counts it is
  // decoded and dropped): its colour samples and visibility chunks, CA_CB /
  // CA_VB per lane at once; the first batch of each is loaded before anything
  // waits, then decoded into the warp's shared memory
  const bool live = wid < nsl;
  // colour: sample it = (c*n + i)*n + j of the slot, which is its place in vc
  const uint16_t* pc = a.planes_c + (size_t)by * n_c * a.crow + (size_t)bx * n_c;
  const auto load_c = [&](int b0, uint32_t(&smp)[CA_CB]) {
#pragma unroll
    for (int u = 0; u < CA_CB; ++u) {
      const int it = b0 + lane + 32 * u;
      smp[u] = 0;
      if (it < 3 * Tc) {
        const int c = pv::fdiv(it, a.rcp_Tc), r = it - c * Tc;
        const int i = pv::fdiv(r, a.rcp_nc), j = r - i * n_c;
        smp[u] = pc[c * a.cplane + (size_t)i * a.crow + j];
      }
    }
  };
  const auto put_c = [&](int b0, const uint32_t(&smp)[CA_CB]) {
#pragma unroll
    for (int u = 0; u < CA_CB; ++u) {
      const int it = b0 + lane + 32 * u;
      if (it < 3 * Tc) vc[it] = color_value(a.lsb ? (smp[u] & 0x3FFu) : (smp[u] >> 6), a.kind);
    }
  };
  // visibility: chunk k of row i, the atlas row's stream bytes 12w..12w+11
  // (texels 3w..3w+2, w = w0 + k), which are the words at column 4w of the
  // three planes; stream byte 12w + b sits in plane b % 3, byte b / 3 of that
  // word. Texels outside the slot's row are dropped.
  const int xs = n_v * bx, w0 = xs / 3, nk = (4 * (xs + n_v) - 1) / 12 - w0 + 1;
  const uint8_t* pw = a.planes_v + (size_t)by * n_v * a.vpitch + 4 * (size_t)w0;
  const auto load_v = [&](int b0, uint32_t(&wv)[CA_VB][3]) {
#pragma unroll
    for (int u = 0; u < CA_VB; ++u) {
      const int it = b0 + lane + 32 * u;
      const int i = pv::fdiv(it, a.rcp_kv), k = it - i * a.kv;
      wv[u][0] = wv[u][1] = wv[u][2] = 0;
      if (it < n_v * a.kv && k < nk) {
        const uint32_t* w = reinterpret_cast<const uint32_t*>(pw + (size_t)i * a.vpitch + 4 * k);
        wv[u][0] = w[0];
        wv[u][1] = w[a.vplane / 4];
        wv[u][2] = w[a.vplane / 2];
      }
    }
  };
  const auto put_v = [&](int b0, const uint32_t(&wv)[CA_VB][3]) {
#pragma unroll
    for (int u = 0; u < CA_VB; ++u) {
      const int it = b0 + lane + 32 * u;
      const int i = pv::fdiv(it, a.rcp_kv), k = it - i * a.kv;
      if (it < n_v * a.kv && k < nk) {
        const uint32_t p0 = wv[u][0], p1 = wv[u][1], p2 = wv[u][2];
        const uint32_t t3[3] = {__byte_perm(__byte_perm(p0, p1, 0x1040), p2, 0x3410),
                                __byte_perm(__byte_perm(p1, p2, 0x2051), p0, 0x3610),
                                __byte_perm(__byte_perm(p2, p0, 0x3072), p1, 0x3710)};
        const int x = 3 * (w0 + k) - xs;               // texel 3w relative to the slot's first
#pragma unroll
        for (int e = 0; e < 3; ++e)
          if (x + e >= 0 && x + e < n_v) vv[i * n_v + x + e] = t3[e];
      }
    }
  };
  uint32_t smp[CA_CB], wv[CA_VB][3];
  if (live) {
    load_c(0, smp);
    load_v(0, wv);
  }

  // ---- block-wide: the tables, the counts, then only the deltas the frame
  // holds: those before the block's first slot when that slot is below the
  // count (in 16-byte words, the first CA_BATCH of each thread staged in dq,
  // where only that thread reads them, and a tail) and the block's own below
  // the count (first warp: lanes 0..SLOTS-1 colour, then visibility)
  for (int q = tid; q < a.src_q; q += CA_THREADS) cp_async16(src_c + 8 * q, a.src + 8 * q);
  const int cnt_c = (int)min(*a.count_c, (uint32_t)a.P), cnt_v = (int)min(*a.count_v, (uint32_t)a.P);
  const int ns_c = max(0, min(nsl, cnt_c - k0)), ns_v = max(0, min(nsl, cnt_v - k0));
  const int na_c = ns_c > 0 ? k0 : 0, na_v = ns_v > 0 ? k0 : 0;
  const int nq_c = na_c >> 3, nq_v = na_v >> 3;
  const uint4* dc4 = reinterpret_cast<const uint4*>(a.delta_c);
  const uint4* dv4 = reinterpret_cast<const uint4*>(a.delta_v);
#pragma unroll
  for (int u = 0; u < CA_BATCH; ++u) {
    const int q = tid + u * CA_THREADS;
    if (q < nq_c) cp_async16(dq + (2 * u) * CA_THREADS + tid, dc4 + q);
    if (q < nq_v) cp_async16(dq + (2 * u + 1) * CA_THREADS + tid, dv4 + q);
  }
  uint32_t sum_c = 0, sum_v = 0, d = 0;
  if (tid < (na_c & 7)) sum_c = a.delta_c[8 * nq_c + tid];
  if (tid < (na_v & 7)) sum_v = a.delta_v[8 * nq_v + tid];
  if (tid < 2 * CA_SLOTS) {
    const int s = tid & (CA_SLOTS - 1);
    const bool vis = tid >= CA_SLOTS;
    if (s < (vis ? ns_v : ns_c)) d = vis ? a.delta_v[k0 + s] : a.delta_c[k0 + s];
  }

  // ---- decode: the first batches, then any further ones one at a time
  if (live) {
    put_c(0, smp);
    for (int b0 = 32 * CA_CB; b0 < 3 * Tc; b0 += 32 * CA_CB) {
      uint32_t t[CA_CB];
      load_c(b0, t);
      put_c(b0, t);
    }
    put_v(0, wv);
    for (int b0 = 32 * CA_VB; b0 < n_v * a.kv; b0 += 32 * CA_VB) {
      uint32_t t[CA_VB][3];
      load_v(b0, t);
      put_v(b0, t);
    }
  }

  // ---- delta sums modulo 2^16, one partial per warp
  cp_async_wait_all();
#pragma unroll
  for (int u = 0; u < CA_BATCH; ++u) {
    const int q = tid + u * CA_THREADS;
    if (q < nq_c) sum_c = sum16(sum_c, dq[(2 * u) * CA_THREADS + tid]);
    if (q < nq_v) sum_v = sum16(sum_v, dq[(2 * u + 1) * CA_THREADS + tid]);
  }
  for (int q = tid + CA_BATCH * CA_THREADS; q < nq_c; q += CA_THREADS) sum_c = sum16(sum_c, dc4[q]);
  for (int q = tid + CA_BATCH * CA_THREADS; q < nq_v; q += CA_THREADS) sum_v = sum16(sum_v, dv4[q]);
  sum_c = __reduce_add_sync(0xffffffffu, sum_c);
  sum_v = __reduce_add_sync(0xffffffffu, sum_v);
  if (ns_c == 0 && ns_v == 0) return;                   // uniform: the block has no slot in the frame
  if (lane == 0) {
    sh.red[2 * wid] = sum_c;
    sh.red[2 * wid + 1] = sum_v;
  }
  __syncthreads();

  // ---- probe ids: the deltas before the block's slots plus the inclusive
  // prefix of its own
  if (wid == 0) {
    const int s = lane & (CA_SLOTS - 1);
    const bool vis = lane >= CA_SLOTS;
    const int ns = vis ? ns_v : ns_c;
    uint32_t base_c = 0, base_v = 0;
#pragma unroll
    for (int w = 0; w < CA_WARPS; ++w) {
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

  // ---- the warp's tiles: interior and guard band, vector stores along each tile
  const int p_c = sh.id_c[wid], p_v = sh.id_v[wid];
  if (p_c >= 0) {
    const int tt = a.tc * a.tc;
    if (a.vw_c == 4) store_color<4, float4>(a.tex_c, a.P, p_c, tt, src_c, vc, Tc, a.rcp_cvec, lane);
    else if (a.vw_c == 2) store_color<2, float2>(a.tex_c, a.P, p_c, tt, src_c, vc, Tc, a.rcp_cvec, lane);
    else store_color<1, float>(a.tex_c, a.P, p_c, tt, src_c, vc, Tc, a.rcp_cvec, lane);
  }
  if (p_v >= 0) {
    const int tt = a.tv * a.tv;
    if (a.vw_v == 8) store_vis<8, uint4>(a.tex_v, a.P, p_v, tt, src_v, vv, lane);
    else if (a.vw_v == 4) store_vis<4, uint2>(a.tex_v, a.P, p_v, tt, src_v, vv, lane);
    else if (a.vw_v == 2) store_vis<2, uint32_t>(a.tex_v, a.P, p_v, tt, src_v, vv, lane);
    else store_vis<1, uint16_t>(a.tex_v, a.P, p_v, tt, src_v, vv, lane);
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
  // the guard-band rule of the two tile sizes as tables: tile position -> interior texel
  // (the visibility table from the first 16-byte boundary after the colour table)
  c->src_voff = (g.tc * g.tc + 7) / 8 * 8;
  c->src_q = (c->src_voff + g.tv * g.tv + 7) / 8;
  std::vector<uint16_t> tab((size_t)c->src_q * 8, 0);
  for (int vis = 0; vis < 2; ++vis) {
    const int t = vis ? g.tv : g.tc, n = vis ? g.nv : g.nc;
    for (int q = 0; q < t * t; ++q) {
      int sr, sc;
      pv::border_source(q / t, q % t, n, &sr, &sc);
      tab[(vis ? c->src_voff : 0) + q] = (uint16_t)((sr - 1) * n + (sc - 1));
    }
  }
  // the decode's shared memory can pass the 48 KB a launch gets by default
  // (up to about 50 KB for 16x16 interiors): raise the kernel's limit to it
  const uint32_t dyn = ca_dyn_layout(g.nc, g.nv, c->src_q).bytes;
  cudaError_t e = dyn > 48u * 1024u
                      ? cudaFuncSetAttribute(k_client_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)
                      : cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->tex_c, bc);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->tex_v, bv);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->src, tab.size() * 2);
  if (e == cudaSuccess) e = cudaMemcpy(c->src, tab.data(), tab.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->tex_c, 0, bc);
  if (e == cudaSuccess) e = cudaMemset(c->tex_v, 0, bv);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(c->tex_c);
    cudaFree(c->tex_v);
    cudaFree(c->src);
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
  cudaFree(c->src);
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
  a.crow = g.cpitch / 2;
  a.vpitch = g.vpitch;
  a.cplane = (size_t)g.cheight * a.crow;
  a.vplane = (size_t)g.vheight * g.vpitch;
  a.kind = c->d.color_code;
  a.lsb = c->d.color_lsb ? 1 : 0;
  a.rcp_nc = pv_rcp31((uint32_t)g.nc);
  a.rcp_Tc = pv_rcp31((uint32_t)(g.nc * g.nc));
  // a slot's row spans 4 nv stream bytes, which touch at most this many 12-byte chunks
  a.kv = (4 * g.nv - 1 + 11) / 12 + 1;
  a.rcp_kv = pv_rcp31((uint32_t)a.kv);
  // widest vector store that divides a tile (the textures are 16-byte aligned)
  const int ttc = g.tc * g.tc, ttv = g.tv * g.tv;
  a.vw_c = ttc % 4 == 0 ? 4 : (ttc % 2 == 0 ? 2 : 1);
  a.vw_v = ttv % 8 == 0 ? 8 : (ttv % 4 == 0 ? 4 : (ttv % 2 == 0 ? 2 : 1));
  a.rcp_cvec = pv_rcp31((uint32_t)(ttc / a.vw_c));
  a.planes_c = f->color_planes;
  a.planes_v = f->vis_planes;
  a.delta_c = f->delta_c;
  a.delta_v = f->delta_v;
  a.count_c = f->count_c_dev;
  a.count_v = f->count_v_dev;
  a.tex_c = c->tex_c;
  a.tex_v = c->tex_v;
  a.src = c->src;
  a.src_q = c->src_q;
  a.src_voff = c->src_voff;
  const CaDyn L = ca_dyn_layout(g.nc, g.nv, c->src_q);
  a.off_src = L.src;
  a.off_warp = L.warp;
  a.warp_bytes = L.warp_bytes;
  pv_host::DeviceGuard guard(c->device);
  const int blocks = (g.P + CA_SLOTS - 1) / CA_SLOTS;
  k_client_apply<<<blocks, CA_THREADS, L.bytes, reinterpret_cast<cudaStream_t>(stream)>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "client apply kernel");
  return PV_OK;
}

}  // extern "C"
