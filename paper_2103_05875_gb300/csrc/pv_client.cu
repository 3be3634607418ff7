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
// stores. Each thread issues all of its global loads (counts, plane samples,
// deltas) before it uses any of them, so a block waits for memory once; slots
// past the frame's counts are read too (they lie inside the planes) and
// dropped. Probe ids at or past P and counts past P are ignored, so a damaged
// frame cannot make the kernel write outside the textures.
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
  int src_q;         // their size in 16-byte words
};

namespace {

constexpr int CA_THREADS = 256;
constexpr int CA_SLOTS = 4;                             // slots per block (a power of two, <= 16)
constexpr int CA_BATCH = 2;                             // 16-byte delta words a thread loads at once

struct CaArgs {
  int P, nc, nv, tc, tv, bw, cheight, cpitch, vheight, vpitch;
  int kind, lsb;
  uint32_t rcp_nc, rcp_nv, rcp_3, rcp_3nc;
  int kv;                                // 12-byte visibility chunks a slot's row can touch
  uint32_t rcp_kv, rcp_wc;
  int vw_c, vw_v;                        // texels per vector store of a colour / visibility tile
  uint32_t rcp_cvec, rcp_vvec;           // ceil(2^31 / vectors per tile)
  const uint16_t* planes_c;
  const uint8_t* planes_v;
  const uint16_t* delta_c;
  const uint16_t* delta_v;
  const uint32_t* count_c;
  const uint32_t* count_v;
  const uint16_t* src;                   // guard-band tables, src_q 16-byte words
  int src_q;
  uint32_t off_vv, off_src, off_rawc, off_rawv, off_dq;   // dynamic shared memory layout (CaDyn)
  float* tex_c;
  uint16_t* tex_v;
};

// 32-bit words holding a row of n colour samples (16-bit) that starts at any
// sample of a plane row.
__host__ __device__ constexpr int ca_words_c(int n) { return n / 2 + 1; }

// Shared memory sized to the volume's interiors (dynamic, after CaShared),
// byte offsets of:
//   float    vc[CA_SLOTS][3][Tc]     decoded colour interiors of the block's slots
//   uint32_t vv[CA_SLOTS][Tv]        visibility interiors: R | G << 16
//   uint16_t src_c[tc*tc], src_v[tv*tv]   per tile position: the interior texel it holds
//   uint32_t rawc[CA_SLOTS][3][nc][wc]    the plane words of each slot's colour rows
//   uint32_t rawv[CA_SLOTS][nv][kv][3]    the three plane words of each visibility chunk
//   uint4    dq[CA_BATCH][2][CA_THREADS]  the first 16-byte delta words each thread sums
struct CaDyn {
  uint32_t vc, vv, src_c, src_v, rawc, rawv, dq, bytes;
};

__host__ __device__ inline CaDyn ca_dyn_layout(int nc, int nv, int tc, int tv, int kv) {
  const auto up16 = [](uint32_t x) { return (x + 15u) & ~15u; };
  CaDyn L;
  L.vc = 0;
  L.vv = up16(L.vc + CA_SLOTS * 3 * nc * nc * 4);
  L.src_c = up16(L.vv + CA_SLOTS * nv * nv * 4);
  L.src_v = L.src_c + tc * tc * 2;
  L.rawc = up16(L.src_v + tv * tv * 2);
  L.rawv = up16(L.rawc + CA_SLOTS * 3 * nc * ca_words_c(nc) * 4);
  L.dq = up16(L.rawv + CA_SLOTS * nv * kv * 3 * 4);
  // (the tables are copied in whole 16-byte words: room up to rawc)
  L.bytes = L.dq + CA_BATCH * 2 * CA_THREADS * 16;
  return L;
}

struct CaShared {
  int id_c[CA_SLOTS], id_v[CA_SLOTS];    // probe of each slot, -1 for none
  uint32_t red[2 * CA_THREADS / 32];
};

// Adds the eight 16-bit deltas of a 16-byte word to acc (each dp2a adds both
// halves of a 32-bit word); ids are taken modulo 2^16, so wrap-around of acc
// is harmless.
__device__ __forceinline__ uint32_t sum16(uint32_t acc, uint4 v) {
  const uint32_t a0 = __dp2a_lo(v.x, 0x0101u, __dp2a_lo(v.y, 0x0101u, acc));
  const uint32_t a1 = __dp2a_lo(v.z, 0x0101u, __dp2a_lo(v.w, 0x0101u, 0u));
  return a0 + a1;
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

// 4- and 16-byte asynchronous copies global -> shared (both addresses aligned
// to the size), and the wait for every copy the thread issued.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__global__ void __launch_bounds__(CA_THREADS, 8) k_client_apply(const CaArgs a) {
  __shared__ __align__(16) CaShared sh;
  extern __shared__ __align__(16) uint8_t ca_dyn[];
  const int n_c = a.nc, n_v = a.nv, Tc = n_c * n_c, Tv = n_v * n_v;
  float* vc = reinterpret_cast<float*>(ca_dyn);
  uint32_t* vv = reinterpret_cast<uint32_t*>(ca_dyn + a.off_vv);
  uint16_t* src_c = reinterpret_cast<uint16_t*>(ca_dyn + a.off_src);
  uint16_t* src_v = src_c + a.tc * a.tc;
  uint32_t* rawc = reinterpret_cast<uint32_t*>(ca_dyn + a.off_rawc);
  uint32_t* rawv = reinterpret_cast<uint32_t*>(ca_dyn + a.off_rawv);
  uint4* dq = reinterpret_cast<uint4*>(ca_dyn + a.off_dq);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int k0 = blockIdx.x * CA_SLOTS;
  const int nsl = min(CA_SLOTS, a.P - k0);             // the block's slots inside the volume
  // block of the update texture of the block's first slot; slot s follows
  const int by0 = k0 / a.bw, bx0 = k0 - by0 * a.bw;
  const auto slot_block = [&](int s, int& bx, int& by) {
    bx = bx0 + s;
    by = by0;
    while (bx >= a.bw) {
      bx -= a.bw;
      ++by;
    }
  };

  // ---- loads, all issued before any is used. Slots past the frame's counts
  // are read too (they lie inside the planes) and dropped below.
  const uint32_t cnt_c_raw = *a.count_c, cnt_v_raw = *a.count_v;
  for (int q = tid; q < a.src_q; q += CA_THREADS) cp_async16(src_c + 8 * q, a.src + 8 * q);
  // colour: the 32-bit words holding row i of slot s in plane c, items
  // (s, c, i, k) with k fastest, copied to rawc[((s*3 + c)*n + i)*wc + k]
  const int wc = ca_words_c(n_c), items_c = CA_SLOTS * 3 * n_c * wc;
  const size_t cplane = (size_t)a.cheight * a.cpitch;
  for (int it = tid; it < items_c; it += CA_THREADS) {
    const int t = pv::fdiv(it, a.rcp_wc), k = it - t * wc;
    const int u = pv::fdiv(t, a.rcp_nc), i = t - u * n_c;
    const int s = pv::fdiv(u, a.rcp_3), c = u - s * 3;
    if (s >= nsl) continue;
    int bx, by;
    slot_block(s, bx, by);
    const int w0 = (bx * n_c) >> 1, w = w0 + k;
    if (w > ((bx * n_c + n_c - 1) >> 1)) continue;
    cp_async4(rawc + it, reinterpret_cast<const uint8_t*>(a.planes_c) + c * cplane +
                             (size_t)(by * n_c + i) * a.cpitch + 4 * (size_t)w);
  }
  // visibility: chunk k of row i of slot s, the atlas row's stream bytes
  // 12w..12w+11 (texels 3w..3w+2), which are the words at column 4w of the
  // three planes; items (s, i, k), copied to rawv[3*it + plane]
  const int items_v = CA_SLOTS * n_v * a.kv;
  const size_t vplane = (size_t)a.vheight * a.vpitch;
  for (int it = tid; it < items_v; it += CA_THREADS) {
    const int t = pv::fdiv(it, a.rcp_kv), k = it - t * a.kv;
    const int s = pv::fdiv(t, a.rcp_nv), i = t - s * n_v;
    if (s >= nsl) continue;
    int bx, by;
    slot_block(s, bx, by);
    const int xs = n_v * bx, w = xs / 3 + k;
    if (w > (4 * (xs + n_v) - 1) / 12) continue;
    const uint8_t* row = a.planes_v + (size_t)(by * n_v + i) * a.vpitch + 4 * (size_t)w;
    cp_async4(rawv + 3 * it, row);
    cp_async4(rawv + 3 * it + 1, row + vplane);
    cp_async4(rawv + 3 * it + 2, row + 2 * vplane);
  }
  // deltas: the k0 before the block's first slot in 16-byte words (the first
  // CA_BATCH of each thread staged in dq, where only that thread reads them)
  // and a tail, and the block's own (first warp: lanes 0..SLOTS-1 colour, then
  // visibility)
  const int nq = k0 >> 3;
  const uint4* dc4 = reinterpret_cast<const uint4*>(a.delta_c);
  const uint4* dv4 = reinterpret_cast<const uint4*>(a.delta_v);
#pragma unroll
  for (int u = 0; u < CA_BATCH; ++u) {
    const int q = tid + u * CA_THREADS;
    if (q < nq) {
      cp_async16(dq + (2 * u) * CA_THREADS + tid, dc4 + q);
      cp_async16(dq + (2 * u + 1) * CA_THREADS + tid, dv4 + q);
    }
  }
  uint32_t sum_c = 0, sum_v = 0, d = 0;
  if (tid < (k0 & 7)) {
    sum_c = a.delta_c[8 * nq + tid];
    sum_v = a.delta_v[8 * nq + tid];
  }
  if (tid < 2 * CA_SLOTS) {
    const int s = tid & (CA_SLOTS - 1);
    if (s < nsl) d = tid >= CA_SLOTS ? a.delta_v[k0 + s] : a.delta_c[k0 + s];
  }

  // ---- delta sums modulo 2^16, one partial per warp
  cp_async_wait_all();
#pragma unroll
  for (int u = 0; u < CA_BATCH; ++u) {
    if (tid + u * CA_THREADS < nq) {
      sum_c = sum16(sum_c, dq[(2 * u) * CA_THREADS + tid]);
      sum_v = sum16(sum_v, dq[(2 * u + 1) * CA_THREADS + tid]);
    }
  }
  for (int q = tid + CA_BATCH * CA_THREADS; q < nq; q += CA_THREADS) {
    sum_c = sum16(sum_c, dc4[q]);
    sum_v = sum16(sum_v, dv4[q]);
  }
  sum_c = __reduce_add_sync(0xffffffffu, sum_c);
  sum_v = __reduce_add_sync(0xffffffffu, sum_v);
  const int cnt_c = (int)min(cnt_c_raw, (uint32_t)a.P), cnt_v = (int)min(cnt_v_raw, (uint32_t)a.P);
  const int ns_c = max(0, min(nsl, cnt_c - k0)), ns_v = max(0, min(nsl, cnt_v - k0));
  if (ns_c == 0 && ns_v == 0) return;                   // uniform: the block has no slot in the frame
  if (lane == 0) {
    sh.red[2 * wid] = sum_c;
    sh.red[2 * wid + 1] = sum_v;
  }
  __syncthreads();

  // ---- probe ids: the deltas before the block's slots plus the inclusive
  // prefix of its own (the sums before k0 are of this frame's deltas whenever
  // the block has a slot below the count)
  if (tid < 32) {
    const int s = lane & (CA_SLOTS - 1);
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
  // ---- interiors from the staged words: colour items (s, c, i, j)
  for (int it = tid; it < ns_c * 3 * Tc; it += CA_THREADS) {
    const int t = pv::fdiv(it, a.rcp_nc), j = it - t * n_c;     // t = (s*3 + c)*n + i
    const int s = pv::fdiv(t, a.rcp_3nc);
    int bx, by;
    slot_block(s, bx, by);
    const int o = ((bx * n_c) & 1) + j;                         // sample o of the row's first word
    const uint32_t word = rawc[t * wc + (o >> 1)];
    const uint32_t sample = (o & 1) ? word >> 16 : word & 0xFFFFu;
    const uint32_t code = a.lsb ? (sample & 0x3FFu) : (sample >> 6);
    vc[t * n_c + j] = color_value(code, a.kind);
  }
  // visibility chunks (s, i, k): stream byte 12w + b sits in plane b % 3, byte
  // b / 3 of that word; keep the texels inside the slot's row
  for (int it = tid; it < ns_v * n_v * a.kv; it += CA_THREADS) {
    const int t = pv::fdiv(it, a.rcp_kv), k = it - t * a.kv;    // t = s*n + i
    const int s = pv::fdiv(t, a.rcp_nv);
    int bx, by;
    slot_block(s, bx, by);
    const int xs = n_v * bx, x = 3 * (xs / 3 + k) - xs;         // texel 3w relative to the slot's first
    if (x >= n_v) continue;
    const uint32_t p0 = rawv[3 * it], p1 = rawv[3 * it + 1], p2 = rawv[3 * it + 2];
    const uint32_t t3[3] = {__byte_perm(__byte_perm(p0, p1, 0x1040), p2, 0x3410),
                            __byte_perm(__byte_perm(p1, p2, 0x2051), p0, 0x3610),
                            __byte_perm(__byte_perm(p2, p0, 0x3072), p1, 0x3710)};
#pragma unroll
    for (int e = 0; e < 3; ++e)
      if (x + e >= 0 && x + e < n_v) vv[t * n_v + x + e] = t3[e];
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
  // the guard-band rule of the two tile sizes as tables: tile position -> interior texel
  const int ntab = g.tc * g.tc + g.tv * g.tv;
  c->src_q = (ntab * 2 + 15) / 16;
  std::vector<uint16_t> tab((size_t)c->src_q * 8, 0);
  for (int e = 0; e < ntab; ++e) {
    const bool vis = e >= g.tc * g.tc;
    const int t = vis ? g.tv : g.tc, n = vis ? g.nv : g.nc, q = vis ? e - g.tc * g.tc : e;
    int sr, sc;
    pv::border_source(q / t, q % t, n, &sr, &sc);
    tab[e] = (uint16_t)((sr - 1) * n + (sc - 1));
  }
  cudaError_t e = cudaMalloc((void**)&c->tex_c, bc);
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
  a.cheight = g.cheight;
  a.cpitch = g.cpitch;
  a.vheight = g.vheight;
  a.vpitch = g.vpitch;
  a.kind = c->d.color_code;
  a.lsb = c->d.color_lsb ? 1 : 0;
  a.rcp_nc = pv_rcp31((uint32_t)g.nc);
  a.rcp_nv = pv_rcp31((uint32_t)g.nv);
  // a slot's row spans 4 nv stream bytes, which touch at most this many 12-byte chunks
  a.kv = (4 * g.nv - 1 + 11) / 12 + 1;
  a.rcp_kv = pv_rcp31((uint32_t)a.kv);
  a.rcp_wc = pv_rcp31((uint32_t)ca_words_c(g.nc));
  a.rcp_3 = pv_rcp31(3u);
  a.rcp_3nc = pv_rcp31(3u * (uint32_t)g.nc);
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
  a.src = c->src;
  a.src_q = c->src_q;
  const CaDyn L = ca_dyn_layout(g.nc, g.nv, g.tc, g.tv, a.kv);
  a.off_vv = L.vv;
  a.off_src = L.src_c;
  a.off_rawc = L.rawc;
  a.off_rawv = L.rawv;
  a.off_dq = L.dq;
  pv_host::DeviceGuard guard(c->device);
  const int blocks = (g.P + CA_SLOTS - 1) / CA_SLOTS;
  k_client_apply<<<blocks, CA_THREADS, L.bytes, reinterpret_cast<cudaStream_t>(stream)>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "client apply kernel");
  return PV_OK;
}

}  // extern "C"
