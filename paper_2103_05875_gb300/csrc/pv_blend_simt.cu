// K1 (SIMT form): the probe blend of Section 3.2 of arXiv 2103.05875 with its
// fused epilogue, on the CUDA cores. Each block owns G probes; each thread
// owns up to MAXU "units", a unit being one (channel, texel) column
// accumulated over the block's G probes:
//   colour units   (c, t), c in {R, G, B}, weight row W_c[:, t]
//   visibility     (ch, t), ch in {d, d^2}, weight row W_v[:, t]
// Rays are streamed through shared memory in chunks of KC; the weights
// (computed once per frame by K0) come from L2.
//
// Epilogue per unit and probe: m = acc / sum(W); new = h*old + (1-h)*m (keep
// old if the weight sum is 0); round to the state format; write the interior
// texel and its guard-band copies (Section 3.4); compute the transmitted code
// and compare it with the last-transmitted one (Section 3.4, Change
// Thresholding), raising the (channel, probe) changed flag.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pv_codes.cuh"
#include "pv_internal.h"

namespace {

constexpr int G = 16;        // probes per block
constexpr int NT = 256;      // threads per block
constexpr int KC = 32;       // rays per shared-memory chunk
constexpr int MAXU = 5;      // units per thread: (2*Tv + 3*Tc) <= 1280 for n <= 16

template <typename Tin>
__device__ __forceinline__ float to_f(Tin v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// d^2 as the contraction sees it: formed on chip from the operand-format d and
// represented as hi + lo in the operand format (binary16 with a 2^-8 scale,
// undone here, so that d up to 4096 stays in range; bfloat16 unscaled).
template <typename Tin>
__device__ __forceinline__ float square_operand(float d);
template <>
__device__ __forceinline__ float square_operand<float>(float d) { return d * d; }
template <>
__device__ __forceinline__ float square_operand<__half>(float d) {
  const float q = d * d * 0.00390625f;                 // exact: d has 11 significant bits
  const float hi = __half2float(__float2half_rn(q));
  const float lo = __half2float(__float2half_rn(q - hi));
  return (hi + lo) * 256.0f;
}
template <>
__device__ __forceinline__ float square_operand<__nv_bfloat16>(float d) {
  const float q = d * d;                                // exact: d has 8 significant bits
  const float hi = __bfloat162float(__float2bfloat16_rn(q));
  const float lo = __bfloat162float(__float2bfloat16_rn(q - hi));
  return hi + lo;
}

template <typename Tin>
__global__ void __launch_bounds__(NT) k_blend_simt(pv_dev k, const Tin* __restrict__ rad,
                                                    const Tin* __restrict__ dist) {
  extern __shared__ float4 smem4[];
  float* xs = reinterpret_cast<float*>(smem4);          // [KC][5][G]
  const int T = k.Tc + k.Tv;
  float* ws = xs + KC * 5 * G;                          // [KC][T]
  __shared__ int flag_s[5 * G];

  const int tid = threadIdx.x;
  const int p0 = blockIdx.x * G;
  const int nunits = 2 * k.Tv + 3 * k.Tc;
  for (int q = tid; q < 5 * G; q += NT) flag_s[q] = 0;

  // unit bookkeeping
  int u_w[MAXU], u_x[MAXU];
  float acc[MAXU][G];
#pragma unroll
  for (int q = 0; q < MAXU; ++q) {
    const int u = tid + q * NT;
    int wcol = 0, xch = 0;
    if (u < 2 * k.Tv) { wcol = k.Tc + (u >> 1); xch = 3 + (u & 1); }
    else if (u < nunits) { const int v = u - 2 * k.Tv; wcol = v % k.Tc; xch = v / k.Tc; }
    u_w[q] = wcol;
    u_x[q] = xch * G;
#pragma unroll
    for (int g = 0; g < G; ++g) acc[q][g] = 0.0f;
  }

  for (int r0 = 0; r0 < k.R; r0 += KC) {
    const int kc = min(KC, k.R - r0);
    __syncthreads();
    // ray payload chunk: colour planes then d (and d^2 formed here)
    for (int e = tid; e < 4 * G * kc; e += NT) {
      const int rr = e % kc;
      const int g = (e / kc) % G;
      const int ch = e / (kc * G);
      const int p = p0 + g;
      float v = 0.0f;
      if (p < k.P) {
        if (ch < 3) v = to_f<Tin>(rad[((size_t)ch * k.P + p) * k.R + r0 + rr]);
        else v = to_f<Tin>(dist[(size_t)p * k.R + r0 + rr]);
      }
      xs[(rr * 5 + ch) * G + g] = v;
      if (ch == 3) xs[(rr * 5 + 4) * G + g] = square_operand<Tin>(v);
    }
    for (int e = tid; e < kc * T; e += NT) ws[e] = k.w_rt[(size_t)r0 * T + e];
    __syncthreads();
    for (int rr = 0; rr < kc; ++rr) {
#pragma unroll
      for (int q = 0; q < MAXU; ++q) {
        if (tid + q * NT < nunits) {
          const float w = ws[rr * T + u_w[q]];
          const float4* xv = reinterpret_cast<const float4*>(xs + rr * 5 * G + u_x[q]);
#pragma unroll
          for (int g4 = 0; g4 < G / 4; ++g4) {
            const float4 x4 = xv[g4];
            acc[q][4 * g4 + 0] = fmaf(w, x4.x, acc[q][4 * g4 + 0]);
            acc[q][4 * g4 + 1] = fmaf(w, x4.y, acc[q][4 * g4 + 1]);
            acc[q][4 * g4 + 2] = fmaf(w, x4.z, acc[q][4 * g4 + 2]);
            acc[q][4 * g4 + 3] = fmaf(w, x4.w, acc[q][4 * g4 + 3]);
          }
        }
      }
    }
  }

  // fused epilogue: loads of old texels and last codes are issued for all G
  // probes of a unit before any of them is used
  const float h = *k.hy;
  const float one_m_h = 1.0f - h;
#pragma unroll
  for (int q = 0; q < MAXU; ++q) {
    const int u = tid + q * NT;
    if (u >= nunits) continue;
    const bool vis = u < 2 * k.Tv;
    const int ch = vis ? (u & 1) : (u - 2 * k.Tv) / k.Tc;
    const int t = vis ? (u >> 1) : (u - 2 * k.Tv) % k.Tc;
    const int n = vis ? k.nv : k.nc;
    const int tile = n + 2;
    const int i = t / n, j = t % n;
    const float S = k.sums[(vis ? k.Tc : 0) + t];
    void* st = vis ? k.state_v : k.state_c;
    const uint16_t* last = vis ? k.last_v : k.last_c;
    const int sstride = vis ? k.sv_stride : k.sc_stride;
    const int lstride = vis ? k.lv_stride : k.lc_stride;
    const int pos = (i + 1) * tile + (j + 1);
    int tr[8], tcl[8];
    const int nb = pv::border_targets(i, j, n, tr, tcl);
    uint32_t oldb[G];
    uint32_t prev[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int p = min(p0 + g, k.P - 1);
      oldb[g] = pv::load_state_bits(st, ((size_t)ch * k.P + p) * sstride + pos, k.state_fmt);
      prev[g] = last[((size_t)ch * k.P + p) * lstride + t];
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int p = p0 + g;
      if (p >= k.P) continue;
      const size_t tile0 = ((size_t)ch * k.P + p) * sstride;
      uint32_t nb_bits = oldb[g];
      if (S > 0.0f) {
        const float m = acc[q][g] / S;
        const float old = pv::state_value_of_bits(oldb[g], k.state_fmt);
        nb_bits = pv::state_bits_of(fmaf(h, old, one_m_h * m), k.state_fmt);
        pv::store_state_bits(st, tile0 + pos, nb_bits, k.state_fmt);
      }
      for (int b = 0; b < nb; ++b)
        pv::store_state_bits(st, tile0 + (size_t)tr[b] * tile + tcl[b], nb_bits, k.state_fmt);
      const uint32_t code = vis ? pv::vis_code_of_bits(nb_bits, k.state_fmt)
                                : pv::color_code_of_bits(nb_bits, k.state_fmt, k.color_code);
      if (code != prev[g]) flag_s[((vis ? 3 : 0) + ch) * G + g] = 1;
      if (k.cur_c) (vis ? k.cur_v : k.cur_c)[((size_t)ch * k.P + p) * lstride + t] = (uint16_t)code;
    }
  }
  __syncthreads();
  if (tid < 2) {                      // changed-probe bits of this block's probes
    uint32_t mask = 0;
    for (int g = 0; g < G && p0 + g < k.P; ++g) {
      const int f = tid == 0 ? (flag_s[0 * G + g] | flag_s[1 * G + g] | flag_s[2 * G + g])
                             : (flag_s[3 * G + g] | flag_s[4 * G + g]);
      if (f) mask |= 1u << ((p0 + g) & 31);
    }
    if (mask) atomicOr(&k.chg[tid * k.chg_words + (p0 >> 5)], mask);
  }
}

}  // namespace

cudaError_t pv_simt_prepare() {
  // largest dynamic shared memory any volume can ask for (n_c = n_v = 16)
  const int smem = KC * (5 * G + 2 * PV_MAX_INTERIOR * PV_MAX_INTERIOR) * (int)sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_blend_simt<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_blend_simt<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_blend_simt<__nv_bfloat16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

cudaError_t pv_launch_blend_simt(const pv_dev& k, const void* rad, const void* dist,
                                 cudaStream_t st) {
  const int blocks = (k.P + G - 1) / G;
  const size_t smem = (size_t)KC * (5 * G + k.Tc + k.Tv) * sizeof(float);
  switch (k.operand_fmt) {
    case PV_FMT_F32:
      k_blend_simt<float><<<blocks, NT, smem, st>>>(k, (const float*)rad, (const float*)dist);
      break;
    case PV_FMT_F16:
      k_blend_simt<__half><<<blocks, NT, smem, st>>>(k, (const __half*)rad, (const __half*)dist);
      break;
    default:
      k_blend_simt<__nv_bfloat16><<<blocks, NT, smem, st>>>(k, (const __nv_bfloat16*)rad,
                                                            (const __nv_bfloat16*)dist);
      break;
  }
  return cudaGetLastError();
}
