// K0: per-frame blend weights of a probe volume (Section 3.2 of arXiv
// 2103.05875, after DDGI): for every colour texel W = max(0, n_t . d_r), for
// every visibility texel W = max(0, n_t . d_r)^sharpness, plus the weight sums
// used for normalisation. One block per texel, threads over rays. Block 0
// also clears the frame's changed-probe bits and sets the frame's hysteresis.
//
// Per-texel scale. The normalised mean sum_r W x_r / sum_r W does not change
// when all of a texel's weights are multiplied by one factor, so each texel's
// weights are taken relative to its largest cosine c_max: colour weights are
// c scaled by the power of two that brings c_max into [1, 2) (exact),
// visibility weights are (c / c_max)^s (the largest is 1). No weight of a
// texel that sees any ray can then underflow, whatever the sharpness or the
// operand format: a texel whose rays all lie more than ~83 degrees away would
// otherwise get cos^50 below the smallest float32, and one beyond ~55 degrees
// would get binary16 zeros. A texel keeps its old value (weight sum 0) only
// when no ray lies in its hemisphere.
//
// Operand forms. FP32: the SIMT blend uses W as is; the tensor-core blend gets
// W = hi + lo with hi = W truncated to TF32 and lo = W - hi (three TF32
// products recover FP32 accuracy). FP16: W in binary16, visibility weights
// scaled by 2^15 (the largest is then 2^15, and relative weights down to 2^-29
// stay normal binary16 numbers). BF16: W = hi + lo, both bfloat16 (two
// products), since one bfloat16 weight alone is only good to 2^-9. The weight
// sums always add the effective (rounded) weights, so every texel's mean stays
// a convex combination.
//
// Accuracy: the octahedral texel direction is q/|q| with an integer vector q
// (u = a/n, v = b/n with integer a, b), so n_t . d_r is evaluated as a
// float-float dot product of exact integers with the float32 ray directions,
// divided by sqrt(|q|^2) in float-float. The cosine is then within half an
// ulp; the ratio c / c_max is formed as a float-float too, and the visibility
// weight (c / c_max)^s is corrected to first order for the ratio's low part
// (s * r_lo / r_hi), which keeps the amplification of rounding by the
// exponent s out of W. Weights are rounded to the operand
// format (FP16/BF16 precision forms) before they are summed, so each texel's
// normalisation uses exactly the weights of the contraction.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pv_internal.h"

namespace {

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

constexpr float kVisScaleF16 = 32768.0f;   // 2^15

// Effective weight of the operand form, and its operand planes.
struct OpWeight {
  float eff;       // value the contraction effectively multiplies with
  float hi, lo;    // plane values (lo unused for F16)
};

__device__ __forceinline__ OpWeight split_weight(float w, int fmt, bool vis) {
  OpWeight o;
  if (fmt == PV_FMT_F16) {
    const float s = vis ? kVisScaleF16 : 1.0f;
    o.hi = __half2float(__float2half_rn(w * s));
    o.lo = 0.0f;
    o.eff = o.hi;
  } else if (fmt == PV_FMT_BF16) {
    o.hi = __bfloat162float(__float2bfloat16_rn(w));
    o.lo = __bfloat162float(__float2bfloat16_rn(w - o.hi));
    o.eff = o.hi + o.lo;                           // exact in binary32
  } else {
    o.hi = __uint_as_float(__float_as_uint(w) & 0xFFFFE000u);   // TF32 truncation
    o.lo = w - o.hi;                               // exact
    o.eff = w;
  }
  return o;
}

__device__ __forceinline__ void store_plane(void* base, size_t i, float w, int fmt) {
  if (fmt == PV_FMT_F16) reinterpret_cast<__half*>(base)[i] = __float2half_rn(w);
  else if (fmt == PV_FMT_BF16) reinterpret_cast<__nv_bfloat16*>(base)[i] = __float2bfloat16_rn(w);
  else reinterpret_cast<float*>(base)[i] = w;
}

// Weights of texel tg (colour texels first) of volume k; one block of 256
// threads, at most PV_MAX_RAYS / 256 rays per thread. All arithmetic (cosine,
// power, operand split, the block's weight sum) runs before the wait for the
// previous kernel; only the stores come after it, since the previous blend of
// the volume may still read the weight images and sums.
constexpr int kRaysPerThread = (PV_MAX_RAYS + 255) / 256;

__device__ __forceinline__ void weights_block(const pv_dev& k, const float* __restrict__ dirs, int want_rt,
                                              int want_op, int tg, bool first_block) {
  const int T = k.Tc + k.Tv;
  const bool vis = tg >= k.Tc;
  const int n = vis ? k.nv : k.nc;
  const int t = vis ? tg - k.Tc : tg;
  const int i = t / n, j = t % n;
  const int a = 2 * j + 1 - n, b = 2 * i + 1 - n;
  const int z = n - abs(a) - abs(b);
  const int x = z < 0 ? (n - abs(b)) * (a >= 0 ? 1 : -1) : a;
  const int y = z < 0 ? (n - abs(a)) * (b >= 0 ? 1 : -1) : b;
  const float fx = (float)x, fy = (float)y, fz = (float)z;
  const float Q = (float)(x * x + y * y + z * z);       // exact small integer
  const float sq = sqrtf(Q);
  const float sq_lo = fmaf(-sq, sq, Q) / (2.0f * sq);   // sqrt(Q) ~= sq + sq_lo
  const float s = k.sharpness;

  // cosines of this thread's rays as float-floats, and the block's largest
  float ch[kRaysPerThread], cl[kRaysPerThread];
  float mh = -2.0f, ml = 0.0f;
#pragma unroll
  for (int u = 0; u < kRaysPerThread; ++u) {
    const int r = threadIdx.x + 256 * u;
    ch[u] = -2.0f;
    cl[u] = 0.0f;
    if (r >= k.R) continue;
    const float dx = dirs[3 * r + 0], dy = dirs[3 * r + 1], dz = dirs[3 * r + 2];
    float p1, e1, p2, e2, p3, e3, s12, f12, sd, f3;
    two_prod(fx, dx, p1, e1);
    two_prod(fy, dy, p2, e2);
    two_prod(fz, dz, p3, e3);
    two_sum(p1, p2, s12, f12);
    two_sum(s12, p3, sd, f3);
    const float sd_lo = ((e1 + e2) + e3) + (f12 + f3);   // q . d ~= sd + sd_lo
    const float c0 = sd / sq;
    float rem = fmaf(-c0, sq, sd);                        // exact remainder of the division
    rem = (rem + sd_lo) - c0 * sq_lo;
    const float c1 = rem / sq;
    two_sum(c0, c1, ch[u], cl[u]);                        // cosine as a float-float
    if (ch[u] > mh || (ch[u] == mh && cl[u] > ml)) {
      mh = ch[u];
      ml = cl[u];
    }
  }
  // block maximum of the cosine (warp shuffles, then the warps' maxima in
  // a fixed order: every thread ends with the same pair)
  __shared__ float smax[2][8];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, mh, off), ol = __shfl_xor_sync(0xffffffffu, ml, off);
    if (oh > mh || (oh == mh && ol > ml)) {
      mh = oh;
      ml = ol;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    smax[0][threadIdx.x >> 5] = mh;
    smax[1][threadIdx.x >> 5] = ml;
  }
  __syncthreads();
  mh = smax[0][0];
  ml = smax[1][0];
  for (int wi = 1; wi < 8; ++wi) {
    if (smax[0][wi] > mh || (smax[0][wi] == mh && smax[1][wi] > ml)) {
      mh = smax[0][wi];
      ml = smax[1][wi];
    }
  }
  const int ce = mh > 0.0f ? ilogbf(mh) : 0;               // colour: c * 2^-ce, largest in [1, 2)

  OpWeight o[kRaysPerThread];
  float part = 0.0f;
#pragma unroll
  for (int u = 0; u < kRaysPerThread; ++u) {
    o[u] = OpWeight{0.0f, 0.0f, 0.0f};
    const float c_hi = ch[u], c_lo = cl[u];
    if (!(c_hi > 0.0f)) continue;                          // no ray, or a ray behind the texel
    float w;
    if (!vis) {
      w = ldexpf(c_hi, -ce);
    } else {
      // r = c / c_max as a float-float (the remainder of r0 * m_hi is exact)
      const float r0 = c_hi / mh;
      const float res = fmaf(-r0, mh, c_hi) + (c_lo - r0 * ml);
      const float r1 = res / mh;
      w = powf(r0, s) * fmaf(s, r1 / r0, 1.0f);
    }
    o[u] = split_weight(w, k.operand_fmt, vis);
    part += o[u].eff;
  }
  // deterministic block reduction of the weight sum
  __shared__ float red[256];
  red[threadIdx.x] = part;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }

  pv_grid_wait();                     // stores only from here on
  // Operand-format copy for the tensor-core blend: shared-memory tile images
  // (pv_w_image_offset), visibility texels in rows 0.., colour from w_vb.
  const int op_row = vis ? t : k.w_vb + t;
  const int eb = k.operand_fmt == PV_FMT_F32 ? 4 : 2;
  const size_t plane = (size_t)k.w_chunks * k.w_rows * k.w_rb;   // bytes per operand plane
#pragma unroll
  for (int u = 0; u < kRaysPerThread; ++u) {
    const int r = threadIdx.x + 256 * u;
    if (r >= k.R) continue;
    if (want_rt) k.w_rt[(size_t)r * T + tg] = o[u].eff;
    if (want_op) {
      uint8_t* img = reinterpret_cast<uint8_t*>(k.w_op) + pv_w_image_offset(k, op_row, r, eb);
      store_plane(img, 0, o[u].hi, k.operand_fmt);
      if (k.operand_fmt != PV_FMT_F16) store_plane(img + plane, 0, o[u].lo, k.operand_fmt);
    }
  }
  if (threadIdx.x == 0) k.sums[tg] = red[0];

  if (first_block) {                // this frame's changed-probe bits start cleared
    for (int w = threadIdx.x; w < 2 * k.chg_words; w += blockDim.x) k.chg[w] = 0u;
  }
  if (first_block && threadIdx.x == 0) {
    unsigned long long f = *k.frame;
    *k.hy = (f == 0ull && k.first_frame_no_hysteresis) ? 0.0f : k.h;
    *k.frame = f + 1ull;
  }
}

__global__ void __launch_bounds__(256) k_weights(pv_dev k, const float* __restrict__ dirs,
                                                 int want_rt, int want_op) {
  pv_grid_launch_dependents();
  weights_block(k, dirs, want_rt, want_op, blockIdx.x, blockIdx.x == 0);
}

// Several volumes in one launch: blockIdx.y is the volume.
struct WeightsBatch {
  pv_dev k[PV_MAX_BATCH];
  const float* dirs[PV_MAX_BATCH];
};

__global__ void __launch_bounds__(256) k_weights_batch(const __grid_constant__ WeightsBatch b, int want_rt,
                                                       int want_op) {
  pv_grid_launch_dependents();
  const pv_dev& k = b.k[blockIdx.y];
  if ((int)blockIdx.x >= k.Tc + k.Tv) return;          // no texel: writes nothing
  weights_block(k, b.dirs[blockIdx.y], want_rt, want_op, blockIdx.x, blockIdx.x == 0);
}

}  // namespace

cudaError_t pv_launch_weights_batch(const pv_dev* ks, const float* const* dirs, int n, int want_rt, int want_op,
                                    cudaStream_t st) {
  if (n < 1 || n > PV_MAX_BATCH) return cudaErrorInvalidValue;
  WeightsBatch* b = new WeightsBatch();
  int most = 0;
  for (int i = 0; i < n; ++i) {
    b->k[i] = ks[i];
    b->dirs[i] = dirs[i];
    most = ks[i].Tc + ks[i].Tv > most ? ks[i].Tc + ks[i].Tv : most;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1] = {pv_pdl_attr()};
  cfg.gridDim = dim3(most, n);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_weights_batch, *b, want_rt, want_op);
  delete b;
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t pv_launch_weights(const pv_dev& k, const float* dirs, int want_rt, int want_op,
                              cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1] = {pv_pdl_attr()};
  cfg.gridDim = dim3(k.Tc + k.Tv);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_weights, k, dirs, want_rt, want_op);
  return e != cudaSuccess ? e : cudaGetLastError();
}
