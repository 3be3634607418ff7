// Device-side transmitted codes (Section 3.3 of arXiv 2103.05875) and storage
// conversions. Integer work only: given identical stored texels the codes are
// bit-exact with any correct implementation of the same definitions.
//
//  * UF10 (default colour code, A2RGB10F's 10-bit unsigned float): 5 exponent
//    bits (bias 15), 5 mantissa bits. One round-to-nearest-even from the
//    stored value, subnormals kept, negative / -0 / NaN -> 0, +inf and values
//    past the largest finite code clamp to 0x3DF.
//  * UNORM10: round(clamp(x, 0, 1) * 1023), ties to even, evaluated exactly.
//  * Visibility code: the binary16 bit pattern of the stored value.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/probe_stream.h"

namespace pv {

// Round-to-nearest-even of x / 2^s (0 < s < 32) without a branch; exact as
// long as x + 2^(s-1) fits in 32 bits.
__device__ __forceinline__ uint32_t rne_shift_fast(uint32_t x, uint32_t s) {
  return (x + ((1u << (s - 1)) - 1u) + ((x >> s) & 1u)) >> s;
}

// UF10 code of a binary16 value given by its bits. Branch-free: the code is
// the magnitude bits with 5 mantissa bits rounded off (binary16 and UF10
// share exponent bias and range, subnormals included); +inf rounds to 0x3E0
// and clamps with the finite overflow to 0x3DF. Bits above 0x7C00 are a set
// sign or a NaN, which give 0.
__device__ __forceinline__ uint32_t uf10_from_half_bits(uint32_t h) {
  const uint32_t a = h & 0x7FFFu;
  const uint32_t c = min(rne_shift_fast(a, 5), 0x3DFu);
  return h <= 0x7C00u ? c : 0u;
}

// UF10 code of a binary32 value given by its bits (one direct rounding),
// evaluated for both the UF10 normal and subnormal ranges and selected.
__device__ __forceinline__ uint32_t uf10_from_float_bits(uint32_t f) {
  const uint32_t e = (f >> 23) & 0xFFu, m = f & 0x7FFFFFu;
  // UF10 normal range (exponent >= -14): rebias the exponent to 15
  const uint32_t mag = ((e - 112u) << 23) | m;
  uint32_t cn = rne_shift_fast(mag, 18);
  cn = cn > 0x3DFu ? 0x3DFu : cn;
  // UF10 subnormal: code = round(value / 2^-19), value = (2^23 + m) * 2^(e-150)
  const uint32_t sh = 131u - e;                       // 19..31 for e in 100..112
  const uint32_t cs = (e >= 100u && e <= 112u) ? rne_shift_fast(0x800000u | m, sh < 31u ? sh : 31u) : 0u;
  uint32_t c = e >= 113u ? cn : cs;                   // e < 100 (incl. subnormal binary32): 0
  c = e == 255u ? (m ? 0u : 0x3DFu) : c;
  return (f & 0x80000000u) ? 0u : c;
}

// round(clamp(x,0,1)*1023) with ties to even, exact for any float x: the
// product's rounding residual decides values that round to a tie. NaN clamps
// to 0 (fmaxf returns the non-NaN operand).
__device__ __forceinline__ uint32_t unorm10_from_float(float x) {
  const float xc = fminf(fmaxf(x, 0.0f), 1.0f);
  const float p = xc * 1023.0f;
  const float e = fmaf(xc, 1023.0f, -p);              // exact residual of the product
  const float fl = floorf(p);
  const float fr = p - fl;                            // exact
  const uint32_t k = (uint32_t)fl;
  const bool up = fr > 0.5f || (fr == 0.5f && (e > 0.0f || (e == 0.0f && (k & 1u))));
  return k + (up ? 1u : 0u);
}

__device__ __forceinline__ float load_state(const void* base, size_t i, int fmt) {
  if (fmt == PV_FMT_F16) return __half2float(reinterpret_cast<const __half*>(base)[i]);
  return reinterpret_cast<const float*>(base)[i];
}

__device__ __forceinline__ void store_state(void* base, size_t i, float v, int fmt) {
  if (fmt == PV_FMT_F16) reinterpret_cast<__half*>(base)[i] = __float2half_rn(v);
  else reinterpret_cast<float*>(base)[i] = v;
}

// Raw bits of a stored texel (binary16 bits zero-extended, or binary32 bits).
__device__ __forceinline__ uint32_t load_state_bits(const void* base, size_t i, int fmt) {
  if (fmt == PV_FMT_F16) return reinterpret_cast<const uint16_t*>(base)[i];
  return reinterpret_cast<const uint32_t*>(base)[i];
}

__device__ __forceinline__ uint32_t color_code_of_bits(uint32_t b, int fmt, int kind);
__device__ __forceinline__ uint32_t vis_code_of_bits(uint32_t b, int fmt);

// Colour code of a stored texel.
__device__ __forceinline__ uint32_t color_code_of(const void* base, size_t i, int fmt, int kind) {
  return color_code_of_bits(load_state_bits(base, i, fmt), fmt, kind);
}

// Visibility code (RG16F channel) of a stored texel.
__device__ __forceinline__ uint32_t vis_code_of(const void* base, size_t i, int fmt) {
  return vis_code_of_bits(load_state_bits(base, i, fmt), fmt);
}

// Bits of a blended value once rounded to the state format.
__device__ __forceinline__ uint32_t state_bits_of(float v, int fmt) {
  return fmt == PV_FMT_F16 ? (uint32_t)__half_as_ushort(__float2half_rn(v)) : __float_as_uint(v);
}

__device__ __forceinline__ void store_state_bits(void* base, size_t i, uint32_t b, int fmt) {
  if (fmt == PV_FMT_F16) reinterpret_cast<uint16_t*>(base)[i] = (uint16_t)b;
  else reinterpret_cast<uint32_t*>(base)[i] = b;
}

__device__ __forceinline__ float state_value_of_bits(uint32_t b, int fmt) {
  return fmt == PV_FMT_F16 ? __half2float(__ushort_as_half((unsigned short)b)) : __uint_as_float(b);
}

__device__ __forceinline__ uint32_t color_code_of_bits(uint32_t b, int fmt, int kind) {
  if (kind == PV_CODE_UNORM10) return unorm10_from_float(state_value_of_bits(b, fmt));
  return fmt == PV_FMT_F16 ? uf10_from_half_bits(b) : uf10_from_float_bits(b);
}

__device__ __forceinline__ uint32_t vis_code_of_bits(uint32_t b, int fmt) {
  if (fmt == PV_FMT_F16) return b;
  return __half_as_ushort(__float2half_rn(__uint_as_float(b)));
}

// Tile positions (row, col in 0..n+1) that copy interior texel (i, j) (0-based),
// following the octahedral guard-band rule of Section 3.4 (reflection across
// each edge; corners by double reflection). Returns how many (at most 3 for
// n >= 2; all eight guard texels for n = 1).
__device__ __forceinline__ int border_targets(int i, int j, int n, int* tr, int* tc) {
  int r = i + 1, c = j + 1, k = 0;
  if (r == 1) { tr[k] = 0; tc[k] = n + 1 - c; ++k; }
  if (r == n) { tr[k] = n + 1; tc[k] = n + 1 - c; ++k; }
  if (c == 1) { tr[k] = n + 1 - r; tc[k] = 0; ++k; }
  if (c == n) { tr[k] = n + 1 - r; tc[k] = n + 1; ++k; }
  if (r == n && c == n) { tr[k] = 0; tc[k] = 0; ++k; }
  if (r == n && c == 1) { tr[k] = 0; tc[k] = n + 1; ++k; }
  if (r == 1 && c == n) { tr[k] = n + 1; tc[k] = 0; ++k; }
  if (r == 1 && c == 1) { tr[k] = n + 1; tc[k] = n + 1; ++k; }
  return k;
}

// x / d for 0 <= x < 2^16 and 1 <= d <= 2^15, with m = ceil(2^31 / d)
// (pv_rcp31): one multiply-high instead of an integer division.
__device__ __forceinline__ int fdiv(int x, uint32_t m) { return (int)__umulhi((uint32_t)x << 1, m); }

// Tile position (r, c) of an (n+2)^2 tile, 0 <= r, c <= n+1: the interior
// texel it holds, in tile coordinates (itself for interior positions; for the
// guard band the texel the reflection rule of Section 3.4 copies from).
__host__ __device__ __forceinline__ void border_source(int r, int c, int n, int* sr, int* sc) {
  const bool top = r == 0, bottom = r == n + 1, left = c == 0, right = c == n + 1;
  if ((top || bottom) && (left || right)) {          // corners: double reflection
    *sr = top ? n : 1;
    *sc = left ? n : 1;
  } else if (top || bottom) {
    *sr = top ? 1 : n;
    *sc = n + 1 - c;
  } else if (left || right) {
    *sr = n + 1 - r;
    *sc = left ? 1 : n;
  } else {
    *sr = r;
    *sc = c;
  }
}

}  // namespace pv
