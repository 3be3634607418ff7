// pv_ray_directions: spherical Fibonacci ray set rotated by a uniformly random
// rotation, a convenience for callers that trace rays for probe_update. The
// blend itself takes directions as an input (Section 3.2 of arXiv 2103.05875
// defers the ray set to DDGI).
//
// Definitions (all in float64, rounded to float32 at the end):
//  * SplitMix64 (Steele, Lea & Flood 2014): output i of the stream keyed by k
//    is mix64(k + (i + 1) * 0x9E3779B97F4A7C15); sub-stream keys are chained
//    through the same function: key(seed, a, b, c) = s(s(s(seed, a), b), c).
//  * uniform in [0, 1): (x >> 11) * 2^-53.
//  * Shoemake (1992) uniform unit quaternion from u1, u2, u3 and its rotation.
//  * Fibonacci point i of R: z = 1 - (2i+1)/R, phi = 2 pi frac(i (sqrt 5 - 1)/2).
#include <math.h>
#include <stdint.h>

#include "pv_internal.h"

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kKindRotation = 1;

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t stream_at(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * kGamma); }

double unit(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

}  // namespace

extern "C" pv_status pv_ray_directions(uint64_t seed, uint64_t volume, uint64_t frame, int32_t rays,
                                       float* out) {
  if (!out || rays <= 0 || rays > PV_MAX_RAYS)
    return pv_set_error(PV_ERR_INVALID, "pv_ray_directions: rays must be 1..%d and out non-NULL",
                        PV_MAX_RAYS);
  uint64_t key = stream_at(stream_at(stream_at(seed, kKindRotation), volume), frame);
  const double u1 = unit(stream_at(key, 0)), u2 = unit(stream_at(key, 1)), u3 = unit(stream_at(key, 2));
  const double pi = 3.141592653589793;
  const double s1 = sqrt(1.0 - u1), s2 = sqrt(u1);
  const double x = s1 * sin(2.0 * pi * u2), y = s1 * cos(2.0 * pi * u2);
  const double z = s2 * sin(2.0 * pi * u3), w = s2 * cos(2.0 * pi * u3);
  const double m[3][3] = {
      {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y)},
      {2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x)},
      {2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)}};
  const double g = (sqrt(5.0) - 1.0) / 2.0;
  for (int i = 0; i < rays; ++i) {
    const double fz = 1.0 - (2.0 * i + 1.0) / rays;
    const double rxy = sqrt(fmax(0.0, 1.0 - fz * fz));
    const double phi = 2.0 * pi * fmod(i * g, 1.0);
    const double f[3] = {rxy * cos(phi), rxy * sin(phi), fz};
    for (int r = 0; r < 3; ++r)
      out[3 * i + r] = (float)(m[r][0] * f[0] + m[r][1] * f[1] + m[r][2] * f[2]);
  }
  return PV_OK;
}
