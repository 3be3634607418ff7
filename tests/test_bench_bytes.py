"""The algorithmic byte counts the bench divides by (CPU only): each restated from what the
kernel must move at the 16^3-probe, 256-ray workload, and the totals the profiles quote.

Blend, per probe (Section 3.2, one update): the R rays of R, G, B and distance read once,
the interior texels of the stored state read (hysteresis), the whole tiles written back
(interior and guard band, Section 3.4), the last-transmitted codes read for the change
test, and five flag bytes. Client decode (Sections 3.3-3.4), every probe selected: the
three colour planes and three visibility byte planes read, both delta buffers read, the
float32 colour and binary16 visibility tiles written."""
import os
import sys

import pv_workload as wl

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_blend_bytes_per_probe_follow_their_definition():
    R = 256
    interior = 3 * 6 * 6 + 2 * 14 * 14            # colour and visibility texels per probe
    tiles = 3 * 8 * 8 + 2 * 16 * 16               # with the one-texel guard band
    for op_bytes in (4, 2):
        rays = 4 * R * op_bytes                   # R, G, B, distance
        want = rays + 2 * interior + 2 * tiles + 2 * interior + 5   # binary16 state and codes
        assert bench.blend_bytes_per_probe(R, op_bytes) == want
    assert bench.blend_bytes_per_probe(R, 4) == 7509
    assert bench.blend_bytes_per_probe(R, 2) == 5461


def test_blend_bytes_per_launch_match_the_profiles():
    P = 16 ** 3
    weights = (36 + 196) * 256                    # shared weight images, one value per texel and ray
    assert bench.blend_bytes_per_probe(256, 4) * P + weights * 8 == 31_232_000      # FP32: hi + lo float
    assert bench.blend_bytes_per_probe(256, 2) * P + weights * 2 == 22_487_040      # FP16: one binary16


def test_client_bytes_follow_their_definition():
    spec = wl.config2()
    P, bw, bh = spec.probes, spec.nx * spec.ny, spec.nz
    colour_planes = 3 * (bh * 6) * (bw * 6) * 2                   # 16-bit samples
    vis_stream = 4 * bw * 14                                      # RG16F bytes per atlas row
    vis_planes = 3 * (bh * 14) * -(-vis_stream // 3)              # one third of each row per plane
    deltas = 2 * P * 2
    tiles = P * (3 * 8 * 8 * 4 + 2 * 16 * 16 * 2)
    assert (colour_planes, vis_planes, deltas, tiles) == (884_736, 3_211_488, 16_384, 7_340_032)
    assert bench.client_bytes(spec) == colour_planes + vis_planes + deltas + tiles == 11_452_640
    assert bench.client_tex_bytes(spec) == tiles
