"""Pins of selection, index buffer and bit packing: round trips, literal layouts, invariants."""
import json
import math
import os

import numpy as np
import pytest

import pv_workload as wl
from oracle import OracleVolume, numerics, octahedral, select_pack as sp

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _rand_codes(rng, P, n_c, n_v):
    cc = rng.integers(0, 0x3E0, size=(3, P, n_c * n_c)).astype(np.uint16)
    cv = rng.integers(0, 1 << 16, size=(2, P, n_v * n_v)).astype(np.uint16)
    return cc, cv


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 2, 5), (1, 1, 1), (16, 16, 2)])
@pytest.mark.parametrize("frac", [0.0, 0.3, 1.0])
def test_pack_unpack_round_trip(dims, frac):
    rng = np.random.default_rng(hash((dims, frac)) & 0xFFFF)
    nx, ny, nz = dims
    P, n_c, n_v = nx * ny * nz, 6, 14
    bw, bh = sp.block_grid(nx, ny, nz)
    cc, cv = _rand_codes(rng, P, n_c, n_v)
    flags = rng.random(P) < frac
    idx, delta, count = sp.select(flags)
    np.testing.assert_array_equal(sp.undelta(delta), idx)
    assert count == flags.sum()
    for lsb in (False, True):
        pc = sp.pack_color(cc, idx, bw, bh, lsb)
        np.testing.assert_array_equal(sp.unpack_color(pc, idx, n_c, bw, lsb), cc[:, idx.astype(int)])
    pv = sp.pack_vis(cv, idx, bw, bh)
    np.testing.assert_array_equal(sp.unpack_vis(pv, idx, n_v, bw), cv[:, idx.astype(int)])
    # sizes: colour 3 x (bh n_c) x (bw n_c) 16-bit; visibility 3 x (bh n_v) x ceil(4 bw n_v / 3) 8-bit
    assert pc.shape == (3, bh * n_c, bw * n_c) and pc.dtype == np.uint16
    assert pv.shape == (3, bh * n_v, math.ceil(4 * bw * n_v / 3)) and pv.dtype == np.uint8


def test_unused_slots_and_pad_bytes_are_zero():
    rng = np.random.default_rng(2)
    nx, ny, nz = 4, 4, 4
    bw, bh = sp.block_grid(nx, ny, nz)
    cc, cv = _rand_codes(rng, 64, 6, 14)
    cv |= 0x0101    # no zero bytes in real data
    idx, _, count = sp.select(np.arange(64) % 3 == 0)
    pc = sp.pack_color(cc, idx, bw, bh)
    pv = sp.pack_vis(cv, idx, bw, bh)
    k = count
    by, bx = divmod(k, bw)
    assert np.all(pc[:, by * 6:(by + 1) * 6, bx * 6:] == 0)
    assert np.all(pc[:, (by + 1) * 6:, :] == 0)
    W = bw * 14
    assert 4 * W % 3 != 0 or True
    nbytes = 4 * W
    # plane q holds bytes q, q+3, ...: plane 2 is short by one byte when 4W = 2 mod 3
    for q in range(3):
        used = len(range(q, nbytes, 3))
        assert np.all(pv[q, :, used:] == 0)


def test_colour_codes_sit_in_the_top_ten_bits():
    cc = np.arange(0x3E0, dtype=np.uint16).reshape(1, 1, -1).repeat(3, 0)
    cc = cc[:, :, :36]
    idx = np.array([0], dtype=np.uint16)
    pc = sp.pack_color(cc, idx, 1, 1)
    assert np.all(pc & 0x3F == 0)
    assert GOLDEN["color_bits_used_of_16"]["value"] == 10
    assert np.all((pc >> 6) < 1024)
    np.testing.assert_array_equal(pc[0].ravel() >> 6, cc[0, 0])


def test_visibility_byte_order_is_yuvy_uvyu_vyuv():
    """Three texels with distinct bytes land in Y,U,V as YUVY / UVYU / VYUV."""
    n = 1
    # texel t has R = (lo=4t+1, hi=4t+2), G = (lo=4t+3, hi=4t+4)
    cv = np.zeros((2, 3, 1), dtype=np.uint16)
    for t in range(3):
        cv[0, t, 0] = (4 * t + 1) | ((4 * t + 2) << 8)
        cv[1, t, 0] = (4 * t + 3) | ((4 * t + 4) << 8)
    idx = np.array([0, 1, 2], dtype=np.uint16)
    pv = sp.pack_vis(cv, idx, bw=3, bh=1)
    assert pv.shape == (3, 1, 4)          # x = 3 texels -> x' = ceil(4*3/3) = 4
    seq = []
    for k in range(12):                   # walk the byte stream through the planes
        q, col = k % 3, k // 3
        seq.append(("YUV"[q], int(pv[q, 0, col])))
    letters = "".join(c for c, _ in seq)
    assert [letters[0:4], letters[4:8], letters[8:12]] == GOLDEN["byte_order_over_three_texels"]["value"]
    assert [v for _, v in seq] == list(range(1, 13))


@pytest.mark.parametrize("x", [1, 2, 3, 4, 5, 14, 84, 3584])
def test_widened_width_is_ceil_four_thirds(x):
    assert sp.vis_width(x, 1) == math.ceil(4 * x / 3) == -(-4 * x // 3)


def test_paper_sizes_eq1_eq2_and_tables():
    g = GOLDEN
    kb, Mb, MB = 1024, 1024 * 1024, 1024 * 1024
    assert sp.full_tile_bits(10) / kb == g["irradiance_kb_per_probe"]["value"]
    assert sp.full_tile_bits(18) / kb == g["visibility_kb_per_probe"]["value"]
    assert 2048 * sp.full_tile_bits(10) / Mb == g["irradiance_texture_2048_probes_Mb"]["value"]
    assert round(2048 * sp.full_tile_bits(10) / 8 / MB, 2) == g["irradiance_texture_2048_probes_MB"]["value"]
    assert 10 * 2048 * sp.full_tile_bits(10) / Mb == g["irradiance_2048_at_10Hz_Mbps"]["value"]
    vis_mb = 2048 * sp.full_tile_bits(18) / Mb
    assert abs(vis_mb - g["visibility_texture_2048_probes_Mb"]["value"]) <= 0.05 + 1e-9
    assert abs(sp.full_tile_bits(18) / sp.full_tile_bits(10) - g["visibility_to_irradiance_ratio"]["value"]) <= 0.005
    assert 10 * vis_mb == g["visibility_2048_at_10Hz_Mbps"]["value"]
    assert abs(10 * (vis_mb + 2048 * sp.full_tile_bits(10) / Mb) - g["total_2048_at_10Hz_Mbps"]["value"]) <= 0.5
    for P, want in zip(g["uncompressed_color_MB"]["probes"], g["uncompressed_color_MB"]["value"]):
        assert abs(P * sp.full_tile_bits(10) / 8 / MB - want) <= 0.005 + 1e-9
    for P, want in zip(g["uncompressed_visibility_MB"]["probes"], g["uncompressed_visibility_MB"]["value"]):
        assert abs(P * sp.full_tile_bits(18) / 8 / MB - want) <= 0.005 + 1e-9


def test_guard_band_savings_section_3_4():
    g = GOLDEN
    sc = 1 - (8 * 8) / (10 * 10)
    sv = 1 - (16 * 16) / (18 * 18)
    assert sc == pytest.approx(g["guard_band_saving_irradiance"]["value"], abs=1e-12)
    assert abs(sv - g["guard_band_saving_visibility"]["value"]) <= 0.005
    # combined with 75% active probes
    assert abs(1 - 0.75 * (1 - sc) - g["combined_saving_irradiance"]["value"]) <= 0.005
    assert abs(1 - 0.75 * (1 - sv) - g["combined_saving_visibility"]["value"]) <= 0.0005
    # packed payload per probe equals the interior share of Eq. 1 / Eq. 2 tiles
    bc, bv = sp.packed_bytes(1, 8, 16)
    assert 8 * bc / 3 * 2 == pytest.approx(8 * 8 * 32)     # 3 x 10-bit codes in 32 bits of A2RGB10
    assert 8 * bv == 16 * 16 * 32


def test_selection_invariants_over_a_stationary_run():
    """Frame 0 selects every probe; unchanged frames select none; a step change selects
    at least the stepped probes (colour) and no visibility probe."""
    spec = wl.VolumeSpec(4, 4, 4, 64, state_fmt="f16", first_frame_no_hysteresis=True)
    fs = wl.FrameStream(spec, 99, mode="stationary", step_frame=4, step_fraction=0.25)
    ov = OracleVolume(spec)
    stepped = wl.step_mask(99, 0, 64, 0.25)
    for f in range(7):
        fr = ov.step(fs.radiance(f), fs.dist(f), fs.directions(f))
        if f == 0:
            assert fr.count_c == fr.count_v == 64
        elif f < 4:
            assert fr.count_c == 0 and fr.count_v == 0
        else:
            assert set(np.nonzero(stepped)[0]) <= set(fr.idx_c.astype(int))
            assert fr.count_v == 0
        # the last-transmitted texture now equals the current codes for every sent probe
        cc, cv = ov.codes()
        np.testing.assert_array_equal(ov.last_c, cc)
        np.testing.assert_array_equal(ov.last_v, cv)


def test_selection_equals_brute_force_texel_comparison():
    rng = np.random.default_rng(8)
    P = 50
    last = rng.integers(0, 4, size=(3, P, 36)).astype(np.uint16)
    codes = last.copy()
    hit = rng.random(P) < 0.4
    for p in np.nonzero(hit)[0]:
        c, t = rng.integers(0, 3), rng.integers(0, 36)
        codes[c, p, t] ^= 1
    sent = rng.random(P) < 0.9
    f = sp.changed(codes, last, sent)
    for p in range(P):
        want = (not sent[p]) or any(codes[c, p, t] != last[c, p, t] for c in range(3) for t in range(36))
        assert bool(f[p]) == want


def test_client_round_trip_recovers_server_textures():
    """pack -> unpack -> client apply reproduces the server's stored texels (guard band too)."""
    spec = wl.VolumeSpec(3, 2, 2, 64, state_fmt="f16")
    fs = wl.FrameStream(spec, 4)
    ov = OracleVolume(spec)
    client_c = np.zeros_like(ov.tiles_c)
    client_v = np.zeros_like(ov.tiles_v)
    for f in range(3):
        fr = ov.step(fs.radiance(f), fs.dist(f), fs.directions(f))
        idx_c = sp.undelta(fr.delta_c)
        idx_v = sp.undelta(fr.delta_v)
        cc = sp.unpack_color(fr.planes_c, idx_c, 6, ov.bw)
        cv = sp.unpack_vis(fr.planes_v, idx_v, 14, ov.bw)
        client_c = sp.client_apply(client_c, idx_c, numerics.uf10_value(cc))
        client_v = sp.client_apply(client_v, idx_v, numerics.fp16_value(cv))
        np.testing.assert_array_equal(client_v, ov.tiles_v)                 # lossless RG16F
        np.testing.assert_array_equal(numerics.uf10_code(client_c), numerics.uf10_code(ov.tiles_c))


# ----------------------------------------------------------------- per-client selection knobs
def test_threshold_zero_is_the_texel_for_texel_rule():
    rng = np.random.default_rng(5)
    codes = rng.integers(0, 1024, (3, 40, 9)).astype(np.uint16)
    last = codes.copy()
    last[:, ::3] ^= 1                                    # one code step apart
    sent = rng.random(40) < 0.8
    np.testing.assert_array_equal(sp.changed_beyond(codes, last, sent, 0), sp.changed(codes, last, sent))


def test_threshold_brute_force():
    rng = np.random.default_rng(6)
    codes = rng.integers(0, 1024, (2, 25, 4)).astype(np.uint16)
    last = (codes.astype(np.int64) + rng.integers(-3, 4, codes.shape)).clip(0, 1023).astype(np.uint16)
    sent = np.ones(25, dtype=bool)
    sent[7] = False
    for th in range(5):
        want = [not sent[p] or any(abs(int(codes[c, p, t]) - int(last[c, p, t])) > th
                                   for c in range(2) for t in range(4)) for p in range(25)]
        np.testing.assert_array_equal(sp.changed_beyond(codes, last, sent, th), want)
    # a never-sent probe (sentinel codes) is changed at any threshold
    assert sp.changed_beyond(codes, np.full_like(codes, sp.SENTINEL), np.zeros(25, bool), 1000).all()


def test_budget_round_robin_sends_each_changed_probe_once_per_cycle():
    P, B = 23, 5
    flags = np.zeros(P, dtype=bool)
    flags[[0, 2, 3, 7, 8, 9, 11, 15, 16, 20, 22]] = True
    cursor, frames = 0, []
    for _ in range(3):                                   # 11 changed probes, 5 per frame
        kept, cursor = sp.budget_select(flags, None, cursor, B)
        assert kept.sum() <= B and not (kept & ~flags).any()
        frames.append(list(np.nonzero(kept)[0]))
    assert frames[0] == [0, 2, 3, 7, 8] and frames[1] == [9, 11, 15, 16, 20]
    assert frames[2] == [0, 2, 3, 7, 22]                 # 22 ends the cycle, 0, 2, 3, 7 start the next
    assert sorted(frames[0] + frames[1] + [22]) == list(np.nonzero(flags)[0])
    assert cursor == 8
    # no budget, or a budget above the count, keeps every changed probe and the cursor
    for b in (0, 11, 40):
        kept, c = sp.budget_select(flags, None, 4, b)
        np.testing.assert_array_equal(kept, flags)
        assert c == 4                                    # one past the last kept probe, cyclically from 4


def test_active_mask_excludes_inactive_probes():
    flags = np.ones(10, dtype=bool)
    active = np.array([1, 0, 1, 1, 0, 0, 1, 0, 1, 1], dtype=bool)
    kept, _ = sp.budget_select(flags, active, 0, 0)
    np.testing.assert_array_equal(kept, active)
    kept, c = sp.budget_select(flags, active, 3, 2)
    np.testing.assert_array_equal(np.nonzero(kept)[0], [3, 6])
    assert c == 7


def test_oracle_volume_budget_catches_up_over_frames():
    """With a budget, probes left out stay changed and go out on the next frames; the
    client's texels end equal to the full selection's after enough frames."""
    spec = wl.VolumeSpec(3, 2, 2, 16, hysteresis=0.0, state_fmt="f16")
    fs = wl.FrameStream(spec, 3, mode="stationary")
    full, lim = OracleVolume(spec), OracleVolume(spec)
    counts = []
    for f in range(5):
        args = tuple(np.asarray(x, dtype=np.float64) for x in (fs.radiance(f), fs.dist(f), fs.directions(f)))
        full.update(*args)
        lim.update(*args)
        full.select_and_pack()
        fr = lim.select_and_pack(budget=5)
        counts.append(fr.count_c)
    assert counts[:3] == [5, 5, 2] and counts[3:] == [0, 0]
    np.testing.assert_array_equal(lim.last_c, full.last_c)
    np.testing.assert_array_equal(lim.last_v, full.last_v)
