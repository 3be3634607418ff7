"""GPU parity tests: the CUDA path, called through the C ABI, against the FP64 oracle.

Tolerances (each derived from the arithmetic: 3xTF32 products carry <= 2^-21 relative error
and FP32 accumulation over <= 1024 terms stays below 1e-5 on the normalised mean; the 16-bit
operand forms carry the weights' and inputs' rounding, the precision form's 2e-3 budget):
  * blended mean m, FP32 operands:      relative error <= 1e-5 vs FP64
  * blended mean m, FP16/BF16 operands: relative error <= 2e-3 vs FP64
  * FP16 state, one frame from identical texels: <= 1 binary16 ulp per texel
  * FP32 state, free-running over all frames:    relative error <= 1e-5
  * selection, index buffers, packed planes, last-transmitted codes: bit-exact
    given identical texels (the oracle is loaded with the GPU's texels).
relative error = |got - ref| / max(|ref|, 1e-6 * max|ref|).
"""
import os

import numpy as np
import pytest
import torch

import pv_workload as wl
from oracle import OracleVolume, blend, numerics, octahedral, select_pack
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _spec(**kw):
    base = dict(nx=4, ny=4, nz=4, rays=64, state_fmt="f32", operand_fmt="f32")
    base.update(kw)
    return wl.VolumeSpec(**base)


def _check_step(spec, vol, fs, frame, kernel_tol):
    """One frame: blend from identical texels, then select/pack from identical texels."""
    ov = H.oracle_from_gpu(spec, vol)
    (rad, dist, dirs), exact = H.device_inputs(fs, frame)
    vol.update(rad, dist, dirs)
    ov.update(*exact)
    tc, tv, lc, lv, _ = H.gpu_state(vol)
    if spec.state_fmt == "f16":
        assert H.fp16_ulp_diff(tc, ov.tiles_c).max() <= 1
        assert H.fp16_ulp_diff(tv, ov.tiles_v).max() <= 1
    else:
        assert H.rel_err(tc, ov.tiles_c).max() <= kernel_tol
        assert H.rel_err(tv, ov.tiles_v).max() <= kernel_tol
    # guard band holds the reflected interior on the GPU too
    np.testing.assert_array_equal(octahedral.fill_border(tc), tc)
    np.testing.assert_array_equal(octahedral.fill_border(tv), tv)
    # selection and packing from the GPU's own texels must be bit-exact
    og = OracleVolume(spec)
    og.load_state(tc, tv, lc, lv, frame=frame + 1)
    fr_o = og.select_and_pack()
    fr_g = vol.select_and_pack()
    H.assert_frames_equal(H.gpu_frame(vol, fr_g), fr_o)
    _, _, lc2, lv2, _ = H.gpu_state(vol)
    np.testing.assert_array_equal(lc2, og.last_c)
    np.testing.assert_array_equal(lv2, og.last_v)
    return fr_o


CHAIN_CASES = {
    "config1_fp32": (_spec(), 10, "noisy"),
    "ragged_fp16": (_spec(nx=3, ny=5, nz=7, rays=37, state_fmt="f16"), 5, "noisy"),
    "ragged_k_fp16": (_spec(nx=5, ny=7, nz=9, rays=36, state_fmt="f16"), 4, "noisy"),
    "bf16_operands": (_spec(nx=6, ny=5, nz=4, rays=64, state_fmt="f16", operand_fmt="bf16"), 3, "noisy"),
    "f16_operands": (_spec(nx=6, ny=5, nz=4, rays=64, state_fmt="f16", operand_fmt="f16"), 3, "noisy"),
    "single_probe": (_spec(nx=1, ny=1, nz=1, rays=8), 3, "noisy"),
    "paper_tiles_10x10_18x18": (_spec(nx=4, ny=2, nz=3, rays=96, color_interior=8, vis_interior=16,
                                      state_fmt="f16"), 4, "noisy"),
    "unorm10_lsb": (_spec(nx=2, ny=3, nz=4, rays=48, color_code="unorm10", color_lsb=True), 3, "noisy"),
    "stationary_first_frame": (_spec(state_fmt="f16", first_frame_no_hysteresis=True), 4, "stationary"),
    # the largest shapes: 1024 rays (64 K chunks of 16), and 65,536 probes (the whole 2-byte
    # index range, 2,048 mask words, many items per CTA)
    "max_rays_1024": (_spec(nx=2, ny=2, nz=2, rays=1024, state_fmt="f16"), 2, "noisy"),
    "max_probes_65536": (_spec(nx=256, ny=16, nz=16, rays=8, state_fmt="f16"), 1, "noisy"),
}


@pytest.mark.parametrize("kernel", ["simt", "auto"])
@pytest.mark.parametrize("case", list(CHAIN_CASES))
def test_chain_step_by_step(case, kernel):
    spec, frames, mode = CHAIN_CASES[case]
    vol = H.lib().ProbeVolume(spec, kernel=kernel)
    fs = wl.FrameStream(spec, wl.config_seed(1) + len(case), mode=mode, step_frame=2)
    free = OracleVolume(spec)
    for f in range(frames):
        _check_step(spec, vol, fs, f, 1e-5)
        _, exact = H.device_inputs(fs, f)
        free.step(*exact)
    tc, tv, *_ = H.gpu_state(vol)
    if spec.operand_fmt != "f32":
        # 16-bit operands: the state is an average of means each within 2e-3, plus
        # one binary16 rounding (2^-11) per stored value
        assert H.rel_err(tc, free.tiles_c).max() <= 2e-3 + 2.0 ** -11
        assert H.rel_err(tv, free.tiles_v).max() <= 2e-3 + 2.0 ** -11
    elif spec.state_fmt == "f32":
        assert H.rel_err(tc, free.tiles_c).max() <= 1e-5
        assert H.rel_err(tv, free.tiles_v).max() <= 1e-5
    else:
        assert H.fp16_ulp_diff(tc, free.tiles_c).max() <= 1
        assert H.fp16_ulp_diff(tv, free.tiles_v).max() <= 1
    vol.close()


@pytest.mark.parametrize("kernel", ["simt", "auto"])
@pytest.mark.parametrize("operand_fmt,tol", [("f32", 1e-5), ("f16", 2e-3), ("bf16", 2e-3)])
def test_blend_mean_accuracy_full_size(operand_fmt, tol, kernel):
    """h = 0 and FP32 state: the stored texel is the frame mean m. 16^3 probes x 256 rays."""
    spec = wl.VolumeSpec(16, 16, 16, 256, hysteresis=0.0, state_fmt="f32", operand_fmt=operand_fmt)
    vol = H.lib().ProbeVolume(spec, kernel=kernel)
    fs = wl.FrameStream(spec, wl.config_seed(3))
    (rad, dist, dirs), exact = H.device_inputs(fs, 0)
    vol.update(rad, dist, dirs)
    tc, tv, *_ = H.gpu_state(vol)
    m_c, m_v = blend.blend_means(*exact, 6, 14, 50.0)
    ec = H.rel_err(octahedral.interior(tc), m_c)
    ev = H.rel_err(octahedral.interior(tv), m_v)
    line = (f"{operand_fmt}/{vol.kernel}: colour max {ec.max():.3e} mean {ec.mean():.3e}; "
            f"visibility max {ev.max():.3e} mean {ev.mean():.3e}")
    print("\n" + line)
    out = os.environ.get("PV_ACCURACY_LOG")            # optional: append the figures to a file
    if out:
        with open(out, "a") as f:
            f.write(line + "\n")
    assert ec.max() <= tol
    assert ev.max() <= tol
    vol.close()


def _selection_from_tiles(spec, tc, tv, lc0, lv0, lc1, lv1, g):
    """Section 3.4 applied to the GPU's own new tiles: the codes of its stored texels against
    its last-transmitted codes before the frame give the probes to send, their delta-coded
    indices and planes, and the last codes after the frame; all must equal the GPU's."""
    bw, bh = select_pack.block_grid(spec.nx, spec.ny, spec.nz)
    codes_c = select_pack.color_codes(tc, spec.color_code)
    codes_v = select_pack.vis_codes(tv)
    for codes, last0, last1, key, pack in (
            (codes_c, lc0, lc1, "c", lambda c, i: select_pack.pack_color(c, i, bw, bh, spec.color_lsb)),
            (codes_v, lv0, lv1, "v", lambda c, i: select_pack.pack_vis(c, i, bw, bh))):
        flags = select_pack.changed(codes, last0, ~np.all(last0 == select_pack.SENTINEL, axis=(0, 2)))
        idx, delta, n = select_pack.select(flags)
        assert g["count_" + key] == n
        np.testing.assert_array_equal(g["idx_" + key], idx)
        np.testing.assert_array_equal(g["delta_" + key], delta)
        np.testing.assert_array_equal(g["planes_" + key], pack(codes, idx))
        want = last0.copy()
        want[:, idx] = codes[:, idx]
        np.testing.assert_array_equal(last1, want)
    return codes_c, codes_v


def test_config2_sixty_frames_with_step_change():
    """16^3 probes, 256 rays, FP16 state, 60 frames, 20% of probes x4 at frame 30; rays held
    fixed and the first frame taken without hysteresis (converged server, Section 3.4). At every
    frame the GPU's tiles stay within one binary16 ulp of the free-running oracle's, and its
    selection, indices, planes and last-code update equal the oracle's rule applied to the
    GPU's own tiles, bit for bit."""
    import dataclasses
    spec = dataclasses.replace(wl.config2(), first_frame_no_hysteresis=True)
    vol = H.lib().ProbeVolume(spec)
    fs = wl.FrameStream(spec, wl.config_seed(2), mode="stationary")
    free = OracleVolume(spec)
    counts = []
    for f in range(60):
        *_, lc0, lv0, _ = H.gpu_state(vol)
        (rad, dist, dirs), exact = H.device_inputs(fs, f)
        vol.update(rad, dist, dirs)
        fr = vol.select_and_pack(want_host_counts=True)
        fo = free.step(*exact)
        counts.append((fr.count_c, fr.count_v, fo.count_c, fo.count_v))
        tc, tv, lc1, lv1, _ = H.gpu_state(vol)
        _selection_from_tiles(spec, tc, tv, lc0, lv0, lc1, lv1, H.gpu_frame(vol, fr))
        assert H.fp16_ulp_diff(tc, free.tiles_c).max() <= 1
        assert H.fp16_ulp_diff(tv, free.tiles_v).max() <= 1
    c = np.array(counts)
    assert c[0, 0] == c[0, 1] == 4096
    assert c[1:30, 0].max() == 0 and c[1:, 1].max() == 0      # converged: nothing to resend
    stepped = wl.step_mask(wl.config_seed(2), 0, 4096, 0.2).sum()
    assert c[30, 0] >= stepped and c[30, 1] == 0
    # against the free-running oracle the counts agree to within a handful: a texel one
    # binary16 ulp away can sit on the other side of a code boundary
    assert np.abs(c[:, 0] - c[:, 2]).max() <= max(8, 0.01 * 4096)
    vol.close()


def test_import_state_select_pack_bit_exact():
    """Random FP16 texels, last codes partly equal: selection and packing bit-exact."""
    rng = np.random.default_rng(5)
    spec = _spec(nx=8, ny=4, nz=5, rays=64, state_fmt="f16")
    vol = H.lib().ProbeVolume(spec)
    P = spec.probes
    tc = numerics.round_fp16(rng.lognormal(0, 2, (3, P, 8, 8)))
    tv = numerics.round_fp16(rng.uniform(0.1, 100, (2, P, 16, 16)))
    tc = octahedral.fill_border(tc)
    tv = octahedral.fill_border(tv)
    lc = select_pack.color_codes(tc)
    lv = select_pack.vis_codes(tv)
    for p in rng.choice(P, 40, replace=False):        # changed probes
        lc[rng.integers(0, 3), p, rng.integers(0, 36)] ^= 1
    for p in rng.choice(P, 15, replace=False):        # never sent
        lc[:, p] = 0xFFFF
    for p in rng.choice(P, 30, replace=False):
        lv[rng.integers(0, 2), p, rng.integers(0, 196)] ^= 0x100
    vol.import_state(torch.from_numpy(tc.astype(np.float16)), torch.from_numpy(tv.astype(np.float16)),
                     torch.from_numpy(lc.view(np.int16)), torch.from_numpy(lv.view(np.int16)), frame=7)
    og = OracleVolume(spec)
    og.load_state(tc, tv, lc, lv, frame=7)
    for rep in range(2):                              # second call: nothing left to send
        fr_o = og.select_and_pack()
        fr_g = vol.select_and_pack()
        g = H.gpu_frame(vol, fr_g)
        H.assert_frames_equal(g, fr_o)
        if rep == 1:
            assert g["count_c"] == 0 and g["count_v"] == 0
            assert not g["planes_c"].any() and not g["planes_v_full"].any()
    vol.close()


@pytest.mark.parametrize("state_fmt", ["f16", "f32"])
@pytest.mark.parametrize("code", ["uf10", "unorm10"])
def test_codes_exhaustive_through_packing(state_fmt, code):
    """Every binary16 pattern (and random binary32 patterns) as colour texels: the packed
    samples equal the oracle's codes."""
    rng = np.random.default_rng(9)
    if state_fmt == "f16":
        vals = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16).view(np.float16).astype(np.float64)
    else:
        bits = rng.integers(0, 1 << 32, 60000, dtype=np.uint64).astype(np.uint32)
        extra = np.array([0, 1, 0x00800000, 0x38800000, 0x387FFFFF, 0x477FE000, 0x477FF000, 0x7F800000,
                          0x7FC00000, 0x80000000, 0x3F800000, 0x3F7FFFFF], dtype=np.uint32)
        vals = np.concatenate([bits, extra]).view(np.float32).astype(np.float64)
    P = -(-len(vals) // (3 * 36))
    nx = 8
    nz = -(-P // nx)
    spec = _spec(nx=nx, ny=1, nz=nz, rays=8, state_fmt=state_fmt, color_code=code)
    P = spec.probes
    flat = np.zeros(3 * P * 36)
    flat[:len(vals)] = vals
    tc = np.zeros((3, P, 8, 8))
    tc[:, :, 1:7, 1:7] = flat.reshape(3, P, 6, 6)
    tv = np.zeros((2, P, 16, 16))
    vol = H.lib().ProbeVolume(spec)
    dt = np.float16 if state_fmt == "f16" else np.float32
    lc = np.full((3, P, 36), 0xFFFF, dtype=np.uint16)
    lv = np.full((2, P, 196), 0xFFFF, dtype=np.uint16)
    with np.errstate(over="ignore", invalid="ignore"):
        vol.import_state(torch.from_numpy(tc.astype(dt)), torch.from_numpy(tv.astype(dt)),
                         torch.from_numpy(lc.view(np.int16)), torch.from_numpy(lv.view(np.int16)), 0)
    fr = vol.select_and_pack()
    g = H.gpu_frame(vol, fr)
    og = OracleVolume(spec)
    og.load_state(tc, tv, lc, lv)
    fo = og.select_and_pack()
    np.testing.assert_array_equal(g["planes_c"], fo.planes_c)
    vol.close()


def test_host_buffer_path_matches_device_path():
    spec = _spec(nx=4, ny=4, nz=2, rays=32, state_fmt="f16")
    a = H.lib().ProbeVolume(spec)
    b = H.lib().ProbeVolume(spec)
    fs = wl.FrameStream(spec, 3)
    pv = H.lib()
    info = a.info
    for f in range(3):
        (rad, dist, dirs), _ = H.device_inputs(fs, f)
        a.update(rad, dist, dirs)
        fa = a.select_and_pack(want_host_counts=True)
        pv.probe_update_host(b.handle, rad.cpu().pin_memory(), dist.cpu().pin_memory(), dirs.cpu())
        b.select_and_pack()
        color = np.zeros((3, info.color_height, info.color_width), dtype=np.uint16)
        vis = np.zeros((3, info.vis_height, info.vis_width), dtype=np.uint8)
        dc = np.zeros(spec.probes, dtype=np.uint16)
        dv = np.zeros(spec.probes, dtype=np.uint16)
        counts = np.zeros(2, dtype=np.uint32)
        pv.probe_frame_download(b.handle, color, vis, dc, dv, counts)
        g = H.gpu_frame(a, fa)
        assert counts[0] == g["count_c"] and counts[1] == g["count_v"]
        np.testing.assert_array_equal(color, g["planes_c"])
        np.testing.assert_array_equal(vis, g["planes_v"])
        np.testing.assert_array_equal(dc[:counts[0]], g["delta_c"])
        np.testing.assert_array_equal(dv[:counts[1]], g["delta_v"])
    a.close()
    b.close()


def test_pipelined_host_path_matches_device_path():
    """Uploads on the volume's copy stream into alternating staging halves and downloads
    queued on its second stream, frame f+1 queued before frame f is waited for: every
    frame must equal the device-buffer path's, the next select waiting for the download
    of the planes it rewrites."""
    spec = _spec(nx=6, ny=4, nz=5, rays=64, state_fmt="f16")
    pv = H.lib()
    a = pv.ProbeVolume(spec)
    b = pv.ProbeVolume(spec)
    fs = wl.FrameStream(spec, 9)
    info = a.info
    frames = 6
    host_in, expect = [], []
    for f in range(frames):
        (rad, dist, dirs), _ = H.device_inputs(fs, f)
        host_in.append((rad.cpu().pin_memory(), dist.cpu().pin_memory(), dirs.cpu().pin_memory()))
        a.update(rad, dist, dirs)
        expect.append(H.gpu_frame(a, a.select_and_pack(want_host_counts=True)))

    def bufs():
        return (torch.zeros((3, info.color_height, info.color_width), dtype=torch.int16).pin_memory(),
                torch.zeros((3, info.vis_height, info.vis_width), dtype=torch.uint8).pin_memory(),
                torch.zeros(spec.probes, dtype=torch.int16).pin_memory(),
                torch.zeros(spec.probes, dtype=torch.int16).pin_memory(),
                torch.zeros(2, dtype=torch.int32).pin_memory())
    out = [bufs(), bufs()]

    def check(f):
        color, vis, dc, dv, counts = out[f % 2]
        g = expect[f]
        nc, nv = int(counts[0]), int(counts[1])
        assert nc == g["count_c"] and nv == g["count_v"]
        np.testing.assert_array_equal(color.numpy().view(np.uint16), g["planes_c"])
        np.testing.assert_array_equal(vis.numpy(), g["planes_v"])
        np.testing.assert_array_equal(dc.numpy().view(np.uint16)[:nc], g["delta_c"])
        np.testing.assert_array_equal(dv.numpy().view(np.uint16)[:nv], g["delta_v"])

    tickets = []
    for f in range(frames):
        pv.probe_update_host(b.handle, *host_in[f])
        b.select_and_pack()
        tickets.append(pv.probe_frame_download_async(b.handle, *out[f % 2]))
        if f:
            pv.probe_frame_wait(b.handle, tickets[f - 1])
            check(f - 1)
    pv.probe_frame_wait(b.handle, tickets[-1])
    check(frames - 1)
    assert tickets == list(range(1, frames + 1))
    with pytest.raises(pv.PVError) as e:
        pv.probe_frame_wait(b.handle, frames + 1)
    assert e.value.status == -1
    a.close()
    b.close()


def test_invalid_arguments_return_errors():
    pv = H.lib()
    with pytest.raises(pv.PVError) as e:
        pv.ProbeVolume(_spec(nx=0))
    assert e.value.status == -1
    with pytest.raises(pv.PVError) as e:
        pv.ProbeVolume(_spec(nx=256, ny=256, nz=2))
    assert e.value.status == -6
    vol = pv.ProbeVolume(_spec())
    with pytest.raises(pv.PVError):
        pv.probe_update(vol.handle, None, None, None)
    vol.close()
