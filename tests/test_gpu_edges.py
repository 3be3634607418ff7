"""Edge cases forced on the tensor-core blend, against the FP64 oracle.

* Rays confined to a cap of the sphere (16 and 32 rays, so the tcgen05 kernel takes the
  shape): texels with no ray in their hemisphere have weight sum 0 and keep their old
  value bit for bit (the reading of Section 3.2 for an undefined mean); every other texel,
  including those whose best ray is far off axis, follows the oracle.
* Visibility weights cos^50 far below the binary16 (and float32) range: the weights kernel
  scales each texel's weights by its largest cosine, so such texels still follow the oracle.
* Checkpoint / resume: state exported mid-run and imported into a fresh volume gives the
  very same following frames (texels, codes and packed output) as the volume that never
  stopped.
* The error word of the bounded waits: set from the host, it is reported by
  probe_select_and_pack(want_host_counts) as PV_ERR_TIMEOUT once, and cleared.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import pv_workload as wl
from oracle import OracleVolume, blend, octahedral
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _cap_dirs(R: int, z_min: float, turn: float) -> np.ndarray:
    """R float32 unit directions with z in [z_min, 1): a golden-angle spiral over the cap,
    turned by `turn` radians about z."""
    i = np.arange(R, dtype=np.float64) + 0.5
    z = 1.0 - (1.0 - z_min) * i / R
    phi = i * np.pi * (3.0 - np.sqrt(5.0)) + turn
    r = np.sqrt(1.0 - z * z)
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return d.astype(np.float32)


def _robust_cap(R: int, z_min: float, n_list=(6, 14)) -> np.ndarray:
    """A cap whose rays keep every texel's cosine at least 1e-3 away from 0, so that the
    sign of max(0, cos) cannot depend on rounding (the first turn that does)."""
    for k in range(64):
        d = _cap_dirs(R, z_min, 0.1 * k)
        cos = np.concatenate([octahedral.texel_directions(n) @ d.astype(np.float64).T for n in n_list])
        if np.abs(cos).min() > 1e-3:
            return d
    raise AssertionError("no robust cap found")


def _inputs(fs, frame, dirs):
    (rad, dist, _), (er, ed, _) = H.device_inputs(fs, frame)
    return (rad, dist, torch.from_numpy(dirs).cuda()), (er, ed, dirs.astype(np.float64))


def _interiors(vol):
    tc, tv, lc, lv, f = H.gpu_state(vol)
    return octahedral.interior(tc), octahedral.interior(tv), (tc, tv, lc, lv, f)


def _assert_follows(spec, got_tiles, ref_tiles, tol):
    if spec.state_fmt == "f16":
        assert H.fp16_ulp_diff(got_tiles, ref_tiles).max() <= 1
    else:
        assert H.rel_err(got_tiles, ref_tiles).max() <= tol


@pytest.mark.parametrize("rays", [16, 32])
@pytest.mark.parametrize("operand_fmt,state_fmt", [("f32", "f32"), ("f32", "f16"), ("f16", "f16"), ("bf16", "f16")])
def test_cap_rays_leave_texels_without_rays_unchanged(rays, operand_fmt, state_fmt):
    spec = wl.VolumeSpec(4, 4, 4, rays, state_fmt=state_fmt, operand_fmt=operand_fmt)
    vol = H.lib().ProbeVolume(spec)
    assert vol.kernel == "tcgen05"
    fs = wl.FrameStream(spec, wl.config_seed(1) + rays, mode="noisy")
    # frame 0 from the whole sphere: every texel gets a value to keep
    (rad, dist, dirs), _ = H.device_inputs(fs, 0)
    vol.update(rad, dist, dirs)
    vol.select_and_pack()
    cap = _robust_cap(rays, 0.5)
    d64 = cap.astype(np.float64)
    zero_c = blend.weights(d64, 6)[1] == 0.0
    zero_v = blend.weights(d64, 14, 50.0)[1] == 0.0
    # the premise: a cap of half-angle 60 degrees leaves the texels around -z without rays
    assert 0 < zero_c.sum() < zero_c.size and 0 < zero_v.sum() < zero_v.size
    for f in range(1, 4):
        old_c, old_v, _ = _interiors(vol)
        ov = H.oracle_from_gpu(spec, vol)
        dev, exact = _inputs(fs, f, cap)
        vol.update(*dev)
        ov.update(*exact)
        new_c, new_v, (tc, tv, *_) = _interiors(vol)
        np.testing.assert_array_equal(new_c[..., zero_c], old_c[..., zero_c])
        np.testing.assert_array_equal(new_v[..., zero_v], old_v[..., zero_v])
        _assert_follows(spec, tc, ov.tiles_c, 1e-5)
        _assert_follows(spec, tv, ov.tiles_v, 1e-5)
        np.testing.assert_array_equal(octahedral.fill_border(tv), tv)
        vol.select_and_pack()
    vol.close()


@pytest.mark.parametrize("operand_fmt,tol", [("f32", 1e-5), ("f16", 2e-3), ("bf16", 2e-3)])
def test_visibility_weights_below_the_operand_range(operand_fmt, tol):
    """32 rays in a cone of half-angle 41 degrees: many visibility texels see their best ray
    at cos < 0.5, where cos^50 < 2^-50 (binary16 zero even after a 2^15 scale). h = 0 and
    FP32 state, so each lit texel holds the frame mean."""
    spec = wl.VolumeSpec(4, 4, 4, 32, hysteresis=0.0, state_fmt="f32", operand_fmt=operand_fmt)
    vol = H.lib().ProbeVolume(spec)
    assert vol.kernel == "tcgen05"
    fs = wl.FrameStream(spec, wl.config_seed(3), mode="noisy")
    (rad, dist, dirs), _ = H.device_inputs(fs, 0)
    vol.update(rad, dist, dirs)
    cap = _robust_cap(32, 0.75)
    d64 = cap.astype(np.float64)
    cos_v = octahedral.texel_directions(14) @ d64.T
    best = cos_v.max(axis=1)
    far = (best > 0.0) & (best < 0.5)
    assert far.sum() >= 8
    old_c, old_v, _ = _interiors(vol)
    dev, exact = _inputs(fs, 1, cap)
    vol.update(*dev)
    got_c, got_v, _ = _interiors(vol)
    m_c, m_v = blend.blend_means(*exact, 6, 14, 50.0)
    lit_c = ~np.isnan(m_c[0, 0])
    lit_v = best > 0.0
    assert H.rel_err(got_c[..., lit_c], m_c[..., lit_c]).max() <= tol
    assert H.rel_err(got_v[..., lit_v], m_v[..., lit_v]).max() <= tol
    assert H.rel_err(got_v[..., far], m_v[..., far]).max() <= tol
    np.testing.assert_array_equal(got_c[..., ~lit_c], old_c[..., ~lit_c])
    np.testing.assert_array_equal(got_v[..., ~lit_v], old_v[..., ~lit_v])
    vol.close()


@pytest.mark.parametrize("operand_fmt", ["f32", "f16"])
def test_export_import_resumes_bit_identically(operand_fmt):
    """Checkpoint after three frames, resume in a fresh volume: the next frames' texels,
    last-transmitted codes and packed output equal those of the volume that ran on."""
    spec = wl.VolumeSpec(4, 4, 4, 64, state_fmt="f16", operand_fmt=operand_fmt)
    pv = H.lib()
    a = pv.ProbeVolume(spec)
    assert a.kernel == "tcgen05"
    fs = wl.FrameStream(spec, wl.config_seed(1), mode="noisy", step_frame=4)
    for f in range(3):
        dev, _ = H.device_inputs(fs, f)
        a.update(*dev)
        a.select_and_pack()
    tc, tv, lc, lv, frame = a.export_state()
    assert frame == 3
    b = pv.ProbeVolume(spec)
    b.import_state(tc, tv, lc, lv, frame)
    for f in range(3, 7):
        dev, _ = H.device_inputs(fs, f)
        a.update(*dev)
        b.update(*dev)
        fa = H.gpu_frame(a, a.select_and_pack())
        fb = H.gpu_frame(b, b.select_and_pack())
        for key in fa:
            np.testing.assert_array_equal(np.asarray(fa[key]), np.asarray(fb[key]))
        sa, sb = a.export_state(), b.export_state()
        for x, y in zip(sa[:4], sb[:4]):
            assert torch.equal(x.view(torch.uint8) if x.dtype != torch.uint16 else x.view(torch.int16),
                               y.view(torch.uint8) if y.dtype != torch.uint16 else y.view(torch.int16))
        assert sa[4] == sb[4] == f + 1
    a.close()
    b.close()


def _error_word(vol):
    return H.lib().device_view(vol.info.error_word, (4,), torch.uint8)


def test_error_word_is_reported_once_and_cleared():
    pv = H.lib()
    spec = wl.VolumeSpec(4, 4, 4, 64, state_fmt="f16")
    vol = pv.ProbeVolume(spec)
    assert vol.info.error_word
    fs = wl.FrameStream(spec, wl.config_seed(1))
    dev, _ = H.device_inputs(fs, 0)
    vol.update(*dev)
    fr = vol.select_and_pack(want_host_counts=True)
    assert fr.count_c >= 0
    word = _error_word(vol)
    assert not word.cpu().any()
    # what the blend kernel does when a bounded wait gives up, done from the host
    word.copy_(torch.tensor([1, 0, 0, 0], dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    vol.select_and_pack(want_host_counts=False)       # not read: stays set
    torch.cuda.synchronize()
    assert word.cpu().tolist() == [1, 0, 0, 0]
    with pytest.raises(pv.PVError) as ei:
        vol.select_and_pack(want_host_counts=True)
    assert ei.value.status == -5                      # PV_ERR_TIMEOUT
    torch.cuda.synchronize()
    assert not word.cpu().any()
    # the volume carries on normally
    dev, _ = H.device_inputs(fs, 1)
    vol.update(*dev)
    fr = vol.select_and_pack(want_host_counts=True)
    assert fr.count_c >= 0 and fr.frame == 2
    vol.close()
