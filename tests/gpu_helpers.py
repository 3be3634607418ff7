"""Shared helpers of the GPU parity tests: run the library and the oracle side by side."""
import numpy as np
import torch

import pv_workload as wl
from oracle import OracleVolume, numerics, octahedral, select_pack

TORCH_OP = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}


def lib():
    import paper_2103_05875_gb300 as pv
    return pv


def device_inputs(fs: wl.FrameStream, frame: int):
    """(radiance, dist, dirs) as CUDA tensors in the operand format, plus the float64 values
    the oracle must see (the operand-rounded ones)."""
    fmt = fs.spec.operand_fmt
    rad = wl.to_operand(fs.radiance(frame), fmt)
    dist = wl.to_operand(fs.dist(frame), fmt)
    dirs = torch.from_numpy(fs.directions(frame))
    exact = (rad.double().numpy(), dist.double().numpy(), dirs.double().numpy())
    return (rad.cuda(), dist.cuda(), dirs.cuda()), exact


def gpu_state(vol):
    tc, tv, lc, lv, f = vol.export_state()
    return (tc.double().numpy(), tv.double().numpy(), lc.numpy().view(np.uint16).copy(),
            lv.numpy().view(np.uint16).copy(), f)


def oracle_from_gpu(spec, vol) -> OracleVolume:
    ov = OracleVolume(spec)
    tc, tv, lc, lv, f = gpu_state(vol)
    ov.load_state(tc, tv, lc, lv, frame=f)
    return ov


def gpu_frame(vol, fr):
    """Host copies of a packed frame: counts, ids, deltas, planes (with pad columns)."""
    counts = vol.counts(fr).cpu().numpy().astype(np.int64)
    nc, nv = int(counts[0]), int(counts[1])
    return dict(
        count_c=nc, count_v=nv,
        idx_c=vol.index(fr, "c", nc).cpu().numpy().view(np.uint16),
        idx_v=vol.index(fr, "v", nv).cpu().numpy().view(np.uint16),
        delta_c=vol.index(fr, "dc", nc).cpu().numpy().view(np.uint16),
        delta_v=vol.index(fr, "dv", nv).cpu().numpy().view(np.uint16),
        planes_c=vol.color_planes(fr).cpu().numpy().view(np.uint16),
        planes_v_full=vol.vis_planes(fr, with_pad=True).cpu().numpy(),
        planes_v=vol.vis_planes(fr).cpu().numpy(),
    )


def assert_frames_equal(g, o):
    assert g["count_c"] == o.count_c and g["count_v"] == o.count_v
    np.testing.assert_array_equal(g["idx_c"], o.idx_c)
    np.testing.assert_array_equal(g["idx_v"], o.idx_v)
    np.testing.assert_array_equal(g["delta_c"], o.delta_c)
    np.testing.assert_array_equal(g["delta_v"], o.delta_v)
    np.testing.assert_array_equal(g["planes_c"], o.planes_c)
    np.testing.assert_array_equal(g["planes_v"], o.planes_v)
    # pad columns of the visibility planes stay zero
    assert not g["planes_v_full"][:, :, o.planes_v.shape[2]:].any()


def rel_err(got, ref):
    """|got-ref| / max(|ref|, 1e-6 max|ref|), elementwise."""
    ref = np.asarray(ref, dtype=np.float64)
    den = np.maximum(np.abs(ref), 1e-6 * np.max(np.abs(ref)))
    return np.abs(np.asarray(got, dtype=np.float64) - ref) / den


def fp16_ulp_diff(a, b):
    """Distance in binary16 ulps between two arrays of finite binary16 values."""
    def ordered(x):
        bits = numerics.fp16_bits(x).astype(np.int64)
        return np.where(bits & 0x8000, -(bits & 0x7FFF), bits)
    return np.abs(ordered(a) - ordered(b))
