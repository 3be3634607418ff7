"""probe_update_static, the allocation-free update for callers that cannot allocate device
memory (code running where cudaMalloc is unavailable or not allowed, e.g. stream callbacks,
graph host nodes, or plugins confined to memory their host application owns).

It must produce what the allocating path (a volume and probe_update) produces: the same
texels, within the tolerance of the parity tests, and the same changed probes, on two calls
in a row. The caller carries the last-transmitted codes between calls, as a streaming server
would after sending a frame. Collected last so that a stop-at-first-failure run has already
run every other test.
"""
import numpy as np
import pytest
import torch

import pv_workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _probe_set(bits: np.ndarray, P: int):
    b = bits.view(np.uint32)
    return {p for p in range(P) if (b[p >> 5] >> (p & 31)) & 1}


# (grid, rays, interiors, state format, operand format). The 16x16 / 16x16 case uses
# 510 rays, the most the scratch array holds for 512 texels, so the whole array is used.
CASES = [
    ((5, 3, 4), 64, (6, 14), "f32", "f32"),
    ((5, 3, 4), 64, (6, 14), "f16", "f32"),
    ((3, 2, 2), 510, (16, 16), "f16", "f32"),
    ((5, 3, 4), 96, (6, 14), "f16", "f16"),
]


@pytest.mark.parametrize("grid,rays,interiors,state_fmt,operand_fmt", CASES)
def test_static_update_matches_volume_update_twice(grid, rays, interiors, state_fmt, operand_fmt):
    pv = H.lib()
    nc, nv = interiors
    spec = wl.VolumeSpec(*grid, rays, state_fmt=state_fmt, operand_fmt=operand_fmt,
                         color_interior=nc, vis_interior=nv)
    P = spec.probes
    W = (P + 31) // 32
    vol = pv.ProbeVolume(spec, kernel="simt")
    desc = pv.make_desc(spec)
    dt = torch.float32 if state_fmt == "f32" else torch.float16
    tiles_c = torch.zeros((3, P, nc + 2, nc + 2), dtype=dt, device="cuda")
    tiles_v = torch.zeros((2, P, nv + 2, nv + 2), dtype=dt, device="cuda")
    last_c = torch.full((3, P, nc * nc), -1, dtype=torch.int16, device="cuda")     # 0xFFFF: never sent
    last_v = torch.full((2, P, nv * nv), -1, dtype=torch.int16, device="cuda")
    bits = torch.zeros(2 * W, dtype=torch.int32, device="cuda")
    fs = wl.FrameStream(spec, 77)
    for f in range(2):
        (rad, dist, dirs), _ = H.device_inputs(fs, f)
        vol.update(rad, dist, dirs)
        pv.probe_update_static(desc, f, rad, dist, dirs, tiles_c, tiles_v, last_c, last_v, bits)
        torch.cuda.synchronize()
        vc, vv, _, _, _ = H.gpu_state(vol)
        sc = tiles_c.double().cpu().numpy()
        sv = tiles_v.double().cpu().numpy()
        if state_fmt == "f32":
            assert H.rel_err(sc, vc).max() <= 1e-5
            assert H.rel_err(sv, vv).max() <= 1e-5
        else:
            assert H.fp16_ulp_diff(sc, vc).max() <= 1
            assert H.fp16_ulp_diff(sv, vv).max() <= 1
        fr = vol.select_and_pack(want_host_counts=True)
        g = H.gpu_frame(vol, fr)
        b = bits.cpu().numpy()
        assert _probe_set(b[:W], P) == set(g["idx_c"].astype(int).tolist())
        assert _probe_set(b[W:], P) == set(g["idx_v"].astype(int).tolist())
        # the caller sends the selected probes: its last-transmitted codes follow the volume's
        _, _, lc, lv, _ = H.gpu_state(vol)
        last_c.copy_(torch.from_numpy(lc.view(np.int16)))
        last_v.copy_(torch.from_numpy(lv.view(np.int16)))
    vol.close()


@pytest.mark.parametrize("rays", [511, 1024])
def test_static_update_rejects_sizes_beyond_its_scratch(rays):
    pv = H.lib()
    spec = wl.VolumeSpec(2, 2, 2, rays, color_interior=16, vis_interior=16)
    desc = pv.make_desc(spec)
    z = torch.zeros(1, device="cuda")
    with pytest.raises(pv.PVError) as e:
        pv.probe_update_static(desc, 0, z, z, z, z, z, z, z, z)
    assert e.value.status == -6
    assert "510" in str(e.value)
