"""Client side (Sections 3.3-3.4): the GPU decode of packed frames into a client's permanent
probe textures must equal the oracle's unpack -> client_apply chain bit for bit, on the
frames the GPU server produced (full, partial and empty selections), and its visibility
textures must reproduce the server's binary16 visibility state exactly."""
import numpy as np
import pytest
import torch

import pv_workload as wl
from oracle import numerics
from oracle import select_pack as sp
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _oracle_client(spec):
    tc, tv = spec.color_interior + 2, spec.vis_interior + 2
    return np.zeros((3, spec.probes, tc, tc)), np.zeros((2, spec.probes, tv, tv))


def _oracle_apply(spec, oc, ov, g):
    bw = spec.nx * spec.ny
    idx_c, idx_v = sp.undelta(g["delta_c"]), sp.undelta(g["delta_v"])
    np.testing.assert_array_equal(idx_c, g["idx_c"])
    np.testing.assert_array_equal(idx_v, g["idx_v"])
    cc = sp.unpack_color(g["planes_c"], idx_c, spec.color_interior, bw, spec.color_lsb)
    cv = sp.unpack_vis(g["planes_v"], idx_v, spec.vis_interior, bw)
    oc = sp.client_apply(oc, idx_c, numerics.color_value(cc, spec.color_code))
    ov = sp.client_apply(ov, idx_v, cv.astype(np.float64))      # binary16 bits, carried exactly
    return oc, ov


def _check(client, oc, ov):
    tex_c, tex_v = client.textures()
    gc = tex_c.cpu().numpy()
    gv = tex_v.cpu().numpy().view(np.uint16)
    np.testing.assert_array_equal(gc, oc.astype(np.float32))
    np.testing.assert_array_equal(gv, ov.astype(np.uint16))


@pytest.mark.parametrize("code,lsb,state_fmt", [("uf10", False, "f16"), ("unorm10", True, "f16"),
                                                ("uf10", False, "f32")])
def test_client_matches_oracle_over_frames(code, lsb, state_fmt):
    """h = 0 on a stationary stream with a step change at frame 2: frame 0 selects every
    probe, frame 1 none, frame 2 the stepped probes' colour only; frames 3-4 are noisy."""
    pv = H.lib()
    spec = wl.VolumeSpec(6, 4, 5, 64, hysteresis=0.0, state_fmt=state_fmt, color_code=code, color_lsb=lsb)
    vol = pv.ProbeVolume(spec)
    client = pv.ProbeClient(spec)
    oc, ov = _oracle_client(spec)
    still = wl.FrameStream(spec, 13, mode="stationary", step_frame=2, step_fraction=0.3)
    noisy = wl.FrameStream(spec, 13, mode="noisy")
    counts = []
    for f in range(5):
        fs = still if f < 3 else noisy
        (r, d, q), _ = H.device_inputs(fs, f)
        vol.update(r, d, q)
        fr = vol.select_and_pack(want_host_counts=True)
        client.apply(fr)
        g = H.gpu_frame(vol, fr)
        counts.append((g["count_c"], g["count_v"]))
        oc, ov = _oracle_apply(spec, oc, ov, g)
        torch.cuda.synchronize()
        _check(client, oc, ov)
    P = spec.probes
    assert counts[0] == (P, P) and counts[1] == (0, 0)
    assert 0 < counts[2][0] < P and counts[2][1] == 0
    client.close()
    vol.close()


def test_client_visibility_equals_server_state():
    """Binary16 state: the visibility code is the state's bit pattern, so after every probe has
    been sent the client's visibility tiles (guard band included) equal the server's."""
    pv = H.lib()
    spec = wl.VolumeSpec(8, 2, 3, 96, state_fmt="f16")
    vol = pv.ProbeVolume(spec)
    client = pv.ProbeClient(spec)
    fs = wl.FrameStream(spec, 4, mode="noisy")
    for f in range(3):
        (r, d, q), _ = H.device_inputs(fs, f)
        vol.update(r, d, q)
        client.apply(vol.select_and_pack())
        tc, tv, lc, lv, _ = vol.export_state()
        torch.cuda.synchronize()
        gv = client.textures()[1].cpu().numpy().view(np.uint16)
        np.testing.assert_array_equal(gv, tv.numpy().view(np.uint16).reshape(gv.shape))
    client.close()
    vol.close()


def test_client_ignores_ids_and_counts_past_the_volume():
    """A damaged frame (count above P, ids running past P) updates only the valid probes."""
    pv = H.lib()
    spec = wl.VolumeSpec(4, 2, 3, 64, state_fmt="f16")
    P = spec.probes
    vol = pv.ProbeVolume(spec)
    fs = wl.FrameStream(spec, 6, mode="noisy")
    (r, d, q), _ = H.device_inputs(fs, 0)
    vol.update(r, d, q)
    fr = vol.select_and_pack(want_host_counts=True)
    assert fr.count_c == P
    g = H.gpu_frame(vol, fr)
    bad = g["delta_c"].astype(np.int64).copy()
    bad[P // 2] += 3 * P                      # ids from slot P/2 on fall outside the volume
    dc = torch.from_numpy(bad.astype(np.uint16).view(np.int16)).cuda()
    cnt = torch.tensor([P + 100, P], dtype=torch.int32).cuda()
    f2 = pv.pv_frame()
    f2.color_planes, f2.vis_planes = fr.color_planes, fr.vis_planes
    f2.delta_c, f2.delta_v = dc.data_ptr(), fr.delta_v
    f2.count_c_dev, f2.count_v_dev = cnt.data_ptr(), cnt.data_ptr() + 4
    client = pv.ProbeClient(spec)
    client.apply(f2)
    oc, ov = _oracle_client(spec)
    good = dict(g)
    good["delta_c"], good["idx_c"] = g["delta_c"][:P // 2], g["idx_c"][:P // 2]
    oc, ov = _oracle_apply(spec, oc, ov, good)
    torch.cuda.synchronize()
    _check(client, oc, ov)
    client.close()
    vol.close()


@pytest.mark.parametrize("nc,nv", [(5, 9), (7, 13), (3, 4), (16, 16)])
def test_client_odd_interiors_and_ragged_blocks(nc, nv):
    """Interiors whose colour rows start at odd samples of the planes' 32-bit words and whose
    visibility rows start anywhere in a 12-byte chunk, and the largest interiors (16x16, whose
    decode needs more than the default 48 KB of shared memory), on a volume whose block rows
    (15 slots) split the decode's groups of slots and whose probe count (45) leaves the last
    group short: full, then partial selections, each equal to the oracle's decode."""
    pv = H.lib()
    spec = wl.VolumeSpec(5, 3, 3, 64, hysteresis=0.0, state_fmt="f16", color_interior=nc, vis_interior=nv)
    vol = pv.ProbeVolume(spec)
    client = pv.ProbeClient(spec)
    oc, ov = _oracle_client(spec)
    fs = wl.FrameStream(spec, 21, mode="stationary", step_frame=1, step_fraction=0.4)
    counts = []
    for f in range(3):
        (r, d, q), _ = H.device_inputs(fs, f)
        vol.update(r, d, q)
        fr = vol.select_and_pack(want_host_counts=True)
        client.apply(fr)
        g = H.gpu_frame(vol, fr)
        counts.append(g["count_c"])
        oc, ov = _oracle_apply(spec, oc, ov, g)
        torch.cuda.synchronize()
        _check(client, oc, ov)
    assert counts[0] == spec.probes and 0 < counts[1] < spec.probes
    client.close()
    vol.close()
