"""Shared-volume multi-client selection (Section 3.4: one last-transmitted texture pair per
client): one update of a volume serves several views, each selecting and packing against
what it has already received. Every view's frames must equal the oracle's selection and
packing of the GPU's state against that client's own last-transmitted codes, bit for bit."""
import numpy as np
import pytest
import torch

import pv_workload as wl
from oracle import OracleVolume
from oracle import select_pack as sp
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


class _OracleClient:
    """The oracle's last-transmitted codes of one client."""

    def __init__(self, spec):
        self.spec = spec
        self.last_c = np.full((3, spec.probes, spec.color_interior ** 2), sp.SENTINEL, dtype=np.uint16)
        self.last_v = np.full((2, spec.probes, spec.vis_interior ** 2), sp.SENTINEL, dtype=np.uint16)

        self.cursor_c = self.cursor_v = 0

    def select(self, tiles_c, tiles_v, frame, **knobs):
        ov = OracleVolume(self.spec)
        ov.load_state(tiles_c, tiles_v, self.last_c, self.last_v, frame=frame)
        ov.cursor_c, ov.cursor_v = self.cursor_c, self.cursor_v
        fr = ov.select_and_pack(**knobs)
        self.last_c, self.last_v = ov.last_c.copy(), ov.last_v.copy()
        self.cursor_c, self.cursor_v = ov.cursor_c, ov.cursor_v
        return fr


def test_views_select_against_their_own_history():
    """View A from the start, view B joining at frame 2 (it gets every probe then), the
    volume's own selection as a third client; stationary stream, h = 0, step at frame 3."""
    pv = H.lib()
    spec = wl.VolumeSpec(6, 4, 5, 64, hysteresis=0.0, state_fmt="f16")
    vol = pv.ProbeVolume(spec)
    a = pv.ProbeView(vol)
    oa, ob, ovol = _OracleClient(spec), None, _OracleClient(spec)
    b = None
    fs = wl.FrameStream(spec, 17, mode="stationary", step_frame=3, step_fraction=0.25)
    P = spec.probes
    for f in range(5):
        (r, d, q), _ = H.device_inputs(fs, f)
        vol.update(r, d, q)
        if f == 2:
            b, ob = pv.ProbeView(vol), _OracleClient(spec)
        tc, tv, _, _, fno = H.gpu_state(vol)
        fa = a.select_and_pack(want_host_counts=True)
        H.assert_frames_equal(H.gpu_frame(a, fa), oa.select(tc, tv, fno))
        if b is not None:
            fb = b.select_and_pack(want_host_counts=True)
            gb = H.gpu_frame(b, fb)
            H.assert_frames_equal(gb, ob.select(tc, tv, fno))
            if f == 2:
                assert gb["count_c"] == P and gb["count_v"] == P
        fv = vol.select_and_pack(want_host_counts=True)
        H.assert_frames_equal(H.gpu_frame(vol, fv), ovol.select(tc, tv, fno))
        if f == 2:
            assert fa.count_c == 0 and fa.count_v == 0      # A already holds the stationary texels
        if f == 3:
            assert 0 < fa.count_c < P and fa.count_v == 0
    # a second select without a new update selects nothing
    assert a.select_and_pack(want_host_counts=True).count_c == 0
    for x in (a, b):
        x.close()
    vol.close()


def test_view_equals_volume_selection_on_a_noisy_stream():
    """A view created with its volume sees exactly the volume's own frames."""
    pv = H.lib()
    spec = wl.VolumeSpec(8, 4, 3, 96, state_fmt="f16")
    vol = pv.ProbeVolume(spec)
    view = pv.ProbeView(vol)
    fs = wl.FrameStream(spec, 2, mode="noisy")
    for f in range(3):
        (r, d, q), _ = H.device_inputs(fs, f)
        vol.update(r, d, q)
        gw = H.gpu_frame(view, view.select_and_pack())
        gv = H.gpu_frame(vol, vol.select_and_pack())
        torch.cuda.synchronize()
        for key in gv:
            np.testing.assert_array_equal(np.asarray(gw[key]), np.asarray(gv[key]), err_msg=key)
    view.close()
    vol.close()


@pytest.mark.parametrize("budget,th_c,th_v,masked", [(0, 2, 40, False), (17, 0, 0, False), (13, 1, 8, True),
                                                     (200, 0, 0, True)])
def test_view_knobs_match_oracle(budget, th_c, th_v, masked):
    """Budget (round robin, colour and visibility cursors), change thresholds and an active
    mask on a noisy stream with h = 0.97: every frame equals the oracle's bit for bit."""
    pv = H.lib()
    spec = wl.VolumeSpec(7, 3, 4, 64, state_fmt="f16")
    P = spec.probes
    vol = pv.ProbeVolume(spec)
    view = pv.ProbeView(vol)
    active = None
    if masked:
        act = (np.arange(P) % 4 != 1)
        active = act
        view.set_options(torch.from_numpy(act.astype(np.uint8)).cuda(), budget, th_c, th_v)
    else:
        view.set_options(None, budget, th_c, th_v)
    oc = _OracleClient(spec)
    fs = wl.FrameStream(spec, 23, mode="noisy")
    for f in range(6):
        (r, d, q), _ = H.device_inputs(fs, f)
        vol.update(r, d, q)
        tc, tv, _, _, fno = H.gpu_state(vol)
        fr = view.select_and_pack(want_host_counts=True)
        ofr = oc.select(tc, tv, fno, threshold_c=th_c, threshold_v=th_v, active=active, budget=budget)
        H.assert_frames_equal(H.gpu_frame(view, fr), ofr)
        if budget:
            assert fr.count_c <= budget and fr.count_v <= budget
    view.close()
    vol.close()
