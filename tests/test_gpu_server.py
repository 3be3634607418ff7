"""Served form: sessions admitted by device memory and slots, updated in per-tick batches.

The contract tested here: admission waits and admits in arrival order as memory and slots
free up; a client's results are the same served alone as in a mix of other clients
(joining and leaving around it), bit for bit; and they equal the plain single-volume path.
"""
import numpy as np
import pytest
import torch

import pv_workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

X = wl.VolumeSpec(5, 3, 4, 96, state_fmt="f16")
OTHERS = [wl.VolumeSpec(4, 4, 2, 64, state_fmt="f16"), wl.VolumeSpec(8, 2, 3, 128, state_fmt="f16"),
          wl.VolumeSpec(3, 3, 3, 192, state_fmt="f16"), wl.VolumeSpec(6, 5, 2, 64, state_fmt="f16")]


def _frame_copy(vol, fr):
    g = H.gpu_frame(vol, fr)
    return {k: np.array(v, copy=True) for k, v in g.items()}


def _wait(server, ticket):
    for _ in range(100000):
        fr = server.poll(ticket)
        if fr is not None:
            return fr
    raise AssertionError("ticket never completed")


def _serve(clients_by_tick, inputs, ticks):
    """clients_by_tick[t]: {client: spec} served at tick t; returns frames and states of client 0."""
    pv = H.lib()
    server = pv.ProbeServer(40 << 30, 64)
    open_ = {}
    out = []
    for t in range(ticks):
        want = clients_by_tick[t]
        for c in list(open_):
            if c not in want:
                server.close(c)
                del open_[c]
        for c, spec in want.items():
            if c not in open_:
                assert server.open(c, spec)
                open_[c] = spec
        tickets = {c: server.submit(c, *inputs[c][t]) for c in want}
        server.tick()
        frames = {c: _wait(server, tk) for c, tk in tickets.items()}
        vol0 = server.volume(0)
        out.append((_frame_copy(vol0, frames[0]), H.gpu_state(vol0)))
    server.close_server()
    return out


def _inputs(specs, ticks, seed=21):
    res = {}
    for c, spec in specs.items():
        fs = wl.FrameStream(spec, seed, volume=c)
        res[c] = [H.device_inputs(fs, t)[0] for t in range(ticks)]
    return res


def test_results_equal_alone_and_in_the_mix():
    ticks = 4
    specs = {0: X, **{i + 1: s for i, s in enumerate(OTHERS)}}
    inputs = _inputs(specs, ticks)
    alone = _serve([{0: X}] * ticks, inputs, ticks)
    # the mix changes around client 0: clients join at ticks 0 and 1, two leave at tick 3
    mix = [{0: X, 1: OTHERS[0], 2: OTHERS[1]},
           {0: X, 1: OTHERS[0], 2: OTHERS[1], 3: OTHERS[2], 4: OTHERS[3]},
           {0: X, 1: OTHERS[0], 2: OTHERS[1], 3: OTHERS[2], 4: OTHERS[3]},
           {0: X, 3: OTHERS[2], 4: OTHERS[3]}]
    mixed = _serve(mix, inputs, ticks)
    for (fa, sa), (fm, sm) in zip(alone, mixed):
        for key in fa:
            np.testing.assert_array_equal(fa[key], fm[key], err_msg=key)
        for x, y in zip(sa[:4], sm[:4]):
            np.testing.assert_array_equal(x, y)
    # and both equal the plain single-volume path
    pv = H.lib()
    vol = pv.ProbeVolume(X)
    for t in range(ticks):
        vol.update(*inputs[0][t])
        fr = vol.select_and_pack()
        g = _frame_copy(vol, fr)
        for key in g:
            np.testing.assert_array_equal(g[key], alone[t][0][key], err_msg=key)
    vol.close()


def test_admission_by_memory_and_slots():
    pv = H.lib()
    desc_bytes = pv.probe_volume_bytes(pv.make_desc(X))
    server = pv.ProbeServer(2 * desc_bytes + desc_bytes // 2, 64)
    assert server.open(0, X) and server.open(1, X)
    assert not server.open(2, X)                          # memory: waits
    assert not server.open(3, X)
    a, used, waiting = server.status(2)
    assert a == 0 and waiting == 2 and used == 2 * desc_bytes
    fs = wl.FrameStream(X, 3, volume=2)
    r, d, q = H.device_inputs(fs, 0)[0]
    with pytest.raises(pv.PVError) as e:
        server.submit(2, r, d, q)                         # not admitted yet
    assert e.value.status == -4
    server.close(0)                                       # frees one volume: the first waiter comes in
    assert server.status(2)[0] == 1 and server.status(3)[0] == 0
    t = server.submit(2, r, d, q)
    with pytest.raises(pv.PVError) as e:
        server.submit(2, r, d, q)                         # one submission per tick
    assert e.value.status == -4
    assert server.poll(t) is None                         # its tick has not been launched
    server.tick()
    assert _wait(server, t) is not None
    server.close(1)
    assert server.status(3)[0] == 1
    server.close_server()
    # slot cap
    server = pv.ProbeServer(40 << 30, 1)
    assert server.open(0, X) and not server.open(1, OTHERS[0])
    server.close(0)
    assert server.status(1)[0] == 1
    # a volume larger than the whole budget is refused outright
    small = pv.ProbeServer(1024, 4)
    with pytest.raises(pv.PVError) as e:
        small.open(0, X)
    assert e.value.status == -2
    server.close_server()
    small.close_server()


def test_clients_update_at_their_own_rates():
    """Variable update rates (Section 5): a client submitting every third tick is updated at a
    third of the rate, and its results equal the same cadence served alone."""
    ticks = 6
    specs = {0: X, 1: OTHERS[0]}
    inputs = _inputs(specs, ticks, seed=31)

    def run(clients):
        pv = H.lib()
        server = pv.ProbeServer(40 << 30, 64)
        for c in clients:
            assert server.open(c, specs[c])
        out = []
        for t in range(ticks):
            due = [c for c in clients if c == 0 or t % 3 == 0]       # client 1 every third tick
            tickets = {c: server.submit(c, *inputs[c][t]) for c in due}
            server.tick()
            frames = {c: _wait(server, tk) for c, tk in tickets.items()}
            if 1 in frames:
                v1 = server.volume(1)
                out.append((t, _frame_copy(v1, frames[1]), H.gpu_state(v1)))
        server.close_server()
        return out

    mixed, alone = run([0, 1]), run([1])
    assert [t for t, _, _ in mixed] == [0, 3] == [t for t, _, _ in alone]
    for (_, fm, sm), (_, fa, sa) in zip(mixed, alone):
        for key in fm:
            np.testing.assert_array_equal(fm[key], fa[key], err_msg=key)
        for x, y in zip(sm[:4], sa[:4]):
            np.testing.assert_array_equal(x, y)
        assert sm[4] == sa[4]
