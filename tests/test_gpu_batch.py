"""Batched form: several volumes of uneven sizes updated in one persistent blend launch (plus
one weights launch and one select/pack launch).

Each texel of a volume depends only on that volume's inputs and state, and the batched
kernels run the same per-item code as the single-volume ones over the same K chunks, so the
batch must reproduce volume-by-volume updates bit for bit: tiles, changed probes, packed
frames and last-transmitted codes. One step is also checked against the oracle.
"""
import numpy as np
import pytest
import torch

import pv_workload as wl
from oracle import OracleVolume, octahedral
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

SMALL = [wl.VolumeSpec(4, 3, 5, 64, state_fmt="f16"), wl.VolumeSpec(6, 2, 3, 96, state_fmt="f16"),
         wl.VolumeSpec(2, 2, 2, 128, state_fmt="f16"), wl.VolumeSpec(7, 5, 3, 64, state_fmt="f16")]


def _streams(specs, seed):
    return [wl.FrameStream(s, seed, volume=i) for i, s in enumerate(specs)]


def _inputs(streams, f):
    dev, exact = [], []
    for fs in streams:
        d, e = H.device_inputs(fs, f)
        dev.append(d)
        exact.append(e)
    return dev, exact


def _run_pair(specs, frames, probes_per_item=0, seed=11):
    pv = H.lib()
    alone = [pv.ProbeVolume(s) for s in specs]
    batched = [pv.ProbeVolume(s) for s in specs]
    assert all(v.kernel == "tcgen05" for v in batched)
    batch = pv.ProbeBatch(batched, probes_per_item)
    streams = _streams(specs, seed)
    for f in range(frames):
        dev, _ = _inputs(streams, f)
        for v, (r, d, q) in zip(alone, dev):
            v.update(r, d, q)
        batch.update([x[0] for x in dev], [x[1] for x in dev], [x[2] for x in dev])
        fr_a = [v.select_and_pack() for v in alone]
        fr_b = batch.select_and_pack()
        torch.cuda.synchronize()
        for va, vb, fa, fb in zip(alone, batched, fr_a, fr_b):
            sa, sb = H.gpu_state(va), H.gpu_state(vb)
            for x, y in zip(sa[:4], sb[:4]):
                np.testing.assert_array_equal(x, y)
            assert sa[4] == sb[4]
            ga, gb = H.gpu_frame(va, fa), H.gpu_frame(vb, fb)
            for key in ga:
                np.testing.assert_array_equal(np.asarray(ga[key]), np.asarray(gb[key]), err_msg=key)
    return alone, batched, batch


@pytest.mark.parametrize("probes_per_item", [0, 8, 13])
def test_batch_equals_volume_by_volume(probes_per_item):
    _, _, batch = _run_pair(SMALL, 3, probes_per_item)
    if probes_per_item:
        assert batch.probes_per_item == probes_per_item
    batch.close()


@pytest.mark.parametrize("operand_fmt", ["f16", "bf16"])
def test_batch_precision_forms_equal_volume_by_volume(operand_fmt):
    specs = [wl.VolumeSpec(s.nx, s.ny, s.nz, s.rays, state_fmt="f16", operand_fmt=operand_fmt) for s in SMALL]
    _, _, batch = _run_pair(specs, 2)
    batch.close()


def test_batch_step_matches_oracle():
    pv = H.lib()
    vols = [pv.ProbeVolume(s) for s in SMALL]
    batch = pv.ProbeBatch(vols)
    streams = _streams(SMALL, 5)
    for f in range(2):
        oracles = [H.oracle_from_gpu(s, v) for s, v in zip(SMALL, vols)]
        dev, exact = _inputs(streams, f)
        batch.update([x[0] for x in dev], [x[1] for x in dev], [x[2] for x in dev])
        torch.cuda.synchronize()
        loaded = []
        for s, v, ov, e in zip(SMALL, vols, oracles, exact):
            ov.update(*e)
            tc, tv, lc, lv, fno = H.gpu_state(v)
            assert H.fp16_ulp_diff(tc, ov.tiles_c).max() <= 1
            assert H.fp16_ulp_diff(tv, ov.tiles_v).max() <= 1
            np.testing.assert_array_equal(octahedral.fill_border(tc), tc)
            np.testing.assert_array_equal(octahedral.fill_border(tv), tv)
            og = OracleVolume(s)
            og.load_state(tc, tv, lc, lv, frame=fno)
            loaded.append(og)
        frames = batch.select_and_pack()
        for v, og, fr in zip(vols, loaded, frames):
            H.assert_frames_equal(H.gpu_frame(v, fr), og.select_and_pack())
    batch.close()


def test_config4_twelve_volumes_one_step_equals_volume_by_volume():
    """The batched workload itself: 12 volumes 8x4x8 .. 32x8x32 (37,376 probes), rays 128/192/256."""
    specs = wl.config4()
    _, _, batch = _run_pair(specs, 1)
    batch.close()


def test_batch_tune_keeps_state():
    pv = H.lib()
    vols = [pv.ProbeVolume(s) for s in SMALL]
    alone = [pv.ProbeVolume(s) for s in SMALL]
    batch = pv.ProbeBatch(vols)
    streams = _streams(SMALL, 3)
    dev, _ = _inputs(streams, 0)
    args = ([x[0] for x in dev], [x[1] for x in dev], [x[2] for x in dev])
    batch.update(*args)
    for v, (r, d, q) in zip(alone, dev):
        v.update(r, d, q)
    torch.cuda.synchronize()
    before = [H.gpu_state(v) for v in vols]
    np_ = batch.tune(*args, reps=2)
    assert np_ in (8, 10, 12, 14, 16, 20, 24, 28, 32)
    assert batch.probes_per_item == np_
    after = [H.gpu_state(v) for v in vols]
    for b, a in zip(before, after):
        for x, y in zip(b[:4], a[:4]):
            np.testing.assert_array_equal(x, y)
        assert b[4] == a[4]
    # the frame selected after tuning is the one of the update before it
    frames = batch.select_and_pack()
    for va, vb, fb in zip(alone, vols, frames):
        ga, gb = H.gpu_frame(va, va.select_and_pack()), H.gpu_frame(vb, fb)
        for key in ga:
            np.testing.assert_array_equal(np.asarray(ga[key]), np.asarray(gb[key]), err_msg=key)
    batch.close()


@pytest.mark.parametrize("operand_fmt", ["f32", "f16"])
def test_autotune_caches_its_plan_and_keeps_results(operand_fmt, tmp_path):
    """The tuner leaves the volumes' state as it found it, writes its plan to the cache file,
    answers the same shape from the cache without timing, and the tuned plan updates the
    volumes bit for bit as volume-by-volume calls do."""
    pv = H.lib()
    specs = [wl.VolumeSpec(s.nx, s.ny, s.nz, s.rays, state_fmt="f16", operand_fmt=operand_fmt) for s in SMALL]
    vols = [pv.ProbeVolume(s) for s in specs]
    alone = [pv.ProbeVolume(s) for s in specs]
    batch = pv.ProbeBatch(vols)
    streams = _streams(specs, 5)
    dev, _ = _inputs(streams, 0)
    args = ([x[0] for x in dev], [x[1] for x in dev], [x[2] for x in dev])
    batch.update(*args)
    for v, (r, d, q) in zip(alone, dev):
        v.update(r, d, q)
    torch.cuda.synchronize()
    before = [H.gpu_state(v) for v in vols]
    cache = tmp_path / "tune.txt"
    r1 = batch.autotune(*args, reps=2, cache_path=str(cache))
    assert r1["from_cache"] == 0 and r1["candidates"] >= 5
    assert 0.0 < r1["best_us"] <= r1["default_us"]
    assert batch.probes_per_item == r1["probes_per_item"]
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and "\t" in lines[0]
    after = [H.gpu_state(v) for v in vols]
    for b, a in zip(before, after):
        for x, y in zip(b[:4], a[:4]):
            np.testing.assert_array_equal(x, y)
        assert b[4] == a[4]
    # a second batch of the same shapes takes the plan from the cache
    vols2 = [pv.ProbeVolume(s) for s in specs]
    batch2 = pv.ProbeBatch(vols2)
    r2 = batch2.autotune(*args, reps=2, cache_path=str(cache))
    assert r2["from_cache"] == 1 and r2["candidates"] == 0
    for k in ("probes_per_item", "ray_stages", "weight_stages", "tmem_stages", "ctas"):
        assert r2[k] == r1[k], k
    assert len(cache.read_text().splitlines()) == 1
    # the tuned plan: next frames equal volume by volume
    for f in (1, 2):
        dev, _ = _inputs(streams, f)
        batch.update([x[0] for x in dev], [x[1] for x in dev], [x[2] for x in dev])
        for v, (r, d, q) in zip(alone, dev):
            v.update(r, d, q)
        frames = batch.select_and_pack()
        for va, vb, fb in zip(alone, vols, frames):
            ga, gb = H.gpu_frame(va, va.select_and_pack()), H.gpu_frame(vb, fb)
            for key in ga:
                np.testing.assert_array_equal(np.asarray(ga[key]), np.asarray(gb[key]), err_msg=key)
            sa, sb = H.gpu_state(va), H.gpu_state(vb)
            for x, y in zip(sa[:4], sb[:4]):
                np.testing.assert_array_equal(x, y)
    batch2.close()
    batch.close()


def test_batch_rejects_mixed_shapes_and_too_many():
    pv = H.lib()
    a = pv.ProbeVolume(wl.VolumeSpec(2, 2, 2, 64, state_fmt="f16"))
    b = pv.ProbeVolume(wl.VolumeSpec(2, 2, 2, 64, state_fmt="f16", vis_interior=8))
    with pytest.raises(pv.PVError) as e:
        pv.ProbeBatch([a, b])
    assert e.value.status == -1
    with pytest.raises(pv.PVError) as e:
        pv.ProbeBatch([a, a])
    assert e.value.status == -1
    many = [pv.ProbeVolume(wl.VolumeSpec(1, 1, 1, 64, state_fmt="f16")) for _ in range(17)]
    with pytest.raises(pv.PVError) as e:
        pv.ProbeBatch(many)
    assert e.value.status == -6
