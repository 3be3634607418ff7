"""The synthetic inputs that stand in for the paper's scenes: each property the design notes
state for them (distributions, seeding, modes, workload sizes), checked on the generators."""
import math

import numpy as np
import pytest

import pv_workload as wl


def test_radiance_is_lognormal_with_the_stated_parameters():
    L = wl.radiance(wl.config_seed(2), 0, 0, 64, 256)
    assert L.shape == (3, 64, 256) and (L > 0).all()
    z = np.log(L).ravel()
    assert abs(z.mean() - (-1.0)) < 0.02 and abs(z.std() - 1.5) < 0.02


def test_hit_distance_is_uniform_with_a_tenth_misses_at_the_far_plane():
    d = wl.hit_distance(wl.config_seed(2), 0, 0, 128, 256)
    assert d.shape == (128, 256) and d.min() >= 0.1 and d.max() <= 10.0
    miss = np.isclose(d, 10.0)
    assert abs(miss.mean() - 0.1) < 0.01
    hits = d[~miss]
    assert abs(hits.mean() - 5.05) < 0.05 and abs(hits.std() - 9.9 / math.sqrt(12)) < 0.05


def test_streams_are_seeded_and_keyed_by_volume_and_frame():
    s = wl.config_seed(2)
    np.testing.assert_array_equal(wl.radiance(s, 0, 3, 8, 16), wl.radiance(s, 0, 3, 8, 16))
    assert not np.array_equal(wl.radiance(s, 0, 3, 8, 16), wl.radiance(s, 0, 4, 8, 16))
    assert not np.array_equal(wl.radiance(s, 0, 3, 8, 16), wl.radiance(s, 1, 3, 8, 16))
    assert not np.array_equal(wl.radiance(s, 0, 3, 8, 16), wl.radiance(s + 1, 0, 3, 8, 16))


@pytest.mark.parametrize("mode", ["noisy", "stationary"])
def test_frame_stream_modes(mode):
    spec = wl.VolumeSpec(4, 2, 2, 32)
    fs = wl.FrameStream(spec, 7, mode=mode, step_frame=5, step_fraction=0.25)
    same = np.array_equal(fs.radiance(1), fs.radiance(2)) and np.array_equal(fs.dist(1), fs.dist(2)) \
        and np.array_equal(fs.directions(1), fs.directions(2))
    assert same == (mode == "stationary")
    # from the step frame on, the seeded fraction of probes has its radiance scaled by the gain
    m = wl.step_mask(7, 0, spec.probes, 0.25)
    before, after = fs.radiance(4), fs.radiance(5)
    if mode == "stationary":
        np.testing.assert_allclose(after[:, m, :], 4.0 * before[:, m, :], rtol=1e-6)
        np.testing.assert_array_equal(after[:, ~m, :], before[:, ~m, :])


def test_workload_sizes():
    c2 = wl.config2()
    assert (c2.nx, c2.ny, c2.nz, c2.rays, c2.state_fmt) == (16, 16, 16, 256, "f16")
    c4 = wl.config4()
    assert len(c4) == 12 and sum(s.probes for s in c4) == 37376
    assert sorted({s.rays for s in c4}) == [128, 192, 256]


def test_served_arrivals_are_poisson_with_exponential_sessions():
    cl = wl.served_clients()
    assert len(cl) == 64
    t = np.array([c.arrive_s for c in cl])
    assert (np.diff(t) >= 0).all()
    gaps = np.diff(np.r_[0.0, t])
    assert 0.15 < gaps.mean() < 0.4                     # about 1 / (4 per second)
    dur = np.array([c.session_s for c in cl])
    assert 4.0 < dur.mean() < 14.0                       # exponential, mean 8 s (64 draws)
