"""Pins of the oracle's blend against closed forms, brute force and hand-computed cases."""
import math

import numpy as np
import pytest

import pv_workload as wl
from oracle import blend, numerics, octahedral


def _zero_state(P, n_c=6, n_v=14):
    return np.zeros((3, P, n_c + 2, n_c + 2)), np.zeros((2, P, n_v + 2, n_v + 2))


def test_uniform_radiance_converges_as_one_minus_h_to_the_k():
    """Uniform inputs: after k frames every texel equals L (1 - h^k) (FP64 state)."""
    P, R, h = 3, 64, 0.97
    dirs = wl.ray_directions(7, 0, 0, R)
    L = np.array([0.25, 1.5, 7.0])
    sc, sv = _zero_state(P)
    for k in range(1, 13):
        rad = np.broadcast_to(L[:, None, None], (3, P, R))
        dist = np.full((P, R), 3.0)
        dirs = wl.ray_directions(7, 0, k, R)     # fresh rotation: the result must not care
        sc, sv = blend.update(sc, sv, rad, dist, dirs, hysteresis=h, sharpness=50.0, state_fmt="f64")
        f = 1.0 - h ** k
        np.testing.assert_allclose(sc, np.broadcast_to(L[:, None, None, None] * f, sc.shape), rtol=1e-13)
        np.testing.assert_allclose(sv[0], 3.0 * f, rtol=1e-13)
        np.testing.assert_allclose(sv[1], 9.0 * f, rtol=1e-13)


def test_first_frame_without_hysteresis_takes_the_mean():
    P, R = 2, 32
    dirs = wl.ray_directions(1, 0, 0, R)
    rad = np.full((3, P, R), 2.0)
    sc, sv = _zero_state(P)
    sc, sv = blend.update(sc, sv, rad, np.full((P, R), 5.0), dirs, hysteresis=0.97, sharpness=50.0,
                          state_fmt="f64", first_frame=True, first_frame_no_hysteresis=True)
    np.testing.assert_allclose(sc, 2.0, rtol=1e-14)
    np.testing.assert_allclose(sv[1], 25.0, rtol=1e-14)


def test_single_ray_along_z_with_zero_hysteresis():
    """One ray: texels facing it take its value exactly; the others keep their old value."""
    P, n_c, n_v = 1, 6, 14
    dirs = np.array([[0.0, 0.0, 1.0]])
    rad = np.array([3.0, 4.0, 5.0]).reshape(3, 1, 1)
    dist = np.array([[2.5]])
    sc = np.full((3, P, n_c + 2, n_c + 2), -1.0)
    sv = np.full((2, P, n_v + 2, n_v + 2), -1.0)
    sc, sv = blend.update(sc, sv, rad, dist, dirs, hysteresis=0.0, sharpness=50.0, state_fmt="f64")
    for n, tiles, want in [(n_c, sc, [3.0, 4.0, 5.0]), (n_v, sv, [2.5, 6.25])]:
        # exact hemisphere test on the integer numerators: z > 0 iff |2j+1-n| + |2i+1-n| < n
        i, j = np.divmod(np.arange(n * n), n)
        nz = n - np.abs(2 * j + 1 - n) - np.abs(2 * i + 1 - n)
        inner = octahedral.interior(tiles)
        for ch, w in enumerate(want):
            np.testing.assert_allclose(inner[ch, 0, nz > 0], w, rtol=1e-15)
            np.testing.assert_array_equal(inner[ch, 0, nz <= 0], -1.0)


def test_two_rays_mean_of_squares_is_not_square_of_mean():
    """Equal weights: mean distance 2 and mean squared distance 5 for distances 1 and 3."""
    n_v = 2
    nt = octahedral.texel_directions(n_v)[0]
    # two directions symmetric about the first texel direction at equal angle
    a = np.cross(nt, [0.0, 0.0, 1.0])
    a /= np.linalg.norm(a)
    d1 = math.cos(0.2) * nt + math.sin(0.2) * a
    d2 = math.cos(0.2) * nt - math.sin(0.2) * a
    w, s = blend.weights(np.stack([d1, d2]), n_v, 50.0)
    assert w[0, 0] == pytest.approx(w[0, 1], rel=1e-14)
    m = blend.weighted_mean(np.array([[1.0, 3.0]]), w, s)
    m2 = blend.weighted_mean(np.array([[1.0, 9.0]]), w, s)
    assert m[0, 0] == pytest.approx(2.0, rel=1e-14)
    assert m2[0, 0] == pytest.approx(5.0, rel=1e-14)


def test_blend_against_pure_python_brute_force():
    rng = np.random.default_rng(11)
    P, R, n_c, n_v, h, s = 2, 5, 2, 2, 0.9, 7.0
    dirs = rng.standard_normal((R, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rad = rng.lognormal(size=(3, P, R))
    dist = rng.uniform(0.1, 10, size=(P, R))
    sc = rng.random((3, P, n_c + 2, n_c + 2))
    sv = rng.random((2, P, n_v + 2, n_v + 2))
    nc_new, nv_new = blend.update(sc, sv, rad, dist, dirs, hysteresis=h, sharpness=s, state_fmt="f64")

    def texdir(i, j, n):
        u = 2 * (j + 0.5) / n - 1
        v = 2 * (i + 0.5) / n - 1
        z = 1 - abs(u) - abs(v)
        if z < 0:
            u, v = (1 - abs(v)) * (1 if u >= 0 else -1), (1 - abs(u)) * (1 if v >= 0 else -1)
        l = math.sqrt(u * u + v * v + z * z)
        return (u / l, v / l, z / l)

    for n, old, new, chans, power in [(n_c, sc, nc_new, [rad[0], rad[1], rad[2]], 1.0),
                                      (n_v, sv, nv_new, [dist, dist * dist], s)]:
        for ch, x in enumerate(chans):
            for p in range(P):
                for i in range(n):
                    for j in range(n):
                        t = texdir(i, j, n)
                        ws = [max(0.0, sum(t[k] * dirs[r][k] for k in range(3))) ** power for r in range(R)]
                        S = math.fsum(ws)
                        if S == 0:
                            want = old[ch, p, i + 1, j + 1]
                        else:
                            mean = math.fsum(ws[r] * x[p][r] for r in range(R)) / S
                            want = h * old[ch, p, i + 1, j + 1] + (1 - h) * mean
                        assert new[ch, p, i + 1, j + 1] == pytest.approx(want, rel=1e-12, abs=1e-300)


def test_weight_integrals_match_the_lobe_closed_forms():
    """Dense uniform rays: sum_r max(0,cos) ~ R/4 and sum_r max(0,cos)^s ~ R/(2(s+1))."""
    R = 200000
    d = wl.fibonacci_sphere(R)
    _, sc = blend.weights(d, 6)
    _, sv = blend.weights(d, 14, 50.0)
    np.testing.assert_allclose(sc / R, 0.25, rtol=2e-4)
    np.testing.assert_allclose(sv / R, 1.0 / (2 * 51), rtol=5e-3)


def test_fp16_state_follows_a_float16_recurrence_and_stalls_short_of_the_target():
    """FP16 state, uniform L = 1: s <- fl16(h s + (1-h) L) as numpy float16 casts; the
    recurrence stalls about 2^-11/(1-h) below 1 instead of reaching L (1 - h^k)."""
    h = float(np.float32(0.97))
    P, R = 1, 16
    dirs = wl.ray_directions(3, 0, 0, R)
    sc, sv = _zero_state(P)
    s_ref = 0.0
    for k in range(1, 400):
        sc, sv = blend.update(sc, sv, np.ones((3, P, R)), np.ones((P, R)), dirs,
                              hysteresis=h, sharpness=50.0, state_fmt="f16")
        s_ref = float(np.float16(h * s_ref + (1.0 - h) * 1.0))
        np.testing.assert_array_equal(sc, s_ref)
    assert s_ref < 1.0 - 2.0 ** -11 and 1.0 - s_ref <= 2.0 ** -11 / (1 - h) + 2 ** -10
    # FP32 state: close to the closed form 1 - h^k
    sc, sv = _zero_state(P)
    for k in range(1, 60):
        sc, sv = blend.update(sc, sv, np.ones((3, P, R)), np.ones((P, R)), dirs,
                              hysteresis=h, sharpness=50.0, state_fmt="f32")
    np.testing.assert_allclose(sc, 1.0 - h ** 59, rtol=2e-6)


def test_zero_weight_texels_keep_their_value():
    P, R = 1, 1
    dirs = np.array([[0.0, 0.0, -1.0]])      # only the lower hemisphere sees this ray
    sc, sv = _zero_state(P)
    sc[:] = 0.5
    sc = octahedral.fill_border(sc)
    new_c, _ = blend.update(sc, sv, np.full((3, P, R), 8.0), np.full((P, R), 1.0), dirs,
                            hysteresis=0.5, sharpness=50.0, state_fmt="f32")
    nz = octahedral.texel_directions(6)[:, 2]
    inner = octahedral.interior(new_c)
    np.testing.assert_array_equal(inner[:, 0, nz >= 0], 0.5)
    np.testing.assert_array_equal(inner[:, 0, nz < 0], 4.25)


def test_border_is_refilled_after_update():
    spec = wl.config1()
    fs = wl.FrameStream(spec, 5)
    sc, sv = _zero_state(spec.probes)
    sc, sv = blend.update(sc, sv, fs.radiance(0), fs.dist(0), fs.directions(0),
                          hysteresis=0.97, sharpness=50.0, state_fmt="f32")
    np.testing.assert_array_equal(octahedral.fill_border(sc), sc)
    np.testing.assert_array_equal(octahedral.fill_border(sv), sv)
    assert np.all(numerics.round_fp32(sc) == sc)
