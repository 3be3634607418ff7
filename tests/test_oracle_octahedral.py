"""Pins of the octahedral texel directions and the guard-band rule."""
import numpy as np
import pytest

from oracle import octahedral as oc


@pytest.mark.parametrize("n", [1, 2, 6, 8, 14, 16])
def test_directions_are_unit_and_encode_back_to_their_texel(n):
    d = oc.texel_directions(n)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=0, atol=1e-15)
    u, v = oc.octa_encode(d)
    j = np.clip(np.floor((u + 1.0) / 2.0 * n), 0, n - 1).astype(int)
    i = np.clip(np.floor((v + 1.0) / 2.0 * n), 0, n - 1).astype(int)
    ii, jj = np.divmod(np.arange(n * n), n)
    np.testing.assert_array_equal(i, ii)
    np.testing.assert_array_equal(j, jj)
    # the centre itself is recovered, not just the cell
    np.testing.assert_allclose(u, 2.0 * (jj + 0.5) / n - 1.0, atol=1e-14)
    np.testing.assert_allclose(v, 2.0 * (ii + 0.5) / n - 1.0, atol=1e-14)


def test_directions_cover_the_sphere_symmetrically():
    d = oc.texel_directions(14)
    np.testing.assert_allclose(d.mean(axis=0), 0.0, atol=1e-12)   # point-symmetric set


def _reflect_into_square(u, v):
    """Continue the map across its edges by reflection: u>1 -> (2-u, -v), v>1 -> (-u, 2-v)."""
    for _ in range(4):
        if u > 1:
            u, v = 2 - u, -v
        elif u < -1:
            u, v = -2 - u, -v
        elif v > 1:
            u, v = -u, 2 - v
        elif v < -1:
            u, v = -u, -2 - v
    return u, v


@pytest.mark.parametrize("n", [2, 6, 8, 14, 16])
def test_guard_band_matches_reflection_of_the_continued_map(n):
    src = oc.border_source(n)
    for r in range(n + 2):
        for c in range(n + 2):
            u = 2.0 * (c - 1 + 0.5) / n - 1.0
            v = 2.0 * (r - 1 + 0.5) / n - 1.0
            u2, v2 = _reflect_into_square(u, v)
            jj = int(np.floor((u2 + 1) / 2 * n))
            ii = int(np.floor((v2 + 1) / 2 * n))
            assert (src[r, c, 0], src[r, c, 1]) == (ii + 1, jj + 1), (r, c)


@pytest.mark.parametrize("n", [6, 14])
def test_edge_guard_texel_copies_a_nearest_interior_texel_across_the_fold(n):
    """Geometric check: the copied texel is one of the two interior texels nearest to the
    edge point between the guard texel and its neighbour, and not that neighbour."""
    dirs = oc.texel_directions(n).reshape(n, n, 3)
    src = oc.border_source(n)

    def dir_at(u, v):
        z = 1 - abs(u) - abs(v)
        if z < 0:
            u, v = (1 - abs(v)) * (1 if u >= 0 else -1), (1 - abs(u)) * (1 if v >= 0 else -1)
        p = np.array([u, v, z])
        return p / np.linalg.norm(p)

    for k in range(1, n + 1):
        t = 2.0 * (k - 1 + 0.5) / n - 1.0
        for (r, c, edge, nb) in [(0, k, (t, -1.0), (1, k)), (n + 1, k, (t, 1.0), (n, k)),
                                 (k, 0, (-1.0, t), (k, 1)), (k, n + 1, (1.0, t), (k, n))]:
            e = dir_at(*edge)
            cosang = dirs.reshape(-1, 3) @ e
            order = np.argsort(-cosang)
            best = set()
            top = cosang[order[0]]
            for o in order:
                if cosang[o] > top - 1e-12:
                    best.add((o // n + 1, o % n + 1))
            s = (int(src[r, c, 0]), int(src[r, c, 1]))
            assert s in best, (r, c, s, best)
            if s != nb:
                assert nb in best


def test_fill_border_against_loop():
    rng = np.random.default_rng(0)
    n = 6
    t = rng.random((3, 5, n + 2, n + 2))
    f = oc.fill_border(t)
    np.testing.assert_array_equal(oc.interior(f), oc.interior(t))
    for r in range(n + 2):
        for c in range(n + 2):
            rr, cc = r, c
            if r == 0 and 1 <= c <= n:
                rr, cc = 1, n + 1 - c
            elif r == n + 1 and 1 <= c <= n:
                rr, cc = n, n + 1 - c
            elif c == 0 and 1 <= r <= n:
                rr, cc = n + 1 - r, 1
            elif c == n + 1 and 1 <= r <= n:
                rr, cc = n + 1 - r, n
            elif (r, c) == (0, 0):
                rr, cc = n, n
            elif (r, c) == (0, n + 1):
                rr, cc = n, 1
            elif (r, c) == (n + 1, 0):
                rr, cc = 1, n
            elif (r, c) == (n + 1, n + 1):
                rr, cc = 1, 1
            np.testing.assert_array_equal(f[..., r, c], t[..., rr, cc])
