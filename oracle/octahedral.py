"""Octahedral texel directions and the 1-texel guard band of a probe tile.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package.

Each probe stores its irradiance and visibility as an octahedral map of
n x n interior texels surrounded by a one-texel guard band used for
filtering (Section 3.2, "Streaming Probe Irradiance": 10x10 texel arrays,
octahedral mapping; Section 3.4, "Light Probe Repacking": the guard band
holds redundant copies of the core texels). The paper names the octahedral
map but gives no formula; this file uses the standard one.

Texel centre of interior texel (i, j) (row i, column j, 0-based):
  u = 2(j + 1/2)/n - 1,  v = 2(i + 1/2)/n - 1,
  p = (u, v, 1 - |u| - |v|); if p_z < 0:
      (p_x, p_y) <- ((1 - |v|) sgn(u), (1 - |u|) sgn(v)), sgn(0) = +1;
  direction = p / |p|.

Guard band, tile coordinates 0..n+1 with the interior at 1..n (reading of
the paper's "redundant information from the core texel array": the map is
continued across each edge by reflection, u > 1 -> (2 - u, -v), likewise for
v, so each border texel copies the interior texel met after the reflection):
  top    (0, c)     <- (1, n+1-c)        bottom (n+1, c) <- (n, n+1-c)
  left   (r, 0)     <- (n+1-r, 1)        right  (r, n+1) <- (n+1-r, n)
  corners (0,0)<-(n,n), (0,n+1)<-(n,1), (n+1,0)<-(1,n), (n+1,n+1)<-(1,1).
"""
from __future__ import annotations

import numpy as np


def _sgn(x):
    return np.where(x >= 0.0, 1.0, -1.0)


def texel_directions(n: int) -> np.ndarray:
    """[n*n, 3] float64 unit directions of the interior texel centres, row-major (i, j).

    The formula of the module docstring is evaluated with its numerators: u = a/n and
    v = b/n with integers a = 2j+1-n, b = 2i+1-n, so p*n has integer components and
    texels on the fold (|u| + |v| = 1) get p_z = 0 exactly; normalising removes the n.
    """
    j, i = np.meshgrid(np.arange(n, dtype=np.int64), np.arange(n, dtype=np.int64))
    a = (2 * j + 1 - n).ravel()
    b = (2 * i + 1 - n).ravel()
    z = n - np.abs(a) - np.abs(b)
    sa = np.where(a >= 0, 1, -1)
    sb = np.where(b >= 0, 1, -1)
    x = np.where(z < 0, (n - np.abs(b)) * sa, a)
    y = np.where(z < 0, (n - np.abs(a)) * sb, b)
    p = np.stack([x, y, z], axis=1).astype(np.float64)
    return p / np.linalg.norm(p, axis=1, keepdims=True)


def octa_encode(d: np.ndarray):
    """Inverse map: unit directions [..., 3] -> (u, v) in [-1, 1]^2."""
    d = np.asarray(d, dtype=np.float64)
    p = d / np.sum(np.abs(d), axis=-1, keepdims=True)
    px, py, pz = p[..., 0], p[..., 1], p[..., 2]
    u = np.where(pz < 0.0, (1.0 - np.abs(py)) * _sgn(px), px)
    v = np.where(pz < 0.0, (1.0 - np.abs(px)) * _sgn(py), py)
    return u, v


def border_source(n: int) -> np.ndarray:
    """[n+2, n+2, 2] int: tile position each texel is copied from (identity inside)."""
    src = np.zeros((n + 2, n + 2, 2), dtype=np.int64)
    for r in range(n + 2):
        for c in range(n + 2):
            src[r, c] = (r, c)
    for c in range(1, n + 1):
        src[0, c] = (1, n + 1 - c)
        src[n + 1, c] = (n, n + 1 - c)
    for r in range(1, n + 1):
        src[r, 0] = (n + 1 - r, 1)
        src[r, n + 1] = (n + 1 - r, n)
    src[0, 0] = (n, n)
    src[0, n + 1] = (n, 1)
    src[n + 1, 0] = (1, n)
    src[n + 1, n + 1] = (1, 1)
    return src


def fill_border(tiles: np.ndarray) -> np.ndarray:
    """Copy interior texels into the guard band of tiles [..., n+2, n+2] (returns a new array)."""
    n = tiles.shape[-1] - 2
    src = border_source(n)
    return tiles[..., src[..., 0], src[..., 1]]


def interior(tiles: np.ndarray) -> np.ndarray:
    """[..., n+2, n+2] -> [..., n*n] interior texels, row-major."""
    n = tiles.shape[-1] - 2
    return tiles[..., 1:n + 1, 1:n + 1].reshape(tiles.shape[:-2] + (n * n,))


def with_interior(tiles: np.ndarray, values: np.ndarray) -> np.ndarray:
    """Return a copy of ``tiles`` whose interior is ``values`` [..., n*n] (border untouched)."""
    n = tiles.shape[-1] - 2
    out = np.array(tiles, copy=True)
    out[..., 1:n + 1, 1:n + 1] = values.reshape(values.shape[:-1] + (n, n))
    return out
