"""Per-frame probe blend: the irradiance and visibility update of every texel.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package.

The paper adopts the DDGI irradiance volume (Section 3.2) without restating
its blend: probe irradiance texels hold a cosine-weighted mean of the traced
ray radiance in the texel direction, visibility texels hold the mean distance
and mean squared distance of the rays (Section 3.2, "Streaming Probe
Visibility"), with a sharper (cosine-power) weight, and both are blended into
the previous value with hysteresis. The readings used here, in plain FP64:

  W_c[t, r] = max(0, n_t . d_r)                 (colour texel t, ray r)
  W_v[t, r] = max(0, n_t . d_r) ^ sharpness     (visibility texel t)
  m = sum_r W[t, r] x_r / sum_r W[t, r]         (weight-sum normalisation)
  new = h * old + (1 - h) * m, then one rounding to the state format.

If a texel's weight sum is zero it keeps its old value. With the
``first_frame_no_hysteresis`` option the very first update uses h = 0.
The ray directions d_r are an input of the blend (they come with the traced
rays); 256 rays per probe is the paper's server setting (Section 4).
"""
from __future__ import annotations

import numpy as np

from . import numerics, octahedral


def weights(dirs: np.ndarray, n: int, power: float | None = None):
    """Weights [n*n, R] and their row sums [n*n] for an n x n octahedral tile.

    ``power=None`` gives the cosine lobe max(0, n.d); otherwise max(0, n.d)^power.
    """
    d = np.asarray(dirs, dtype=np.float64)
    nt = octahedral.texel_directions(n)
    cos = nt @ d.T
    w = np.maximum(0.0, cos)
    if power is not None:
        w = w ** float(power)
    return w, w.sum(axis=1)


def weighted_mean(x: np.ndarray, w: np.ndarray, s: np.ndarray) -> np.ndarray:
    """m[..., t] = sum_r w[t, r] x[..., r] / s[t]; entries with s == 0 are NaN."""
    num = np.asarray(x, dtype=np.float64) @ w.T
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(s > 0.0, num / np.where(s > 0.0, s, 1.0), np.nan)


def hysteresis_blend(old: np.ndarray, m: np.ndarray, h: float, fmt: str) -> np.ndarray:
    """h*old + (1-h)*m rounded once to ``fmt``; texels whose mean is undefined keep ``old``."""
    new = numerics.round_state(h * old + (1.0 - h) * np.nan_to_num(m), fmt)
    return np.where(np.isnan(m), old, new)


def blend_means(radiance, dist, dirs, n_c: int, n_v: int, sharpness: float):
    """Per-frame means before hysteresis.

    radiance [3, P, R], dist [P, R] -> (m_c [3, P, n_c^2], m_v [2, P, n_v^2]),
    where m_v[0] is the mean distance and m_v[1] the mean squared distance.
    """
    L = np.asarray(radiance, dtype=np.float64)
    D = np.asarray(dist, dtype=np.float64)
    wc, sc = weights(dirs, n_c)
    wv, sv = weights(dirs, n_v, sharpness)
    m_c = weighted_mean(L, wc, sc)
    m_v = np.stack([weighted_mean(D, wv, sv), weighted_mean(D * D, wv, sv)])
    return m_c, m_v


def update(state_c, state_v, radiance, dist, dirs, *, hysteresis: float, sharpness: float,
           state_fmt: str, first_frame: bool = False, first_frame_no_hysteresis: bool = False):
    """One probe-volume update.

    state_c [3, P, n_c+2, n_c+2] and state_v [2, P, n_v+2, n_v+2] hold float64
    values representable in ``state_fmt``. Returns the new tiles, interior
    blended and guard band refilled.
    """
    n_c = state_c.shape[-1] - 2
    n_v = state_v.shape[-1] - 2
    h = 0.0 if (first_frame and first_frame_no_hysteresis) else float(hysteresis)
    m_c, m_v = blend_means(radiance, dist, dirs, n_c, n_v, sharpness)
    new_c = hysteresis_blend(octahedral.interior(state_c), m_c, h, state_fmt)
    new_v = hysteresis_blend(octahedral.interior(state_v), m_v, h, state_fmt)
    tiles_c = octahedral.fill_border(octahedral.with_interior(state_c, new_c))
    tiles_v = octahedral.fill_border(octahedral.with_interior(state_v, new_v))
    return tiles_c, tiles_v
