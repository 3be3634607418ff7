"""A probe volume stepped frame by frame: blend, guard band, codes, selection, packing.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package.

Arrays use the same layouts as the CUDA library so that states can be moved
between the two:

  colour tiles  [3, P, n_c+2, n_c+2]   (R, G, B planes)
  vis tiles     [2, P, n_v+2, n_v+2]   (mean distance, mean squared distance)
  last codes    colour [3, P, n_c^2] uint16, vis [2, P, n_v^2] uint16,
                0xFFFF for a probe never sent
  probe id      p = x + nx*(y + ny*z)

Every tile value is a float64 holding a number representable in the state
format, so the stored state converts to float16/float32 without rounding.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from . import blend, numerics, select_pack


@dataclasses.dataclass
class Frame:
    """One packed update, as handed to the (out-of-scope) video encoder."""
    flags_c: np.ndarray
    flags_v: np.ndarray
    idx_c: np.ndarray
    idx_v: np.ndarray
    delta_c: np.ndarray
    delta_v: np.ndarray
    count_c: int
    count_v: int
    planes_c: np.ndarray   # [3, bh*n_c, bw*n_c] uint16
    planes_v: np.ndarray   # [3, bh*n_v, x'] uint8


class OracleVolume:
    """FP64 reference for one probe volume (Sections 3.2-3.4)."""

    def __init__(self, spec, state_fmt: Optional[str] = None):
        self.spec = spec
        self.P = spec.nx * spec.ny * spec.nz
        self.n_c = spec.color_interior
        self.n_v = spec.vis_interior
        self.state_fmt = state_fmt or spec.state_fmt
        # the library stores hysteresis and sharpness as float32
        self.h = float(np.float32(spec.hysteresis))
        self.s = float(np.float32(spec.sharpness))
        self.bw, self.bh = select_pack.block_grid(spec.nx, spec.ny, spec.nz)
        self.tiles_c = np.zeros((3, self.P, self.n_c + 2, self.n_c + 2))
        self.tiles_v = np.zeros((2, self.P, self.n_v + 2, self.n_v + 2))
        self.last_c = np.full((3, self.P, self.n_c ** 2), select_pack.SENTINEL, dtype=np.uint16)
        self.last_v = np.full((2, self.P, self.n_v ** 2), select_pack.SENTINEL, dtype=np.uint16)
        self.sent_c = np.zeros(self.P, dtype=bool)
        self.sent_v = np.zeros(self.P, dtype=bool)
        self.frame = 0

    # ------------------------------------------------------------ state I/O
    def load_state(self, tiles_c, tiles_v, last_c, last_v, frame: int = 0):
        """Replace the whole state (values must be representable in the state format)."""
        self.tiles_c = np.asarray(tiles_c, dtype=np.float64).copy()
        self.tiles_v = np.asarray(tiles_v, dtype=np.float64).copy()
        self.last_c = np.asarray(last_c, dtype=np.uint16).copy()
        self.last_v = np.asarray(last_v, dtype=np.uint16).copy()
        self.sent_c = ~np.all(self.last_c == select_pack.SENTINEL, axis=(0, 2))
        self.sent_v = ~np.all(self.last_v == select_pack.SENTINEL, axis=(0, 2))
        self.frame = frame

    # ------------------------------------------------------------ per-frame steps
    def update(self, radiance, dist, dirs):
        """Blend one frame of traced rays into the tiles (and refill the guard bands)."""
        self.tiles_c, self.tiles_v = blend.update(
            self.tiles_c, self.tiles_v, radiance, dist, dirs,
            hysteresis=self.h, sharpness=self.s, state_fmt=self.state_fmt,
            first_frame=(self.frame == 0),
            first_frame_no_hysteresis=self.spec.first_frame_no_hysteresis)
        self.frame += 1

    def codes(self):
        return (select_pack.color_codes(self.tiles_c, self.spec.color_code),
                select_pack.vis_codes(self.tiles_v))

    def select_and_pack(self, threshold_c: int = 0, threshold_v: int = 0, active=None, budget: int = 0) -> Frame:
        """Compare with last-transmitted codes, select, pack, and record what is sent.

        Defaults are Section 3.4's rule (every probe not texel-for-texel identical). The
        options are the per-client selection knobs of the same section: a change threshold in
        code steps, an active-probe mask and a per-frame probe budget taken round-robin
        (separate cursors for the colour and visibility textures).
        """
        codes_c, codes_v = self.codes()
        fc = select_pack.changed_beyond(codes_c, self.last_c, self.sent_c, threshold_c)
        fv = select_pack.changed_beyond(codes_v, self.last_v, self.sent_v, threshold_v)
        if active is not None or budget > 0:
            fc, self.cursor_c = select_pack.budget_select(fc, active, getattr(self, "cursor_c", 0), budget)
            fv, self.cursor_v = select_pack.budget_select(fv, active, getattr(self, "cursor_v", 0), budget)
        idx_c, dc, nc = select_pack.select(fc)
        idx_v, dv, nv = select_pack.select(fv)
        planes_c = select_pack.pack_color(codes_c, idx_c, self.bw, self.bh, self.spec.color_lsb)
        planes_v = select_pack.pack_vis(codes_v, idx_v, self.bw, self.bh)
        ic = idx_c.astype(np.int64)
        iv = idx_v.astype(np.int64)
        self.last_c[:, ic] = codes_c[:, ic]
        self.last_v[:, iv] = codes_v[:, iv]
        self.sent_c[ic] = True
        self.sent_v[iv] = True
        return Frame(fc, fv, idx_c, idx_v, dc, dv, nc, nv, planes_c, planes_v)

    def step(self, radiance, dist, dirs) -> Frame:
        self.update(radiance, dist, dirs)
        return self.select_and_pack()

    # ------------------------------------------------------------ conversions
    def tiles_as(self, dtype):
        """Tiles in the library's storage dtype (exact for representable values)."""
        return self.tiles_c.astype(dtype), self.tiles_v.astype(dtype)
