"""Change selection, probe index buffer and lossless-video bit packing (and its inverse).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package.

Section 3.4 ("Light Probe Change Thresholding"): per client the server keeps
one last-transmitted texture for irradiance and one for visibility; a probe is
a candidate iff it is not texel-for-texel identical to its last transmitted
state, and its data is written to the last-transmitted texture when it is
sent. Readings: the comparison is on the transmitted codes; colour and
visibility are selected separately; a probe never sent is changed; every
changed probe is sent (no budget, no view culling).

Section 3.4 ("Light Probe Repacking", "Light Probe Update Textures"): only the
selected probes go out, guard bands removed, in a temporary update texture,
with a probe index buffer of one 2-byte unsigned integer per probe, reduced by
delta encoding. Reading: slots are filled in ascending probe id, slot k sits
at block (k div B_w, k mod B_w) of a block grid B_w = nx*ny wide and
B_h = nz high; unused slots are zero.

Section 3.3 ("Encoding Irradiance", memory-layout figure): each 10-bit colour
code is bit-shifted into a 16-bit Y/U/V value with the unused bits zero; the
tuples are reordered into planar Y, U, V. Reading: R->Y, G->U, B->V, code in
the most significant bits (code << 6); ``lsb=True`` keeps it in the low bits.

Section 3.3 ("Encoding Visibility"): the RG16F texel's four bytes are spread
over 8-bit Y, U, V in the repeating order YUVY, UVYU, VYUV, and the plane
width grows from x to x' = ceil(4x/3). Reading: per atlas row the byte
stream is (R.lo, R.hi, G.lo, G.hi) per texel, byte k goes to plane k mod 3 at
column k div 3, trailing pad bytes are zero.
"""
from __future__ import annotations

import math

import numpy as np

from . import numerics, octahedral

SENTINEL = 0xFFFF   # last-transmitted code of a probe that was never sent


def color_codes(tiles_c: np.ndarray, kind: str = "uf10") -> np.ndarray:
    """[3, P, n+2, n+2] stored values -> [3, P, n*n] uint16 10-bit codes."""
    return numerics.color_code(octahedral.interior(tiles_c), kind)


def vis_codes(tiles_v: np.ndarray) -> np.ndarray:
    """[2, P, n+2, n+2] stored values -> [2, P, n*n] uint16 RG16F bit patterns."""
    return numerics.fp16_bits(numerics.round_fp16(octahedral.interior(tiles_v)))


def changed(codes: np.ndarray, last: np.ndarray, sent: np.ndarray) -> np.ndarray:
    """[C, P, T] codes vs last-transmitted codes -> [P] bool (not identical, or never sent)."""
    differs = np.any(codes != last, axis=(0, 2))
    return differs | ~np.asarray(sent, dtype=bool)


def changed_beyond(codes: np.ndarray, last: np.ndarray, sent: np.ndarray, threshold: int) -> np.ndarray:
    """Section 3.4's change test with a threshold: [C, P, T] codes vs last-transmitted codes ->
    [P] bool, true when some texel's code moved by more than ``threshold`` code steps (or the
    probe was never sent). Reading: colour codes are 10-bit unsigned integers, visibility codes
    binary16 bit patterns of non-negative values, so a step is one code value / one ulp;
    threshold 0 is the texel-for-texel rule."""
    dist = np.abs(codes.astype(np.int64) - last.astype(np.int64))
    return np.any(dist > threshold, axis=(0, 2)) | ~np.asarray(sent, dtype=bool)


def budget_select(flags: np.ndarray, active, cursor: int, budget: int):
    """Per-client probe budget (Section 3.4, the per-client 'knob'): of the changed, active
    probes, the first ``budget`` in cyclic probe order from ``cursor`` (0: no limit). Returns the
    kept flags and the next cursor (one past the last kept probe; unchanged if none kept).
    Reading: the cursor walks round-robin so that probes left out are sent on later frames."""
    f = np.asarray(flags, dtype=bool).copy()
    if active is not None:
        f &= np.asarray(active, dtype=bool)
    P = f.size
    if budget <= 0 or int(f.sum()) <= budget:
        kept = f
    else:
        order = np.r_[cursor:P, 0:cursor]
        take = order[f[order]][:budget]
        kept = np.zeros(P, dtype=bool)
        kept[take] = True
    if budget > 0 and kept.any():
        order = np.r_[cursor:P, 0:cursor]
        last = order[kept[order]][-1]
        cursor = (int(last) + 1) % P
    return kept, cursor


def select(flags: np.ndarray):
    """Probe index buffer: (ids ascending uint16, delta-encoded uint16, count)."""
    idx = np.nonzero(np.asarray(flags, dtype=bool))[0]
    if idx.size and idx[-1] > 0xFFFF:
        raise ValueError("probe id exceeds the 2-byte index buffer")
    delta = np.diff(idx, prepend=0) if idx.size else idx
    return idx.astype(np.uint16), delta.astype(np.uint16), int(idx.size)


def undelta(delta: np.ndarray) -> np.ndarray:
    """Inverse of the delta encoding (cumulative sum)."""
    return np.cumsum(np.asarray(delta, dtype=np.int64)).astype(np.uint16)


def block_grid(nx: int, ny: int, nz: int):
    """(B_w, B_h) of the update-texture block grid."""
    return nx * ny, nz


def vis_width(bw: int, n_v: int) -> int:
    """Plane width x' = ceil(4x/3) for an atlas x = bw * n_v texels wide."""
    x = bw * n_v
    return (4 * x + 2) // 3


def pack_color(codes_c: np.ndarray, idx: np.ndarray, bw: int, bh: int, lsb: bool = False):
    """[3, P, n*n] codes + index buffer -> planar Y, U, V uint16 [3, bh*n, bw*n]."""
    n = int(round(math.sqrt(codes_c.shape[-1])))
    planes = np.zeros((3, bh * n, bw * n), dtype=np.uint16)
    shift = 0 if lsb else 6
    for k, p in enumerate(np.asarray(idx, dtype=np.int64)):
        by, bx = divmod(k, bw)
        block = codes_c[:, p, :].reshape(3, n, n).astype(np.uint32) << shift
        planes[:, by * n:(by + 1) * n, bx * n:(bx + 1) * n] = block.astype(np.uint16)
    return planes


def vis_atlas(codes_v: np.ndarray, idx: np.ndarray, bw: int, bh: int) -> np.ndarray:
    """Selected RG16F interiors in slot order: [bh*n, bw*n, 2] uint16 (zeros in empty slots)."""
    n = int(round(math.sqrt(codes_v.shape[-1])))
    atlas = np.zeros((bh * n, bw * n, 2), dtype=np.uint16)
    for k, p in enumerate(np.asarray(idx, dtype=np.int64)):
        by, bx = divmod(k, bw)
        atlas[by * n:(by + 1) * n, bx * n:(bx + 1) * n, :] = \
            codes_v[:, p, :].reshape(2, n, n).transpose(1, 2, 0)
    return atlas


def pack_vis(codes_v: np.ndarray, idx: np.ndarray, bw: int, bh: int) -> np.ndarray:
    """[2, P, n*n] RG16F codes + index buffer -> 8-bit Y, U, V planes [3, bh*n, x']."""
    atlas = vis_atlas(codes_v, idx, bw, bh)
    H, W, _ = atlas.shape
    stream = np.zeros((H, 4 * W), dtype=np.uint8)
    stream[:, 0::4] = atlas[:, :, 0] & 0xFF
    stream[:, 1::4] = atlas[:, :, 0] >> 8
    stream[:, 2::4] = atlas[:, :, 1] & 0xFF
    stream[:, 3::4] = atlas[:, :, 1] >> 8
    n = int(round(math.sqrt(codes_v.shape[-1])))
    xp = vis_width(bw, n)
    planes = np.zeros((3, H, xp), dtype=np.uint8)
    for q in range(3):
        lane = stream[:, q::3]
        planes[q, :, :lane.shape[1]] = lane
    return planes


def unpack_color(planes: np.ndarray, idx: np.ndarray, n: int, bw: int, lsb: bool = False):
    """Inverse of pack_color for the first len(idx) slots -> codes [3, len(idx), n*n]."""
    shift = 0 if lsb else 6
    out = np.zeros((3, len(idx), n * n), dtype=np.uint16)
    for k in range(len(idx)):
        by, bx = divmod(k, bw)
        blk = planes[:, by * n:(by + 1) * n, bx * n:(bx + 1) * n].astype(np.uint32) >> shift
        out[:, k, :] = blk.reshape(3, n * n).astype(np.uint16)
    return out


def unpack_vis(planes: np.ndarray, idx: np.ndarray, n: int, bw: int):
    """Inverse of pack_vis for the first len(idx) slots -> codes [2, len(idx), n*n]."""
    _, H, xp = planes.shape
    W = bw * n
    stream = np.zeros((H, 4 * W), dtype=np.uint8)
    for q in range(3):
        cols = stream[:, q::3].shape[1]
        stream[:, q::3] = planes[q, :, :cols]
    R = stream[:, 0::4].astype(np.uint16) | (stream[:, 1::4].astype(np.uint16) << 8)
    G = stream[:, 2::4].astype(np.uint16) | (stream[:, 3::4].astype(np.uint16) << 8)
    out = np.zeros((2, len(idx), n * n), dtype=np.uint16)
    for k in range(len(idx)):
        by, bx = divmod(k, bw)
        out[0, k] = R[by * n:(by + 1) * n, bx * n:(bx + 1) * n].ravel()
        out[1, k] = G[by * n:(by + 1) * n, bx * n:(bx + 1) * n].ravel()
    return out


def client_apply(client_tiles: np.ndarray, idx: np.ndarray, values: np.ndarray) -> np.ndarray:
    """Client side of Section 3.4: write received interiors of the probes in ``idx`` into the
    permanent textures [C, P, n+2, n+2] and rebuild their guard bands."""
    out = np.array(client_tiles, copy=True)
    ids = np.asarray(idx, dtype=np.int64)
    if ids.size:
        sub = octahedral.with_interior(out[:, ids], values)
        out[:, ids] = octahedral.fill_border(sub)
    return out


# ---------------------------------------------------------------- sizes (Section 3.2)
def full_tile_bits(tile: int) -> int:
    """Uncompressed bits of one probe tile at 32 bits per texel (Eq. 1 and Eq. 2 constants)."""
    return tile * tile * 32


def packed_bytes(count: int, n_c: int, n_v: int):
    """Payload bytes of the selected interiors: (colour 3 x 16-bit, visibility 4 x 8-bit)."""
    return count * n_c * n_c * 3 * 2, count * n_v * n_v * 4
