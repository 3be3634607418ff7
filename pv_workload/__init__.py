"""Seeded synthetic inputs for irradiance-volume probe updates.

This module is shared by the FP64 oracle (``oracle/``), the tests and the
benchmark. It only *draws inputs*: traced-ray radiance and hit distances, the
per-frame ray directions, and the workload descriptions. It holds none of the
blend, selection or packing arithmetic of the method.

Every random number comes from one counter-based generator, SplitMix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): the i-th output of a stream keyed by ``k`` is
``mix64(k + (i + 1) * 0x9E3779B97F4A7C15)``. Keys for sub-streams are derived
by chaining that same function.

Ray directions follow the usual irradiance-probe recipe (a spherical Fibonacci
set of R points, rotated each frame by a uniformly random rotation built from
a uniform unit quaternion, Shoemake, "Uniform random rotations", Graphics Gems
III, 1992). The paper uses 256 rays per probe on the server (Section 4, Full
Pipeline Latency) and leaves the direction set to the DDGI paper it builds on;
the directions are an *input* to the blend, exactly as they would be handed
over by the ray tracer.

Value distributions stand in for the paper's scenes (Section 4, scene
statistics table), which are not available: radiance per channel is
lognormal(mu=-1, sigma=1.5); hit distance is uniform on [0.1, 10] with 10% of
rays missing and set to 10.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

KIND_ROTATION = 1
KIND_RADIANCE = 2
KIND_DIST = 3
KIND_STEP = 4
KIND_CLIENTS = 5

BASE_SEED = 210305875


def mix64(z):
    """SplitMix64 output function on uint64 (arrays or scalars), wrapping."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream(key, index):
    """The ``index``-th output (0-based) of the SplitMix64 stream seeded by ``key``."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key) + (idx + np.uint64(1)) * GAMMA)


def derive(seed: int, *parts: int) -> np.uint64:
    """Chain ``stream`` over ``parts`` to obtain the key of a sub-stream."""
    k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    for p in parts:
        k = np.uint64(stream(k, np.uint64(p & 0xFFFFFFFFFFFFFFFF)))
    return k


def u01(x):
    """Uniform double in [0, 1) from the top 53 bits of a uint64."""
    return (np.asarray(x, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def u01_open0(x):
    """Uniform double in (0, 1] from the top 53 bits of a uint64."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


# ---------------------------------------------------------------- directions
def fibonacci_sphere(R: int) -> np.ndarray:
    """Spherical Fibonacci point set, [R, 3] float64 unit vectors.

    z_i = 1 - (2i+1)/R, phi_i = 2*pi*frac(i*(sqrt(5)-1)/2).
    """
    i = np.arange(R, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / R
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    g = (math.sqrt(5.0) - 1.0) / 2.0
    phi = 2.0 * math.pi * np.mod(i * g, 1.0)
    return np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)


def uniform_rotation(seed: int, volume: int, frame: int) -> np.ndarray:
    """3x3 rotation matrix from a uniform unit quaternion (Shoemake 1992)."""
    key = derive(seed, KIND_ROTATION, volume, frame)
    u = u01(stream(key, np.arange(3, dtype=np.uint64)))
    u1, u2, u3 = float(u[0]), float(u[1]), float(u[2])
    s1, s2 = math.sqrt(1.0 - u1), math.sqrt(u1)
    x = s1 * math.sin(2.0 * math.pi * u2)
    y = s1 * math.cos(2.0 * math.pi * u2)
    z = s2 * math.sin(2.0 * math.pi * u3)
    w = s2 * math.cos(2.0 * math.pi * u3)
    return np.array(
        [
            [1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y)],
            [2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x)],
            [2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)],
        ],
        dtype=np.float64,
    )


def ray_directions(seed: int, volume: int, frame: int, R: int) -> np.ndarray:
    """Rotated spherical Fibonacci directions, [R, 3] float64 (d_r = Rot * fib_r)."""
    rot = uniform_rotation(seed, volume, frame)
    return fibonacci_sphere(R) @ rot.T


# ---------------------------------------------------------------- ray payloads
def radiance(seed: int, volume: int, frame: int, P: int, R: int,
             mu: float = -1.0, sigma: float = 1.5) -> np.ndarray:
    """Planar traced radiance [3, P, R] float64, lognormal(mu, sigma) per channel."""
    key = derive(seed, KIND_RADIANCE, volume, frame)
    n = 3 * P * R
    e = np.arange(n, dtype=np.uint64)
    a = u01_open0(stream(key, e * np.uint64(2)))
    b = u01(stream(key, e * np.uint64(2) + np.uint64(1)))
    z = np.sqrt(-2.0 * np.log(a)) * np.cos(2.0 * math.pi * b)
    return np.exp(mu + sigma * z).reshape(3, P, R)


def hit_distance(seed: int, volume: int, frame: int, P: int, R: int,
                 dmin: float = 0.1, dmax: float = 10.0, miss: float = 0.1) -> np.ndarray:
    """Hit distances [P, R] float64: U[dmin, dmax], a ``miss`` fraction set to dmax."""
    key = derive(seed, KIND_DIST, volume, frame)
    n = P * R
    e = np.arange(n, dtype=np.uint64)
    a = u01(stream(key, e * np.uint64(2)))
    b = u01(stream(key, e * np.uint64(2) + np.uint64(1)))
    d = dmin + (dmax - dmin) * a
    d = np.where(b < miss, dmax, d)
    return d.reshape(P, R)


def step_mask(seed: int, volume: int, P: int, fraction: float = 0.2) -> np.ndarray:
    """Seeded Bernoulli(fraction) mask over probes that receive the step change."""
    key = derive(seed, KIND_STEP, volume)
    return u01(stream(key, np.arange(P, dtype=np.uint64))) < fraction


# ---------------------------------------------------------------- workloads
@dataclasses.dataclass(frozen=True)
class VolumeSpec:
    """Shape and blend parameters of one irradiance volume (see the C header's pv_desc)."""
    nx: int
    ny: int
    nz: int
    rays: int
    color_interior: int = 6
    vis_interior: int = 14
    hysteresis: float = 0.97
    sharpness: float = 50.0
    state_fmt: str = "f16"        # "f32" | "f16"
    operand_fmt: str = "f32"      # "f32" | "f16" | "bf16"
    color_code: str = "uf10"      # "uf10" | "unorm10"
    color_lsb: bool = False
    first_frame_no_hysteresis: bool = False

    @property
    def probes(self) -> int:
        return self.nx * self.ny * self.nz


@dataclasses.dataclass(frozen=True)
class FrameStream:
    """A seeded sequence of traced frames for one volume.

    mode "noisy": fresh rotation and fresh ray payloads every frame (the
    throughput worst case: nearly every probe changes).
    mode "stationary": rotation and payloads drawn once and held, so that only
    the step change moves texels (the paper assumes converged irradiance with
    scene changes as the only source of variance, Section 3.4).
    In both modes a seeded ``step_fraction`` of probes has its radiance
    multiplied by ``step_gain`` from frame ``step_frame`` on.
    """
    spec: VolumeSpec
    seed: int
    volume: int = 0
    mode: str = "noisy"
    step_frame: int = 30
    step_fraction: float = 0.2
    step_gain: float = 4.0

    def _key_frame(self, frame: int) -> int:
        return frame if self.mode == "noisy" else 0

    def directions(self, frame: int) -> np.ndarray:
        """[R, 3] float32 ray directions for ``frame`` (as the tracer hands them over)."""
        d = ray_directions(self.seed, self.volume, self._key_frame(frame), self.spec.rays)
        return d.astype(np.float32)

    def radiance(self, frame: int) -> np.ndarray:
        """[3, P, R] float32 radiance for ``frame`` (step change applied)."""
        P, R = self.spec.probes, self.spec.rays
        L = radiance(self.seed, self.volume, self._key_frame(frame), P, R)
        if self.step_frame is not None and frame >= self.step_frame and self.step_fraction > 0:
            m = step_mask(self.seed, self.volume, P, self.step_fraction)
            L[:, m, :] *= self.step_gain
        return L.astype(np.float32)

    def dist(self, frame: int) -> np.ndarray:
        """[P, R] float32 hit distances for ``frame``."""
        P, R = self.spec.probes, self.spec.rays
        return hit_distance(self.seed, self.volume, self._key_frame(frame), P, R).astype(np.float32)


def config_seed(config_id: int) -> int:
    return BASE_SEED + config_id


def config1() -> VolumeSpec:
    """Plain FP32 single volume: 4x4x4 probes, 64 rays, FP32 state."""
    return VolumeSpec(4, 4, 4, 64, state_fmt="f32", operand_fmt="f32")


def config2(operand_fmt: str = "f32") -> VolumeSpec:
    """16x16x16 probes, 256 rays, FP16 state (config 3 = same with f16/bf16 operands)."""
    return VolumeSpec(16, 16, 16, 256, state_fmt="f16", operand_fmt=operand_fmt)


BATCHED_SIZES: Tuple[Tuple[int, int, int], ...] = (
    (8, 4, 8), (8, 8, 16), (16, 4, 16), (16, 8, 16), (16, 8, 24), (24, 8, 24),
    (24, 8, 32), (32, 8, 32), (8, 4, 16), (16, 8, 32), (24, 4, 24), (32, 4, 32),
)
BATCHED_RAYS: Tuple[int, ...] = (128, 192, 256)


def config4(operand_fmt: str = "f32") -> List[VolumeSpec]:
    """Twelve volumes of uneven sizes, rays cycling 128/192/256, FP16 state (37,376 probes)."""
    return [VolumeSpec(nx, ny, nz, BATCHED_RAYS[i % 3], state_fmt="f16", operand_fmt=operand_fmt)
            for i, (nx, ny, nz) in enumerate(BATCHED_SIZES)]


@dataclasses.dataclass(frozen=True)
class ClientArrival:
    client: int
    arrive_s: float
    session_s: float
    spec: VolumeSpec


def served_clients(n_clients: int = 64, rate_hz: float = 4.0, mean_session_s: float = 8.0,
                   seed: Optional[int] = None, operand_fmt: str = "f32") -> List[ClientArrival]:
    """Poisson(rate) arrivals with exponential session lengths; volume sizes from the batched list."""
    seed = config_seed(5) if seed is None else seed
    key = derive(seed, KIND_CLIENTS)
    u = u01_open0(stream(key, np.arange(3 * n_clients, dtype=np.uint64))).reshape(n_clients, 3)
    t = 0.0
    out = []
    for c in range(n_clients):
        t += -math.log(u[c, 0]) / rate_hz
        sess = -math.log(u[c, 1]) * mean_session_s
        i = int(u[c, 2] * len(BATCHED_SIZES)) % len(BATCHED_SIZES)
        nx, ny, nz = BATCHED_SIZES[i]
        spec = VolumeSpec(nx, ny, nz, BATCHED_RAYS[i % 3], state_fmt="f16", operand_fmt=operand_fmt)
        out.append(ClientArrival(c, t, sess, spec))
    return out


def to_operand(x: np.ndarray, fmt: str):
    """Cast float32 inputs to the operand format; returns a torch CPU tensor.

    f16/bf16 use round-to-nearest-even casts. The oracle receives the very same
    (rounded) values, converted exactly back to float64.
    """
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    if fmt == "f32":
        return t
    if fmt == "f16":
        return t.to(torch.float16)
    if fmt == "bf16":
        return t.to(torch.bfloat16)
    raise ValueError(fmt)
