"""Python binding of the GB300 probe-streaming library (include/probe_stream.h).

Argument marshalling only: every step of the per-frame path (weights, blend,
guard band, change flags, selection, packing) runs in the CUDA kernels of
``libprobestream.so``. PyTorch provides device memory and streams. Importing
this package fails loudly when the library has not been built; there is no
CPU fallback.

Low-level functions carry the C names (``probe_volume_create``,
``probe_update``, ``probe_select_and_pack``, ...); :class:`ProbeVolume` wraps a
volume handle for convenience.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libprobestream.so")

FMT = {"f32": 0, "f16": 1, "bf16": 2}
CODE = {"uf10": 0, "unorm10": 1}
KERNEL = {"auto": 0, "simt": 1, "tcgen05": 2}
KERNEL_NAME = {v: k for k, v in KERNEL.items()}

PV_OK, PV_PENDING = 0, 1
STATUS = {0: "PV_OK", 1: "PV_PENDING", -1: "PV_ERR_INVALID", -2: "PV_ERR_OOM", -3: "PV_ERR_CUDA",
          -4: "PV_ERR_BUSY", -5: "PV_ERR_TIMEOUT", -6: "PV_ERR_RANGE", -7: "PV_ERR_UNSUPPORTED"}


class PVError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class pv_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("rays_per_probe", C.c_int32), ("color_interior", C.c_int32),
                ("vis_interior", C.c_int32), ("hysteresis", C.c_float), ("sharpness", C.c_float),
                ("state_fmt", C.c_int32), ("operand_fmt", C.c_int32), ("color_code", C.c_int32),
                ("color_lsb", C.c_int32), ("first_frame_no_hysteresis", C.c_int32),
                ("kernel", C.c_int32)]


class pv_volume_info(C.Structure):
    _fields_ = [("probes", C.c_int32), ("rays", C.c_int32), ("color_tile", C.c_int32),
                ("vis_tile", C.c_int32), ("blocks_w", C.c_int32), ("blocks_h", C.c_int32),
                ("color_width", C.c_int32), ("color_height", C.c_int32),
                ("color_pitch_bytes", C.c_int32), ("vis_width", C.c_int32),
                ("vis_height", C.c_int32), ("vis_pitch_bytes", C.c_int32), ("kernel", C.c_int32),
                ("state_bytes_per_texel", C.c_int32), ("device_bytes", C.c_uint64),
                ("error_word", C.c_void_p)]


class pv_tune_result(C.Structure):
    _fields_ = [("probes_per_item", C.c_int32), ("ray_stages", C.c_int32), ("weight_stages", C.c_int32),
                ("tmem_stages", C.c_int32), ("ctas", C.c_int32), ("candidates", C.c_int32),
                ("from_cache", C.c_int32), ("best_us", C.c_float), ("default_us", C.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class pv_frame(C.Structure):
    _fields_ = [("color_planes", C.c_void_p), ("vis_planes", C.c_void_p),
                ("index_c", C.c_void_p), ("index_v", C.c_void_p),
                ("delta_c", C.c_void_p), ("delta_v", C.c_void_p),
                ("count_c_dev", C.c_void_p), ("count_v_dev", C.c_void_p),
                ("count_c", C.c_int64), ("count_v", C.c_int64), ("frame", C.c_uint64)]


class pv_view_opts(C.Structure):
    _fields_ = [("active", C.c_void_p), ("budget", C.c_int32), ("threshold_c", C.c_int32),
                ("threshold_v", C.c_int32)]


class pv_server_desc(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_uint64), ("max_slots", C.c_int32), ("max_batch", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libprobestream.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = C.CDLL(LIB_PATH)
    vp, i32, u64 = C.c_void_p, C.c_int32, C.c_uint64
    sigs = {
        "pv_status_string": (C.c_char_p, [i32]),
        "pv_last_error": (C.c_char_p, []),
        "pv_version": (C.c_char_p, []),
        "pv_ray_directions": (i32, [u64, u64, u64, i32, vp]),
        "probe_volume_bytes": (i32, [C.POINTER(pv_desc), C.POINTER(u64)]),
        "probe_volume_create": (i32, [C.POINTER(pv_desc), C.POINTER(vp)]),
        "probe_volume_destroy": (i32, [vp]),
        "probe_volume_info": (i32, [vp, C.POINTER(pv_volume_info)]),
        "probe_update": (i32, [vp, vp, vp, vp, vp]),
        "probe_update_weights": (i32, [vp, vp, vp]),
        "probe_update_blend": (i32, [vp, vp, vp, vp]),
        "probe_select_and_pack": (i32, [vp, C.POINTER(pv_frame), i32, vp]),
        "probe_update_host": (i32, [vp, vp, vp, vp, vp]),
        "probe_frame_download": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "probe_frame_download_async": (i32, [vp, vp, vp, vp, vp, vp, C.POINTER(u64), vp]),
        "probe_frame_wait": (i32, [vp, u64]),
        "probe_volume_export_state": (i32, [vp, vp, vp, vp, vp, C.POINTER(u64), vp]),
        "probe_volume_import_state": (i32, [vp, vp, vp, vp, vp, u64, vp]),
        "probe_update_static": (i32, [C.POINTER(pv_desc), u64, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "probe_batch_create": (i32, [C.POINTER(vp), i32, i32, C.POINTER(vp)]),
        "probe_batch_destroy": (i32, [vp]),
        "probe_batch_info": (i32, [vp, C.POINTER(i32)]),
        "probe_batch_update": (i32, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), vp]),
        "probe_batch_select_and_pack": (i32, [vp, C.POINTER(pv_frame), vp]),
        "probe_batch_tune": (i32, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), i32, C.POINTER(i32), vp]),
        "probe_batch_autotune": (i32, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), i32, C.c_char_p,
                                       C.POINTER(pv_tune_result), vp]),
        "pv_server_create": (i32, [C.POINTER(pv_server_desc), C.POINTER(vp)]),
        "pv_server_destroy": (i32, [vp]),
        "pv_server_open": (i32, [vp, i32, C.POINTER(pv_desc)]),
        "pv_server_close": (i32, [vp, i32]),
        "pv_server_status": (i32, [vp, i32, C.POINTER(i32), C.POINTER(u64), C.POINTER(i32)]),
        "pv_server_volume": (i32, [vp, i32, C.POINTER(vp)]),
        "pv_submit": (i32, [vp, i32, vp, vp, vp, C.POINTER(u64)]),
        "pv_server_tick": (i32, [vp, vp, C.POINTER(u64)]),
        "pv_poll": (i32, [vp, u64, C.POINTER(pv_frame)]),
        "pv_client_create": (i32, [C.POINTER(pv_desc), C.POINTER(vp)]),
        "pv_client_destroy": (i32, [vp]),
        "pv_client_apply": (i32, [vp, C.POINTER(pv_frame), vp]),
        "pv_client_textures": (i32, [vp, C.POINTER(vp), C.POINTER(vp)]),
        "pv_view_create": (i32, [vp, C.POINTER(vp)]),
        "pv_view_destroy": (i32, [vp]),
        "pv_view_select_and_pack": (i32, [vp, C.POINTER(pv_frame), i32, vp]),
        "pv_view_set_options": (i32, [vp, C.POINTER(pv_view_opts)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(status: int, where: str):
    if status < 0:
        raise PVError(status, where, lib.pv_last_error().decode())
    return status


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr()
    return t.ctypes.data  # numpy


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ C names
def make_desc(spec=None, **kw) -> pv_desc:
    """pv_desc from an object with VolumeSpec-like attributes and/or keyword overrides."""
    def get(name, default=None):
        if name in kw:
            return kw[name]
        return getattr(spec, name, default) if spec is not None else default
    d = pv_desc()
    d.nx, d.ny, d.nz = int(get("nx")), int(get("ny")), int(get("nz"))
    d.rays_per_probe = int(get("rays"))
    d.color_interior = int(get("color_interior", 6))
    d.vis_interior = int(get("vis_interior", 14))
    d.hysteresis = float(get("hysteresis", 0.97))
    d.sharpness = float(get("sharpness", 50.0))
    d.state_fmt = FMT[get("state_fmt", "f16")]
    d.operand_fmt = FMT[get("operand_fmt", "f32")]
    d.color_code = CODE[get("color_code", "uf10")]
    d.color_lsb = int(bool(get("color_lsb", False)))
    d.first_frame_no_hysteresis = int(bool(get("first_frame_no_hysteresis", False)))
    d.kernel = KERNEL[get("kernel", "auto")]
    return d


def pv_ray_directions(seed: int, volume: int, frame: int, rays: int):
    import numpy as np
    out = np.empty((rays, 3), dtype=np.float32)
    _check(lib.pv_ray_directions(seed, volume, frame, rays, out.ctypes.data), "pv_ray_directions")
    return out


def probe_volume_bytes(desc: pv_desc) -> int:
    n = C.c_uint64()
    _check(lib.probe_volume_bytes(C.byref(desc), C.byref(n)), "probe_volume_bytes")
    return n.value


def probe_volume_create(desc: pv_desc) -> int:
    h = C.c_void_p()
    _check(lib.probe_volume_create(C.byref(desc), C.byref(h)), "probe_volume_create")
    return h.value


def probe_volume_destroy(vol: int):
    _check(lib.probe_volume_destroy(vol), "probe_volume_destroy")


def probe_volume_info(vol: int) -> pv_volume_info:
    info = pv_volume_info()
    _check(lib.probe_volume_info(vol, C.byref(info)), "probe_volume_info")
    return info


def probe_update(vol: int, radiance, dist, dirs, stream=None):
    _check(lib.probe_update(vol, _ptr(radiance), _ptr(dist), _ptr(dirs), _stream(stream)),
           "probe_update")


def probe_update_weights(vol: int, dirs, stream=None):
    _check(lib.probe_update_weights(vol, _ptr(dirs), _stream(stream)), "probe_update_weights")


def probe_update_blend(vol: int, radiance, dist, stream=None):
    _check(lib.probe_update_blend(vol, _ptr(radiance), _ptr(dist), _stream(stream)),
           "probe_update_blend")


def probe_select_and_pack(vol: int, want_host_counts: bool = False, stream=None) -> pv_frame:
    fr = pv_frame()
    _check(lib.probe_select_and_pack(vol, C.byref(fr), int(want_host_counts), _stream(stream)),
           "probe_select_and_pack")
    return fr


def probe_update_host(vol: int, radiance, dist, dirs, stream=None):
    _check(lib.probe_update_host(vol, _ptr(radiance), _ptr(dist), _ptr(dirs), _stream(stream)),
           "probe_update_host")


def probe_frame_download(vol: int, color=None, vis=None, delta_c=None, delta_v=None, counts=None,
                         stream=None):
    _check(lib.probe_frame_download(vol, _ptr(color), _ptr(vis), _ptr(delta_c), _ptr(delta_v),
                                    _ptr(counts), _stream(stream)), "probe_frame_download")


def probe_frame_download_async(vol: int, color=None, vis=None, delta_c=None, delta_v=None,
                               counts=None, stream=None) -> int:
    t = C.c_uint64()
    _check(lib.probe_frame_download_async(vol, _ptr(color), _ptr(vis), _ptr(delta_c), _ptr(delta_v),
                                          _ptr(counts), C.byref(t), _stream(stream)),
           "probe_frame_download_async")
    return t.value


def probe_frame_wait(vol: int, ticket: int):
    _check(lib.probe_frame_wait(vol, ticket), "probe_frame_wait")


def probe_volume_export_state(vol: int, tiles_c, tiles_v, last_c, last_v, stream=None) -> int:
    f = C.c_uint64()
    _check(lib.probe_volume_export_state(vol, _ptr(tiles_c), _ptr(tiles_v), _ptr(last_c),
                                         _ptr(last_v), C.byref(f), _stream(stream)),
           "probe_volume_export_state")
    return f.value


def probe_volume_import_state(vol: int, tiles_c, tiles_v, last_c, last_v, frame: int, stream=None):
    _check(lib.probe_volume_import_state(vol, _ptr(tiles_c), _ptr(tiles_v), _ptr(last_c),
                                         _ptr(last_v), int(frame), _stream(stream)),
           "probe_volume_import_state")


def probe_update_static(desc: pv_desc, frame: int, radiance, dist, dirs, tiles_c, tiles_v, last_c, last_v,
                        changed_bits, stream=None):
    """Allocation-free update on caller buffers (see include/probe_stream.h)."""
    _check(lib.probe_update_static(C.byref(desc), int(frame), _ptr(radiance), _ptr(dist), _ptr(dirs),
                                   _ptr(tiles_c), _ptr(tiles_v), _ptr(last_c), _ptr(last_v),
                                   _ptr(changed_bits), _stream(stream)), "probe_update_static")


# ------------------------------------------------------------------ device views
def _ptr_array(items):
    arr = (C.c_void_p * len(items))()
    for i, t in enumerate(items):
        arr[i] = _ptr(t)
    return arr


def probe_batch_create(vols, probes_per_item: int = 0) -> int:
    arr = _ptr_array(vols)
    out = C.c_void_p()
    _check(lib.probe_batch_create(arr, len(vols), int(probes_per_item), C.byref(out)), "probe_batch_create")
    return out.value


def probe_batch_destroy(batch: int):
    _check(lib.probe_batch_destroy(batch), "probe_batch_destroy")


def probe_batch_info(batch: int) -> int:
    n = C.c_int32()
    _check(lib.probe_batch_info(batch, C.byref(n)), "probe_batch_info")
    return n.value


def probe_batch_update(batch: int, radiance, dist, dirs, stream=None):
    _check(lib.probe_batch_update(batch, _ptr_array(radiance), _ptr_array(dist), _ptr_array(dirs), _stream(stream)),
           "probe_batch_update")


def probe_batch_select_and_pack(batch: int, n: int, stream=None):
    out = (pv_frame * n)()
    _check(lib.probe_batch_select_and_pack(batch, out, _stream(stream)), "probe_batch_select_and_pack")
    return list(out)


def probe_batch_tune(batch: int, radiance, dist, dirs, reps: int = 3, stream=None) -> int:
    n = C.c_int32()
    _check(lib.probe_batch_tune(batch, _ptr_array(radiance), _ptr_array(dist), _ptr_array(dirs), int(reps),
                                C.byref(n), _stream(stream)), "probe_batch_tune")
    return n.value


def probe_batch_autotune(batch: int, radiance, dist, dirs, reps: int = 3, cache_path=None,
                         stream=None) -> pv_tune_result:
    r = pv_tune_result()
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(lib.probe_batch_autotune(batch, _ptr_array(radiance), _ptr_array(dist), _ptr_array(dirs), int(reps),
                                    path, C.byref(r), _stream(stream)), "probe_batch_autotune")
    return r


class _DeviceArray:
    """Exposes a device pointer to torch through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr: int, shape, typestr: str, strides=None):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": strides}


def device_view(ptr: int, shape, dtype, strides_bytes=None):
    """A torch tensor aliasing library-owned device memory."""
    import torch
    typestr = {torch.uint8: "|u1", torch.uint16: "<u2", torch.int16: "<i2",
               torch.uint32: "<u4", torch.float16: "<f2", torch.float32: "<f4"}[dtype]
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr, strides_bytes), device="cuda")


class ProbeVolume:
    """A probe volume on the current CUDA device (see probe_volume_create)."""

    def __init__(self, spec=None, _handle=None, **kw):
        self.desc = make_desc(spec, **kw)
        self._owned = _handle is None
        self.handle = probe_volume_create(self.desc) if _handle is None else _handle
        self.info = probe_volume_info(self.handle)
        self.P = self.info.probes
        self.R = self.info.rays
        self.nc = self.desc.color_interior
        self.nv = self.desc.vis_interior
        self.kernel = KERNEL_NAME[self.info.kernel]

    def close(self):
        if getattr(self, "handle", None):
            if self._owned:
                probe_volume_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, radiance, dist, dirs, stream=None):
        probe_update(self.handle, radiance, dist, dirs, stream)

    def select_and_pack(self, want_host_counts: bool = False, stream=None) -> pv_frame:
        return probe_select_and_pack(self.handle, want_host_counts, stream)

    # views of the last packed frame (valid until the next select_and_pack)
    def color_planes(self, fr: pv_frame):
        import torch
        i = self.info
        full = device_view(fr.color_planes, (3, i.color_height, i.color_pitch_bytes // 2), torch.uint16)
        return full[:, :, :i.color_width]

    def vis_planes(self, fr: pv_frame, with_pad: bool = False):
        import torch
        i = self.info
        full = device_view(fr.vis_planes, (3, i.vis_height, i.vis_pitch_bytes), torch.uint8)
        return full if with_pad else full[:, :, :i.vis_width]

    def index(self, fr: pv_frame, which: str, count: int):
        import torch
        ptr = {"c": fr.index_c, "v": fr.index_v, "dc": fr.delta_c, "dv": fr.delta_v}[which]
        return device_view(ptr, (self.P,), torch.uint16)[:count]

    def counts(self, fr: pv_frame):
        import torch
        return device_view(fr.count_c_dev, (2,), torch.uint32)

    # state transfer (torch tensors, host or device)
    def state_buffers(self, device="cpu"):
        import torch
        dt = torch.float16 if self.desc.state_fmt == FMT["f16"] else torch.float32
        tc, tv = self.nc + 2, self.nv + 2
        return (torch.empty((3, self.P, tc, tc), dtype=dt, device=device),
                torch.empty((2, self.P, tv, tv), dtype=dt, device=device),
                torch.empty((3, self.P, self.nc ** 2), dtype=torch.uint16, device=device),
                torch.empty((2, self.P, self.nv ** 2), dtype=torch.uint16, device=device))

    def export_state(self, stream=None):
        tc, tv, lc, lv = self.state_buffers("cpu")
        f = probe_volume_export_state(self.handle, tc, tv, lc, lv, stream)
        return tc, tv, lc, lv, f

    def import_state(self, tiles_c, tiles_v, last_c, last_v, frame: int, stream=None):
        probe_volume_import_state(self.handle, tiles_c.contiguous(), tiles_v.contiguous(),
                                  last_c.contiguous(), last_v.contiguous(), frame, stream)


class ProbeBatch:
    """Several ProbeVolumes of equal tile shapes and formats updated together
    (see probe_batch_create). The volumes must outlive the batch."""

    def __init__(self, volumes, probes_per_item: int = 0):
        self.volumes = list(volumes)
        self.handle = probe_batch_create([v.handle for v in self.volumes], probes_per_item)

    @property
    def probes_per_item(self) -> int:
        return probe_batch_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            probe_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, radiance, dist, dirs, stream=None):
        probe_batch_update(self.handle, radiance, dist, dirs, stream)

    def select_and_pack(self, stream=None):
        return probe_batch_select_and_pack(self.handle, len(self.volumes), stream)

    def tune(self, radiance, dist, dirs, reps: int = 3, stream=None) -> int:
        return probe_batch_tune(self.handle, radiance, dist, dirs, reps, stream)

    def autotune(self, radiance, dist, dirs, reps: int = 3, cache_path=None, stream=None) -> dict:
        """Tune the plan (probes per item, ring depths, TMEM stages, CTAs); see probe_batch_autotune."""
        return probe_batch_autotune(self.handle, radiance, dist, dirs, reps, cache_path, stream).as_dict()


PV_PENDING_STATUS = 1


def _desc_kwargs(d: pv_desc) -> dict:
    inv_fmt = {v: k for k, v in FMT.items()}
    inv_code = {v: k for k, v in CODE.items()}
    return dict(nx=d.nx, ny=d.ny, nz=d.nz, rays=d.rays_per_probe, color_interior=d.color_interior,
                vis_interior=d.vis_interior, hysteresis=d.hysteresis, sharpness=d.sharpness,
                state_fmt=inv_fmt[d.state_fmt], operand_fmt=inv_fmt[d.operand_fmt],
                color_code=inv_code[d.color_code], color_lsb=bool(d.color_lsb),
                first_frame_no_hysteresis=bool(d.first_frame_no_hysteresis))


class ProbeServer:
    """The served form (pv_server_*): sessions admitted by device memory and slots, batched
    per tick. open() returns True when admitted, False while waiting."""

    def __init__(self, mem_budget_bytes: int, max_slots: int, max_batch: int = 16):
        d = pv_server_desc(int(mem_budget_bytes), int(max_slots), int(max_batch))
        h = C.c_void_p()
        _check(lib.pv_server_create(C.byref(d), C.byref(h)), "pv_server_create")
        self.handle = h.value
        self.descs = {}

    def close_server(self):
        if getattr(self, "handle", None):
            _check(lib.pv_server_destroy(self.handle), "pv_server_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close_server()
        except Exception:
            pass

    def open(self, client: int, spec=None, **kw) -> bool:
        d = make_desc(spec, **kw)
        st = _check(lib.pv_server_open(self.handle, int(client), C.byref(d)), "pv_server_open")
        self.descs[client] = d
        return st == 0

    def close(self, client: int):
        _check(lib.pv_server_close(self.handle, int(client)), "pv_server_close")
        self.descs.pop(client, None)

    def status(self, client: int = -1):
        a, used, w = C.c_int32(), C.c_uint64(), C.c_int32()
        _check(lib.pv_server_status(self.handle, int(client), C.byref(a), C.byref(used), C.byref(w)),
               "pv_server_status")
        return a.value, used.value, w.value

    def submit(self, client: int, radiance, dist, dirs) -> int:
        t = C.c_uint64()
        _check(lib.pv_submit(self.handle, int(client), _ptr(radiance), _ptr(dist), _ptr(dirs), C.byref(t)),
               "pv_submit")
        return t.value

    def tick(self, stream=None) -> int:
        t = C.c_uint64()
        _check(lib.pv_server_tick(self.handle, _stream(stream), C.byref(t)), "pv_server_tick")
        return t.value

    def volume(self, client: int) -> "ProbeVolume":
        """A view of the admitted client's volume (owned by the server)."""
        h = C.c_void_p()
        _check(lib.pv_server_volume(self.handle, int(client), C.byref(h)), "pv_server_volume")
        return ProbeVolume(None, _handle=h.value, **_desc_kwargs(self.descs[client]))

    def poll(self, ticket: int):
        """None while pending, else the client's pv_frame."""
        fr = pv_frame()
        st = _check(lib.pv_poll(self.handle, int(ticket), C.byref(fr)), "pv_poll")
        return None if st == PV_PENDING_STATUS else fr


class ProbeClient:
    """A client's permanent probe textures on the current CUDA device (pv_client_create);
    ``apply`` decodes one packed frame into them on the GPU."""

    def __init__(self, spec=None, **kw):
        self.desc = make_desc(spec, **kw)
        h = C.c_void_p()
        _check(lib.pv_client_create(C.byref(self.desc), C.byref(h)), "pv_client_create")
        self.handle = h.value
        self.P = self.desc.nx * self.desc.ny * self.desc.nz
        self.tc = self.desc.color_interior + 2
        self.tv = self.desc.vis_interior + 2

    def apply(self, frame: pv_frame, stream=None):
        _check(lib.pv_client_apply(self.handle, C.byref(frame), _stream(stream)), "pv_client_apply")

    def textures(self):
        """(colour [3, P, tc, tc] float32, visibility [2, P, tv, tv] binary16 bits as uint16),
        views of the client's device memory."""
        import torch
        pc, pv_ = C.c_void_p(), C.c_void_p()
        _check(lib.pv_client_textures(self.handle, C.byref(pc), C.byref(pv_)), "pv_client_textures")
        return (device_view(pc.value, (3, self.P, self.tc, self.tc), torch.float32),
                device_view(pv_.value, (2, self.P, self.tv, self.tv), torch.uint16))

    def close(self):
        if getattr(self, "handle", None):
            lib.pv_client_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ProbeView:
    """One client's view of a shared ProbeVolume (pv_view_create): its own last-transmitted
    codes, selection and packed frames. The frame accessors are the volume's."""

    def __init__(self, vol: "ProbeVolume"):
        h = C.c_void_p()
        _check(lib.pv_view_create(vol.handle, C.byref(h)), "pv_view_create")
        self.handle = h.value
        self.vol = vol
        self.desc, self.info, self.P = vol.desc, vol.info, vol.P
        self.nc, self.nv = vol.nc, vol.nv

    def select_and_pack(self, want_host_counts: bool = False, stream=None) -> pv_frame:
        fr = pv_frame()
        _check(lib.pv_view_select_and_pack(self.handle, C.byref(fr), int(want_host_counts), _stream(stream)),
               "pv_view_select_and_pack")
        return fr

    def set_options(self, active=None, budget: int = 0, threshold_c: int = 0, threshold_v: int = 0):
        """Per-client knobs: active (device uint8 [P] tensor, kept alive here), probe budget per
        texture and frame, change thresholds in code steps (see pv_view_set_options)."""
        self._active = active
        o = pv_view_opts(_ptr(active), int(budget), int(threshold_c), int(threshold_v))
        _check(lib.pv_view_set_options(self.handle, C.byref(o)), "pv_view_set_options")

    color_planes = ProbeVolume.color_planes
    vis_planes = ProbeVolume.vis_planes
    index = ProbeVolume.index
    counts = ProbeVolume.counts

    def close(self):
        if getattr(self, "handle", None):
            lib.pv_view_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
