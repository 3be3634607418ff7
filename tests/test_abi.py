"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and exports every
function include/*.h declares; host-only entry points behave (no GPU needed)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "pv_build", os.path.join(ROOT, "paper_2103_05875_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def built_lib():
    path = _build_module().build()
    return ctypes.CDLL(path), path


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s+\**([A-Za-z_]\w*)\s*\(", text, re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_path_entry_points():
    names = _declared_functions()
    for required in ("probe_volume_create", "probe_update", "probe_select_and_pack",
                     "probe_volume_destroy", "pv_ray_directions"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    lib, path = built_lib
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, f"{path} lacks {missing}"


def test_library_targets_sm_103a(built_lib):
    b = _build_module()
    assert "arch=compute_103a,code=sm_103a" in " ".join(b.ARCH)


def test_host_only_entry_points(built_lib):
    import paper_2103_05875_gb300 as pv
    import pv_workload as wl
    d = pv.pv_ray_directions(42, 3, 7, 256)
    ref = wl.ray_directions(42, 3, 7, 256)
    assert np.abs(d - ref).max() < 1e-6
    np.testing.assert_allclose(np.linalg.norm(d.astype(np.float64), axis=1), 1.0, atol=1e-6)
    n = pv.probe_volume_bytes(pv.make_desc(wl.config2()))
    assert 10e6 < n < 40e6
    with pytest.raises(pv.PVError) as e:
        pv.probe_volume_bytes(pv.make_desc(wl.config2(), nx=64, ny=64, nz=64))
    assert e.value.status == -6
    with pytest.raises(pv.PVError) as e:
        pv.probe_volume_bytes(pv.make_desc(wl.config2(), hysteresis=1.5))
    assert e.value.status == -1
    assert pv.lib.pv_status_string(-5) == b"PV_ERR_TIMEOUT"


def test_select_kernel_reciprocal_division_is_exact():
    """The select kernel divides small indices (x < 2^16) by d <= 2^15 as umulhi(2x, ceil(2^31/d));
    the run-length table in its source must hold ceil(2^31/d) for d = 1..8."""
    import re
    x = np.arange(1 << 16, dtype=np.uint64)
    for d in list(range(1, 257)) + [4097, 12345, 32767, 1 << 15]:
        m = ((1 << 31) + d - 1) // d
        np.testing.assert_array_equal(((2 * x) * m) >> 32, x // d, err_msg=f"d={d}")
    src = open(os.path.join(ROOT, "paper_2103_05875_gb300", "csrc", "pv_select_pack.cu")).read()
    table = re.search(r"c_rcp_run\[[^\]]*\]\s*=\s*\{([^}]*)\}", src).group(1)
    vals = [int(v.strip().rstrip("u"), 16) for v in table.split(",")]
    assert vals[1:] == [((1 << 31) + d - 1) // d for d in range(1, len(vals))]


def test_view_and_client_entry_points_reject_bad_arguments_before_any_cuda_call(built_lib):
    """Host-side validation of the view and client entry points (no device needed)."""
    import ctypes as C

    import paper_2103_05875_gb300 as pv
    import pv_workload as wl
    lib = pv.lib
    h = C.c_void_p()
    # a description that fails validation never reaches the device
    bad = pv.make_desc(wl.config2(), hysteresis=1.5)
    assert lib.pv_client_create(C.byref(bad), C.byref(h)) == -1 and not h.value
    too_big = pv.make_desc(wl.config2(), nx=64, ny=64, nz=64)
    assert lib.pv_client_create(C.byref(too_big), C.byref(h)) == -6
    assert lib.pv_client_create(C.byref(pv.make_desc(wl.config2())), None) == -1
    fr = pv.pv_frame()
    assert lib.pv_client_apply(None, C.byref(fr), None) == -1
    assert lib.pv_client_textures(None, None, None) == -1
    assert lib.pv_client_destroy(None) == 0
    # views: NULL volume, NULL view, and negative knobs
    assert lib.pv_view_create(None, C.byref(h)) == -1
    assert lib.pv_view_select_and_pack(None, C.byref(fr), 0, None) == -1
    opts = pv.pv_view_opts(None, 0, 0, 0)
    assert lib.pv_view_set_options(None, C.byref(opts)) == -1
    assert lib.pv_view_destroy(None) == 0
    assert b"NULL" in lib.pv_last_error()
