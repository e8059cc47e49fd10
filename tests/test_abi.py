"""The C ABI library builds for sm_103a, loads, and exports every function that
include/nlos.h declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "nlos.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+(nlos_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_03747_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["nlos_scene_create", "nlos_simulate", "nlos_simulate_backward",
                     "nlos_serve_submit", "nlos_forward", "nlos_detect", "nlos_jitter",
                     "nlos_noise", "nlos_philox", "nlos_reduce", "nlos_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared in nlos.h but not exported: {missing}"


def test_struct_layouts_match_binding(lib):
    from paper_2506_03747_gb300 import nlos
    nlos.load()
    p = nlos.Params()
    lib.nlos_params_default(ctypes.byref(p))
    assert p.struct_size == ctypes.sizeof(nlos.Params)
    assert p.num_bins == 256 and p.scan_nx == 32 and p.cos_mode == nlos.COS_OBJECT


def test_host_side_argument_checks_without_gpu(lib):
    """Calls that fail validation before touching the device return EINVAL and
    set a message (no CUDA context needed)."""
    from paper_2506_03747_gb300 import nlos
    nlos.load()
    p = nlos.Params()
    lib.nlos_params_default(ctypes.byref(p))
    h = ctypes.c_void_p()
    lib.nlos_scene_create.restype = ctypes.c_int
    lib.nlos_scene_create.argtypes = [ctypes.POINTER(nlos.Params), ctypes.c_void_p,
                                      ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]
    p.num_bins = 0
    assert lib.nlos_scene_create(ctypes.byref(p), None, 0, 0, None, ctypes.byref(h)) == nlos.EINVAL
    assert b"num_bins" in nlos.load().nlos_last_error()
    lib.nlos_params_default(ctypes.byref(p))
    p.struct_size = 4
    assert lib.nlos_scene_create(ctypes.byref(p), None, 0, 0, None, ctypes.byref(h)) == nlos.EINVAL
    lib.nlos_params_default(ctypes.byref(p))
    p.bin_mode = nlos.BIN_SPLAT  # splat without jitter width
    assert lib.nlos_scene_create(ctypes.byref(p), None, 0, 0, None, ctypes.byref(h)) == nlos.EINVAL
    assert lib.nlos_simulate(None, None, None, None, None, None) == nlos.EINVAL
    assert lib.nlos_scene_set_occluders(None, None, 0, None) == nlos.EINVAL
    assert b"scene is NULL" in nlos.load().nlos_last_error()
    assert lib.nlos_scene_set_albedo_depth(None, None, None, None) == nlos.EINVAL
    assert b"scene is NULL" in nlos.load().nlos_last_error()
    assert lib.nlos_measure_peaks(None, None) == nlos.EINVAL
    pk = nlos.Peaks()
    pk.struct_size = 8  # too small for the struct: rejected before any device work
    assert lib.nlos_measure_peaks(ctypes.byref(pk), None) == nlos.EINVAL
    assert lib.nlos_abi_version() == 1


def test_no_cpu_fallback_when_library_missing(tmp_path):
    from paper_2506_03747_gb300 import nlos
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        nlos.load(str(tmp_path / "missing.so")) if nlos._lib is None else (_ for _ in ()).throw(
            RuntimeError("no CPU fallback"))
