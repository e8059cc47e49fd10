"""Python binding of the C ABI in ``include/nlos.h`` (ctypes).

Argument marshalling only: every step of the simulator runs in the CUDA
kernels of ``libnlos.so``. PyTorch supplies device memory and streams. There
is no CPU fallback: if the library is missing or CUDA is unavailable, calls
raise.

The functions keep the C names without the ``nlos_`` prefix
(``scene_create``, ``simulate``, ``simulate_backward``, ``jitter``, ``reduce``,
``noise``, ``philox``, ``pair_table``, ``server_create``, ``serve_submit``,
``serve_poll``, ``serve_release``, ``server_destroy``).
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the in-tree build; NLOS_LIBRARY may name another build of the same sources
LIB_PATH = os.environ.get("NLOS_LIBRARY") or os.path.join(_HERE, "libnlos.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ECANCELLED, ENOTFOUND = range(8)
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EBUSY",
           6: "ECANCELLED", 7: "ENOTFOUND"}

CONFOCAL, NONCONFOCAL = 0, 1
STANDOFF_EUCLIDEAN, STANDOFF_CONSTANT = 0, 1
COS_NONE, COS_OBJECT, COS_OBJECT_WALL = 0, 1, 2
NOISE_NONE, NOISE_PEAK, NOISE_PAPER_NR = 0, 1, 2
BIN_NEAREST, BIN_SPLAT = 0, 1


class NlosError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"nlos {_STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("scan_nx", ctypes.c_uint32), ("scan_ny", ctypes.c_uint32),
        ("wall_half_x", ctypes.c_double), ("wall_half_y", ctypes.c_double),
        ("scan_mode", ctypes.c_int32),
        ("laser_x", ctypes.c_double), ("laser_y", ctypes.c_double),
        ("standoff_m", ctypes.c_double), ("standoff_mode", ctypes.c_int32),
        ("bin_width_s", ctypes.c_double), ("num_bins", ctypes.c_uint32),
        ("window_start_m", ctypes.c_double),
        ("jitter_fwhm_s", ctypes.c_double),
        ("bin_mode", ctypes.c_int32), ("cos_mode", ctypes.c_int32),
        ("noise_mode", ctypes.c_int32),
        ("peak_photons", ctypes.c_float), ("dark_per_bin", ctypes.c_float),
        ("nr_db", ctypes.c_float),
        ("seed", ctypes.c_uint64), ("stream_tag", ctypes.c_uint32),
        ("boundary_eps", ctypes.c_float),
        ("jitter_padding", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("pairs", ctypes.c_uint64),
        ("peak", ctypes.c_double), ("noise_scale", ctypes.c_double),
        ("noise_dark", ctypes.c_double), ("mean", ctypes.c_double),
        ("variance", ctypes.c_double), ("boundary_pairs", ctypes.c_uint64),
        ("device_error", ctypes.c_uint32),
        ("pairs_full", ctypes.c_uint64),
        ("pairs_tested", ctypes.c_uint64),
    ]

    def to_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "struct_size"}


class Peaks(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("num_sms", ctypes.c_int32)] + [
        (n, ctypes.c_double) for n in (
            "ffma", "ffma2", "sqrt_approx", "rcp_approx", "rsqrt_approx", "lds128_broadcast",
            "red_f32", "red_u32", "red_u64", "rmw_f32", "red_f32_quarter", "red_u32_quarter",
            "dfma", "atom_f32")]

    def to_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "struct_size"}


_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_U32 = ctypes.c_uint32


def load(path: str | None = None):
    """Loads libnlos.so (built by ``paper_2506_03747_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} not found: build it with paper_2506_03747_gb300.build.build() "
                               "(nvcc, sm_103a); there is no CPU fallback")
        lib = ctypes.CDLL(p)
        S = ctypes.c_int
        sig = {
            "nlos_params_default": (None, [ctypes.POINTER(Params)]),
            "nlos_abi_version": (ctypes.c_int, []),
            "nlos_last_error": (ctypes.c_char_p, []),
            "nlos_scene_create": (S, [ctypes.POINTER(Params), _P, _U64, ctypes.c_int, _P,
                                      ctypes.POINTER(ctypes.c_void_p)]),
            "nlos_scene_destroy": (S, [_P]),
            "nlos_scene_create_rows": (S, [ctypes.POINTER(Params), _P, _U64, ctypes.c_int, _U32,
                                           _U32, _P, ctypes.POINTER(ctypes.c_void_p)]),
            "nlos_noise_part": (S, [_P, _P, _P, _P, _U64, _P]),
            "nlos_scene_shape": (S, [_P, ctypes.POINTER(_U64), ctypes.POINTER(_U32),
                                     ctypes.POINTER(_U64)]),
            "nlos_simulate": (S, [_P, _P, _P, _P, ctypes.POINTER(Stats), _P]),
            "nlos_scene_set_points": (S, [_P, _P, _U64, ctypes.c_int, _P]),
            "nlos_scene_set_albedo_depth": (S, [_P, _P, _P, _P]),
            "nlos_scene_set_occluders": (S, [_P, _P, _U32, _P]),
            "nlos_scene_check": (S, [_P, _P]),
            "nlos_forward": (S, [_P, _P, _P]),
            "nlos_detect": (S, [_P, _P, _P, _P, _P]),
            "nlos_simulate_backward": (S, [_P, _P, _P, _P, _P]),
            "nlos_jitter": (S, [_P, _P, _U64, _U32, ctypes.c_double, ctypes.c_double, _P]),
            "nlos_jitter_padded": (S, [_P, _P, _U64, _U32, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int32, _P]),
            "nlos_reduce": (S, [_P, _U64, _U32, _P, _P, _P]),
            "nlos_reduce_static": (S, [_P, _U64, _U32, _P, _P, _P]),
            "nlos_noise": (S, [_P, _U64, ctypes.c_float, ctypes.c_float, _U64, _U32, _U64, _P,
                               _P]),
            "nlos_philox": (S, [_P, _U64, _U32, _U32, _P, _P]),
            "nlos_pair_table": (S, [_P, _U64, _U64, _P, _P, _P]),
            "nlos_server_create": (S, [_U64, ctypes.POINTER(ctypes.c_void_p)]),
            "nlos_serve_submit": (S, [_P, ctypes.POINTER(Params), _P, _U64,
                                      ctypes.POINTER(_U64)]),
            "nlos_serve_poll": (S, [_P, _U64, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Stats)]),
            "nlos_serve_release": (S, [_P, _U64]),
            "nlos_server_destroy": (S, [_P]),
            "nlos_server_stats": (S, [_P, ctypes.POINTER(_U64), ctypes.POINTER(_U32),
                                      ctypes.POINTER(_U32)]),
            "nlos_server_inject": (S, [_P, ctypes.c_int]),
            "nlos_server_device_cycles": (S, [_P, ctypes.POINTER(_U64)]),
            "nlos_lct_create": (S, [_U32, _U32, ctypes.c_double, ctypes.c_double, _P,
                                    ctypes.POINTER(ctypes.c_void_p)]),
            "nlos_lct_forward": (S, [_P, _P, _P, _P, _P]),
            "nlos_lct_destroy": (S, [_P]),
            "nlos_measure_peaks": (S, [ctypes.POINTER(Peaks), _P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        p0 = Params()
        lib.nlos_params_default(ctypes.byref(p0))
        if p0.struct_size != ctypes.sizeof(Params):
            raise RuntimeError("nlos_params layout mismatch between libnlos.so and the binding")
        _lib = lib
        return lib


def _check(status: int):
    if status != OK:
        raise NlosError(status, _lib.nlos_last_error().decode(errors="replace"))


def _ptr(t) -> int | None:
    """Device (or host) address of a torch tensor / numpy array; None passes NULL."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


_ENUM = {
    "scan_mode": {"confocal": CONFOCAL, "nonconfocal": NONCONFOCAL},
    "standoff_mode": {"euclidean": STANDOFF_EUCLIDEAN, "constant": STANDOFF_CONSTANT},
    "bin_mode": {"nearest": BIN_NEAREST, "splat": BIN_SPLAT},
    "cos_mode": {"none": COS_NONE, "object": COS_OBJECT, "object_wall": COS_OBJECT_WALL},
    "noise_mode": {"none": NOISE_NONE, "peak": NOISE_PEAK, "paper_nr": NOISE_PAPER_NR},
    "jitter_padding": {"zero": 0, "replicate": 1},
}


def params(d: dict | None = None, **kw) -> Params:
    """nlos_params from a dict with the keys of ``scenes.default_params()``
    (string enums accepted), on top of the library defaults."""
    lib = load()
    p = Params()
    lib.nlos_params_default(ctypes.byref(p))
    src = dict(d or {})
    src.update(kw)
    for k, v in src.items():
        if k == "laser_xy":
            p.laser_x, p.laser_y = float(v[0]), float(v[1])
            continue
        if k in _ENUM and isinstance(v, str):
            v = _ENUM[k][v]
        if not hasattr(p, k):
            raise KeyError(f"unknown nlos parameter {k!r}")
        setattr(p, k, v)
    return p


def last_error() -> str:
    return load().nlos_last_error().decode(errors="replace")


def abi_version() -> int:
    return load().nlos_abi_version()


# ---------------------------------------------------------------------------
# Scenes and the forward / backward passes.
# ---------------------------------------------------------------------------
class Scene:
    """Owning handle of an ``nlos_scene``."""

    def __init__(self, handle: int, S: int, B: int, P: int, prm: Params):
        self.handle = handle
        self.num_scan, self.num_bins, self.num_points = S, B, P
        self.params = prm
        self.version = 0  # bumped by every scene_set_albedo_depth

    def destroy(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(_lib.nlos_scene_destroy(h))

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def scene_create(prm, points, stream=None) -> Scene:
    """Creates a scene from [P, 8] float32 points: a CUDA tensor (device) or a
    CPU tensor / numpy array (host, copied). Waits for the stream."""
    lib = load()
    if isinstance(prm, dict):
        prm = params(prm)
    on_dev = 0
    if hasattr(points, "is_cuda"):
        on_dev = int(points.is_cuda)
        if points.dtype.__str__() != "torch.float32" or not points.is_contiguous():
            raise ValueError("points must be a contiguous float32 tensor")
        n = points.shape[0] if points.numel() else 0
    else:
        points = np.ascontiguousarray(points, dtype=np.float32)
        n = points.shape[0] if points.size else 0
    h = ctypes.c_void_p()
    _check(lib.nlos_scene_create(ctypes.byref(prm), _ptr(points) if n else None, n, on_dev,
                                 _stream(stream), ctypes.byref(h)))
    S, B, P = _U64(), _U32(), _U64()
    _check(lib.nlos_scene_shape(h, ctypes.byref(S), ctypes.byref(B), ctypes.byref(P)))
    return Scene(h.value, S.value, B.value, P.value, prm)


def scene_create_rows(prm, points, row_begin: int, row_count: int, stream=None) -> Scene:
    """A scene for scan rows [row_begin, row_begin + row_count) of the grid of
    ``prm`` (a part of a cube split by rows); points as in scene_create."""
    lib = load()
    if isinstance(prm, dict):
        prm = params(prm)
    on_dev = 0
    if hasattr(points, "is_cuda"):
        on_dev = int(points.is_cuda)
        if points.dtype.__str__() != "torch.float32" or not points.is_contiguous():
            raise ValueError("points must be a contiguous float32 tensor")
        n = points.shape[0] if points.numel() else 0
    else:
        points = np.ascontiguousarray(points, dtype=np.float32)
        n = points.shape[0] if points.size else 0
    h = ctypes.c_void_p()
    _check(lib.nlos_scene_create_rows(ctypes.byref(prm), _ptr(points) if n else None, n, on_dev,
                                      int(row_begin), int(row_count), _stream(stream),
                                      ctypes.byref(h)))
    S, B, P = _U64(), _U32(), _U64()
    _check(lib.nlos_scene_shape(h, ctypes.byref(S), ctypes.byref(B), ctypes.byref(P)))
    return Scene(h.value, S.value, B.value, P.value, prm)


def noise_part(scene: Scene, tau, counts, cube_stats, cube_bins: int, stream=None):
    """Noise of a part with the whole cube's statistics (float64 CUDA tensor
    [3]: max, sum, sum of squares) over cube_bins bins."""
    _check(_lib.nlos_noise_part(scene.handle, _ptr(tau), _ptr(counts), _ptr(cube_stats),
                                int(cube_bins), _stream(stream)))


def scene_destroy(scene: Scene):
    scene.destroy()


def simulate(scene: Scene, tau, counts=None, energy=None, stats: bool = False, stream=None):
    """Runs the forward hot path into caller-owned CUDA tensors: tau [S, B]
    float32 (required), counts [S, B] int32/uint32 (noise), energy [S]
    float64. Returns a stats dict when ``stats`` (waits for the stream)."""
    st = Stats(struct_size=ctypes.sizeof(Stats)) if stats else None
    _check(_lib.nlos_simulate(scene.handle, _ptr(tau), _ptr(counts), _ptr(energy),
                              ctypes.byref(st) if st is not None else None, _stream(stream)))
    return st.to_dict() if st is not None else None


def scene_set_points(scene: Scene, points, stream=None):
    """Replaces the scene's points (same count): CUDA tensor or host array."""
    on_dev = int(getattr(points, "is_cuda", False))
    if not on_dev and not hasattr(points, "data_ptr"):
        points = np.ascontiguousarray(points, dtype=np.float32)
    n = points.shape[0]
    _check(_lib.nlos_scene_set_points(scene.handle, _ptr(points) if n else None, n, on_dev,
                                      _stream(stream)))


def scene_set_albedo_depth(scene: Scene, albedo=None, depth=None, stream=None):
    """Albedo [P] and normal-offset depth [P] (float32 CUDA tensors, each
    optional) applied to the scene's given records on the device."""
    for t in (albedo, depth):
        if t is not None and (not getattr(t, "is_cuda", False) or t.dtype.__str__() != "torch.float32"
                              or not t.is_contiguous() or t.numel() != scene.num_points):
            raise ValueError("albedo and depth must be contiguous float32 CUDA tensors of "
                             "num_points elements")
    _check(_lib.nlos_scene_set_albedo_depth(scene.handle, _ptr(albedo), _ptr(depth),
                                            _stream(stream)))
    scene.version += 1


def scene_set_occluders(scene: Scene, occluders, stream=None):
    """Occluder records [n, 8] (kind, a0, a1, a2, b0, b1, b2, unused; kind 0 =
    sphere with centre a and radius b0, kind 1 = box with corners a < b), host
    memory; None or an empty array removes them."""
    rec = np.ascontiguousarray(np.zeros((0, 8)) if occluders is None else occluders,
                               dtype=np.float32).reshape(-1, 8)
    n = rec.shape[0]
    _check(_lib.nlos_scene_set_occluders(scene.handle, rec.ctypes.data if n else None, n,
                                         _stream(stream)))


def scene_check(scene: Scene, stream=None):
    _check(_lib.nlos_scene_check(scene.handle, _stream(stream)))


def forward(scene: Scene, tau, stream=None):
    _check(_lib.nlos_forward(scene.handle, _ptr(tau), _stream(stream)))


def detect(scene: Scene, tau, counts=None, energy=None, stream=None):
    _check(_lib.nlos_detect(scene.handle, _ptr(tau), _ptr(counts), _ptr(energy), _stream(stream)))


def simulate_backward(scene: Scene, grad_tau, grad_albedo=None, grad_depth=None, stream=None):
    _check(_lib.nlos_simulate_backward(scene.handle, _ptr(grad_tau), _ptr(grad_albedo),
                                       _ptr(grad_depth), _stream(stream)))


def jitter(inp, out, num_traces: int, num_bins: int, fwhm_s: float, bin_width_s: float,
           stream=None, padding: str = "zero"):
    if padding == "zero":
        _check(load().nlos_jitter(_ptr(inp), _ptr(out), num_traces, num_bins, float(fwhm_s),
                                  float(bin_width_s), _stream(stream)))
    else:
        _check(load().nlos_jitter_padded(_ptr(inp), _ptr(out), num_traces, num_bins,
                                         float(fwhm_s), float(bin_width_s),
                                         _ENUM["jitter_padding"][padding], _stream(stream)))


def reduce(tau, num_traces: int, num_bins: int, energy=None, stats=None, stream=None):
    _check(load().nlos_reduce(_ptr(tau), num_traces, num_bins, _ptr(energy), _ptr(stats),
                              _stream(stream)))


def reduce_static(tau, num_traces: int, num_bins: int, energy=None, stats=None, stream=None):
    """nlos_reduce without device allocation (fixed 1.5 MiB device array,
    at most 65536 transients per call; overlapping calls race)."""
    _check(load().nlos_reduce_static(_ptr(tau), num_traces, num_bins, _ptr(energy), _ptr(stats),
                                     _stream(stream)))


def noise(tau, n: int, scale: float, dark: float, seed: int, stream_tag: int, index_base: int,
          counts, stream=None):
    _check(load().nlos_noise(_ptr(tau), n, ctypes.c_float(scale), ctypes.c_float(dark),
                             int(seed) & (2**64 - 1), int(stream_tag), int(index_base),
                             _ptr(counts), _stream(stream)))


def philox(ctr, n: int, key0: int, key1: int, out, stream=None):
    _check(load().nlos_philox(_ptr(ctr), n, key0, key1, _ptr(out), _stream(stream)))


def pair_table(scene: Scene, s_begin: int, s_count: int, u=None, w=None, stream=None):
    _check(_lib.nlos_pair_table(scene.handle, s_begin, s_count, _ptr(u), _ptr(w),
                                _stream(stream)))


# ---------------------------------------------------------------------------
# Serving.
# ---------------------------------------------------------------------------
class Server:
    def __init__(self, hbm_budget_bytes: int):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.nlos_server_create(int(hbm_budget_bytes), ctypes.byref(h)))
        self.handle = h.value

    def submit(self, prm, points) -> int:
        if isinstance(prm, dict):
            prm = params(prm)
        pts = np.ascontiguousarray(points, dtype=np.float32)
        t = _U64()
        _check(_lib.nlos_serve_submit(self.handle, ctypes.byref(prm),
                                      pts.ctypes.data if pts.size else None,
                                      pts.shape[0] if pts.size else 0, ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, wait_ms: int = 0):
        """(status, tau_ptr, counts_ptr, stats dict); status OK / EBUSY / ..."""
        tau = ctypes.c_void_p()
        cnt = ctypes.c_void_p()
        st = Stats(struct_size=ctypes.sizeof(Stats))
        s = _lib.nlos_serve_poll(self.handle, ticket, int(wait_ms), ctypes.byref(tau),
                                 ctypes.byref(cnt), ctypes.byref(st))
        if s not in (OK, EBUSY):
            _check(s)
        return s, tau.value, cnt.value, st.to_dict()

    def release(self, ticket: int):
        _check(_lib.nlos_serve_release(self.handle, ticket))

    def stats(self) -> dict:
        r, p, a = _U64(), _U32(), _U32()
        _check(_lib.nlos_server_stats(self.handle, ctypes.byref(r), ctypes.byref(p),
                                      ctypes.byref(a)))
        return dict(resident_bytes=r.value, pending=p.value, active=a.value)

    def device_cycles(self) -> dict:
        c = (_U64 * 3)()
        _check(_lib.nlos_server_device_cycles(self.handle, c))
        return dict(wait=c[0], forward=c[1], other=c[2])

    def inject(self, fault: int):
        _check(_lib.nlos_server_inject(self.handle, int(fault)))

    def destroy(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(_lib.nlos_server_destroy(h))

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def server_create(hbm_budget_bytes: int) -> Server:
    return Server(hbm_budget_bytes)


def serve_submit(server: Server, prm, points) -> int:
    return server.submit(prm, points)


def serve_poll(server: Server, ticket: int, wait_ms: int = 0):
    return server.poll(ticket, wait_ms)


def serve_release(server: Server, ticket: int):
    server.release(ticket)


def server_destroy(server: Server):
    server.destroy()


class Lct:
    """Owning handle of an ``nlos_lct`` plan (the paper's FFT forward model)."""

    def __init__(self, n: int, m: int, wall_half_m: float, bin_width_s: float, stream=None):
        h = ctypes.c_void_p()
        _check(load().nlos_lct_create(n, m, float(wall_half_m), float(bin_width_s),
                                      _stream(stream), ctypes.byref(h)))
        self.handle, self.n, self.m = h.value, n, m

    def forward(self, depth, albedo, tau, stream=None):
        """depth [n, n] int32, albedo [n, n] float32 or None, tau [n, n, m] float32
        (CUDA tensors)."""
        _check(load().nlos_lct_forward(self.handle, _ptr(depth), _ptr(albedo), _ptr(tau),
                                       _stream(stream)))

    def destroy(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(load().nlos_lct_destroy(h))

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def measure_peaks(stream=None) -> dict:
    """Element operations per SM clock per SM of the units the forward is bound
    by (``nlos_measure_peaks``); waits for the stream."""
    lib = load()
    pk = Peaks()
    pk.struct_size = ctypes.sizeof(Peaks)
    _check(lib.nlos_measure_peaks(ctypes.byref(pk), _stream(stream)))
    return pk.to_dict()
