"""Python binding of libhai.so (include/hai.h): argument marshalling only.

Every function keeps the C name and forwards to the C ABI; torch tensors
provide device memory and streams.  Each step of the imaging path runs in the
library's CUDA kernels: this module computes nothing, and it raises if the
library is missing rather than falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

HAI_OK = 0
STATUS_NAMES = {0: "HAI_OK", 1: "HAI_ERR_INVALID_ARG", 2: "HAI_ERR_OFF_GRID",
                3: "HAI_ERR_OVERFLOW_RISK", 4: "HAI_ERR_UNSUPPORTED", 5: "HAI_ERR_CUDA",
                6: "HAI_ERR_TIMEOUT", 7: "HAI_ERR_NO_MEMORY"}
HAI_PREC_FP32 = 0
HAI_PREC_FP16 = 1
HAI_PREC_FP16_SPLIT = 2
HAI_PREC_BF16 = 3
HAI_PREC_BF16_SPLIT = 4


class HaiError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class _LayoutDesc(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int), ("grid_n", ctypes.c_int), ("ksize", ctypes.c_int),
                ("n_pol", ctypes.c_int), ("anchors", ctypes.c_void_p), ("taps", ctypes.c_void_p)]


class _PositionDesc(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int), ("pos_m", ctypes.c_void_p), ("lambda_m", ctypes.c_double),
                ("cell_lambda", ctypes.c_double), ("grid_n", ctypes.c_int), ("ksize", ctypes.c_int),
                ("sigma_cells", ctypes.c_double), ("n_pol", ctypes.c_int)]


class _VisLayoutDesc(ctypes.Structure):
    _fields_ = [("n_station", ctypes.c_int), ("pos_m", ctypes.c_void_p), ("lambda_m", ctypes.c_double),
                ("cell_m", ctypes.c_double), ("grid_n", ctypes.c_int), ("n_pol", ctypes.c_int),
                ("n_dir", ctypes.c_int), ("dir", ctypes.c_void_p)]


class _PlanHierDesc(ctypes.Structure):
    _fields_ = [("n_beam", ctypes.c_int), ("weights", ctypes.c_void_p), ("weight_off", ctypes.c_void_p),
                ("requant_shift", ctypes.c_int), ("xfft", ctypes.c_void_p), ("epic", ctypes.c_void_p),
                ("epic_prec", ctypes.c_int)]


class _PlanHierBuffers(ctypes.Structure):
    _fields_ = [("beams", ctypes.c_void_p), ("corr", ctypes.c_void_p), ("vis", ctypes.c_void_p),
                ("xfft_img", ctypes.c_void_p), ("epic_img", ctypes.c_void_p), ("n_saturated", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_int = ctypes.c_int


def _declare(L):
    L.hai_version.restype = _int
    L.hai_last_error.restype = ctypes.c_char_p
    L.hai_status_string.restype = ctypes.c_char_p
    L.hai_status_string.argtypes = [_int]
    L.hai_create.argtypes = [_int, ctypes.POINTER(_vp)]
    L.hai_destroy.argtypes = [_vp]
    L.hai_destroy.restype = None
    L.hai_sync.argtypes = [_vp, _vp]
    L.hai_layout_create.argtypes = [_vp, ctypes.POINTER(_LayoutDesc), ctypes.POINTER(_vp)]
    L.hai_layout_destroy.argtypes = [_vp]
    L.hai_layout_destroy.restype = None
    L.hai_layout_box.argtypes = [_vp, ctypes.POINTER(_int)]
    L.hai_epic_image.argtypes = [_vp, _vp, _vp, _int, _int, _int, _vp, _int, _vp]
    L.hai_epic_image_host.argtypes = [_vp, _vp, _vp, _int, _int, _int, _vp, _int, _int, _vp]
    L.hai_correlate.argtypes = [_vp, _vp, _int, _int, _int, _int, _vp, _int, _vp]
    L.hai_xfft_image.argtypes = [_vp, _vp, _vp, _int, _vp, _int, _vp]
    L.hai_fft_correlate.argtypes = [_vp, _vp, _int, _int, _int, _vp, _vp]
    L.hai_beamform.argtypes = [_vp, _vp, _vp, _int, _int, _int, _int, _int, _int, _int, _vp, _vp, _vp]
    L.hai_epic_image_fp32_static.argtypes = [_int, ctypes.POINTER(_LayoutDesc), _vp, _int, _int, _vp, _int,
                                             _vp]
    L.hai_plan_create.argtypes = [_vp, ctypes.POINTER(_vp), _int, _int, _int, _int, ctypes.POINTER(_vp)]
    L.hai_plan_destroy.argtypes = [_vp]
    L.hai_plan_destroy.restype = None
    L.hai_plan_layout.argtypes = [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.hai_plan_run.argtypes = [_vp, _vp, _vp, _vp]
    L.hai_plan_autotune.argtypes = [_vp, _vp, _vp, _int, _vp]
    L.hai_plan_autotune_cached.argtypes = [_vp, _vp, _vp, _int, ctypes.c_char_p, ctypes.POINTER(_int), _vp]
    L.hai_plan_schedule.argtypes = [_vp, ctypes.POINTER(_int), _vp, _vp, _vp]
    L.hai_plan_set_hierarchy.argtypes = [_vp, ctypes.POINTER(_PlanHierDesc)]
    L.hai_plan_hier_sizes.argtypes = [_vp] + [ctypes.POINTER(ctypes.c_int64)] * 4
    L.hai_plan_run_hier.argtypes = [_vp, _vp, _vp, ctypes.POINTER(_PlanHierBuffers), _vp]
    L.hai_beams_to_corr.argtypes = [_vp, _vp, _int, _int, _int, _int, _int, _vp, _vp]
    L.hai_vis_layout_create.argtypes = [_vp, ctypes.POINTER(_VisLayoutDesc), ctypes.POINTER(_vp)]
    L.hai_vis_layout_destroy.argtypes = [_vp]
    L.hai_vis_layout_destroy.restype = None
    L.hai_vis_layout_offgrid.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong)]
    L.hai_station_epic_layout_create.argtypes = [_vp, ctypes.POINTER(_VisLayoutDesc), _int, ctypes.POINTER(_vp),
                                                 ctypes.POINTER(ctypes.c_longlong)]
    L.hai_xbf_layout_create.argtypes = [_vp, ctypes.POINTER(_VisLayoutDesc), _int, _int, _int, ctypes.POINTER(_vp)]
    L.hai_xbf_layout_destroy.argtypes = [_vp]
    L.hai_xbf_layout_destroy.restype = None
    L.hai_xbf_layout_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    L.hai_xbf_station_image.argtypes = [_vp, _vp, _vp, _int, _vp, _int, _vp]
    L.hai_xfft_station_image.argtypes = [_vp, _vp, _vp, _int, _vp, _vp]
    L.hai_profile_enable.argtypes = [_vp, _int, _int]
    L.hai_check_device_wait.argtypes = [_vp, ctypes.c_longlong, _vp]
    L.hai_layout_create_from_positions.argtypes = [_vp, ctypes.POINTER(_PositionDesc), ctypes.POINTER(_vp)]
    L.hai_layout_anchors.argtypes = [_vp, _vp, _vp]
    L.hai_layout_workspace_size.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t)]
    L.hai_ctx_workspace_size.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t)]
    L.hai_workspace_size.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t)]
    L.hai_autotune.argtypes = [_vp, _vp, _int, _int, _int, ctypes.c_char_p, ctypes.POINTER(_int)]
    L.hai_probe_peak.argtypes = [_vp, _int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double), _vp]
    L.hai_check_device_wait_result.argtypes = [_vp, ctypes.POINTER(_int)]
    L.hai_profile_read.argtypes = [_vp, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]


def load(build: bool = True):
    """Load (building first if needed) the in-tree libhai.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIBPATH
            if not os.path.exists(path):
                raise RuntimeError(f"libhai.so missing at {path}; build it with __graft_entry__.build()")
            L = ctypes.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != HAI_OK:
        raise HaiError(rc, where, load().hai_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _host_ptr(t, dtype, name, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise ValueError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


def _dev_ptr(t, dtype, name, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


# ------------------------------------------------------------------ C API
def hai_version() -> int:
    return load().hai_version()


def hai_status_string(s: int) -> str:
    return load().hai_status_string(s).decode()


def hai_last_error() -> str:
    return load().hai_last_error().decode()


def hai_create(device: int = 0):
    h = _vp()
    _check(load().hai_create(device, ctypes.byref(h)), "hai_create")
    return h


def hai_destroy(ctx):
    load().hai_destroy(ctx)


def hai_sync(ctx, stream=None):
    _check(load().hai_sync(ctx, _stream(stream)), "hai_sync")


def hai_check_device_wait(ctx, limit_cycles: int, stream=None):
    _check(load().hai_check_device_wait(ctx, int(limit_cycles), _stream(stream)), "hai_check_device_wait")


def hai_probe_peak(ctx, kind: int, iters: int, stream=None) -> float:
    """Launch the peak-rate probe; returns the launch's operation count."""
    ops = ctypes.c_double()
    _check(load().hai_probe_peak(ctx, kind, int(iters), ctypes.byref(ops), _stream(stream)), "hai_probe_peak")
    return ops.value


def hai_check_device_wait_result(ctx) -> int:
    g = _int()
    _check(load().hai_check_device_wait_result(ctx, ctypes.byref(g)), "hai_check_device_wait_result")
    return g.value


def hai_profile_enable(ctx, enable: bool = True, max_records: int = 4096):
    _check(load().hai_profile_enable(ctx, int(enable), max_records), "hai_profile_enable")


def hai_profile_read(ctx):
    """(dominant-kernel ms summed, timed launches, all kernel launches)."""
    ms, nd, na = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().hai_profile_read(ctx, ctypes.byref(ms), ctypes.byref(nd), ctypes.byref(na)),
           "hai_profile_read")
    return ms.value, nd.value, na.value


class Layout:
    """Handle of a hai_layout plus the sizes the binding checks buffers with."""

    def __init__(self, handle, n_elem, grid_n, ksize, n_pol):
        self.handle, self.n_elem, self.grid_n, self.ksize, self.n_pol = handle, n_elem, grid_n, ksize, n_pol

    @property
    def n_planes(self):
        return 4 if self.n_pol == 2 else 1


def hai_layout_create(ctx, anchors, taps, grid_n: int, n_pol: int) -> Layout:
    anchors = np.ascontiguousarray(anchors, np.int32)
    taps = np.ascontiguousarray(taps, np.float32)
    ne, k = anchors.shape[0], taps.shape[1]
    if anchors.shape != (ne, 2) or taps.shape != (ne, k, k, 2):
        raise ValueError("anchors must be [n][2] and taps [n][K][K][2]")
    d = _LayoutDesc(ne, grid_n, k, n_pol, anchors.ctypes.data, taps.ctypes.data)
    h = _vp()
    _check(load().hai_layout_create(ctx, ctypes.byref(d), ctypes.byref(h)), "hai_layout_create")
    return Layout(h, ne, grid_n, k, n_pol)


def hai_layout_destroy(layout: Layout):
    load().hai_layout_destroy(layout.handle)


def hai_layout_create_from_positions(ctx, pos_m, lambda_m: float, cell_lambda: float, grid_n: int, ksize: int,
                                     sigma_cells: float, n_pol: int) -> Layout:
    pos = np.ascontiguousarray(pos_m, np.float64)
    if pos.ndim != 2 or pos.shape[1] != 2:
        raise ValueError("pos_m must be [n][2]")
    d = _PositionDesc(len(pos), pos.ctypes.data, lambda_m, cell_lambda, grid_n, ksize, sigma_cells, n_pol)
    h = _vp()
    _check(load().hai_layout_create_from_positions(ctx, ctypes.byref(d), ctypes.byref(h)),
           "hai_layout_create_from_positions")
    return Layout(h, len(pos), grid_n, ksize, n_pol)


def hai_layout_anchors(layout: Layout):
    """(anchors int32 [n][2], taps float32 [n][K][K][2]) the layout uses."""
    a = np.empty((layout.n_elem, 2), np.int32)
    t = np.empty((layout.n_elem, layout.ksize, layout.ksize, 2), np.float32)
    _check(load().hai_layout_anchors(layout.handle, a.ctypes.data, t.ctypes.data), "hai_layout_anchors")
    return a, t


def hai_autotune(ctx, layout: Layout, C: int, T: int, prec: int, cache_path=None) -> int:
    """Tune the layout's tensor-core path for cadences of C x T; returns the
    chosen channels per chunk (0: nothing to tune)."""
    c = _int()
    path = cache_path.encode() if cache_path else None
    _check(load().hai_autotune(ctx, layout.handle, C, T, prec, path, ctypes.byref(c)), "hai_autotune")
    return c.value


def hai_layout_workspace_size(layout: Layout) -> int:
    b = ctypes.c_size_t()
    _check(load().hai_layout_workspace_size(layout.handle, ctypes.byref(b)), "hai_layout_workspace_size")
    return b.value


def hai_ctx_workspace_size(ctx) -> int:
    b = ctypes.c_size_t()
    _check(load().hai_ctx_workspace_size(ctx, ctypes.byref(b)), "hai_ctx_workspace_size")
    return b.value


def hai_workspace_size(plan) -> int:
    b = ctypes.c_size_t()
    _check(load().hai_workspace_size(plan.handle, ctypes.byref(b)), "hai_workspace_size")
    return b.value


def hai_layout_box(layout: Layout):
    box = (_int * 4)()
    _check(load().hai_layout_box(layout.handle, box), "hai_layout_box")
    return tuple(box)


def hai_epic_image(ctx, layout: Layout, volt, C: int, T: int, prec: int, img, accumulate: int = 0,
                   stream=None):
    import torch
    P, ne, n = layout.n_pol, layout.n_elem, layout.grid_n
    vp = _dev_ptr(volt, torch.int8, "volt", C * T * P * ne * 2) if C * T > 0 else 0
    ip = _dev_ptr(img, torch.float32, "img", C * layout.n_planes * n * n) if C > 0 else 0
    _check(load().hai_epic_image(ctx, layout.handle, vp, C, T, prec, ip, accumulate, _stream(stream)),
           "hai_epic_image")


def hai_epic_image_host(ctx, layout: Layout, volt, C: int, T: int, prec: int, img, accumulate: int = 0,
                        chunk: int = 0, stream=None):
    """hai_epic_image on host tensors (pin them for the copies to overlap)."""
    import torch
    P, ne, n = layout.n_pol, layout.n_elem, layout.grid_n
    vp = _host_ptr(volt, torch.int8, "volt", C * T * P * ne * 2) if C * T > 0 else 0
    ip = _host_ptr(img, torch.float32, "img", C * layout.n_planes * n * n) if C > 0 else 0
    _check(load().hai_epic_image_host(ctx, layout.handle, vp, C, T, prec, ip, accumulate, chunk, _stream(stream)),
           "hai_epic_image_host")


def hai_correlate(ctx, volt, C: int, T: int, N: int, P: int, vis, accumulate: int = 0, stream=None):
    import torch
    vp = _dev_ptr(volt, torch.int8, "volt", C * T * P * N * 2) if C * T > 0 else 0
    op = _dev_ptr(vis, torch.int32, "vis", C * (N * (N + 1) // 2) * P * P * 2) if C > 0 else 0
    _check(load().hai_correlate(ctx, vp, C, T, N, P, op, accumulate, _stream(stream)), "hai_correlate")


def hai_xfft_image(ctx, layout: Layout, vis, C: int, img, accumulate: int = 0, stream=None):
    import torch
    ne, P, n = layout.n_elem, layout.n_pol, layout.grid_n
    vp = _dev_ptr(vis, torch.int32, "vis", C * (ne * (ne + 1) // 2) * P * P * 2) if C > 0 else 0
    ip = _dev_ptr(img, torch.float32, "img", C * layout.n_planes * n * n) if C > 0 else 0
    _check(load().hai_xfft_image(ctx, layout.handle, vp, C, ip, accumulate, _stream(stream)), "hai_xfft_image")


def hai_fft_correlate(ctx, img, C: int, N: int, P: int, grid, stream=None):
    """Gridded visibilities from accumulated EPIC images (inverse FFT);
    grid: float32 [C][P][P][N][N][2] (or complex64 of [C][P][P][N][N])."""
    import torch
    q = 4 if P == 2 else 1
    ip = _dev_ptr(img, torch.float32, "img", C * q * N * N) if C > 0 else 0
    if C > 0 and isinstance(grid, torch.Tensor) and grid.dtype == torch.complex64:
        gp = _dev_ptr(torch.view_as_real(grid), torch.float32, "grid", C * P * P * N * N * 2)
    else:
        gp = _dev_ptr(grid, torch.float32, "grid", C * P * P * N * N * 2) if C > 0 else 0
    _check(load().hai_fft_correlate(ctx, ip, C, N, P, gp, _stream(stream)), "hai_fft_correlate")


def hai_epic_image_fp32_static(device: int, anchors, taps, grid_n: int, n_pol: int, volt, C: int, T: int, img,
                               accumulate: int = 0, stream=None):
    """FP32 EPIC image with no device allocation (static scratch in the library)."""
    import torch
    anchors = np.ascontiguousarray(anchors, np.int32)
    taps = np.ascontiguousarray(taps, np.float32)
    ne, k = anchors.shape[0], taps.shape[1]
    d = _LayoutDesc(ne, grid_n, k, n_pol, anchors.ctypes.data, taps.ctypes.data)
    q = 4 if n_pol == 2 else 1
    vp = _dev_ptr(volt, torch.int8, "volt", C * T * n_pol * ne * 2) if C * T > 0 else 0
    ip = _dev_ptr(img, torch.float32, "img", C * q * grid_n * grid_n) if C > 0 else 0
    _check(load().hai_epic_image_fp32_static(device, ctypes.byref(d), vp, C, T, ip, accumulate, _stream(stream)),
           "hai_epic_image_fp32_static")


def hai_beamform(ctx, volt, w, S: int, C: int, T: int, K: int, N: int, P: int, requant_shift: int, beams,
                 n_saturated=None, stream=None):
    import torch
    vp = _dev_ptr(volt, torch.int8, "volt", S * C * T * P * N * 2)
    wp = _dev_ptr(w, torch.int8, "w", S * K * P * N * 2)
    bdt = torch.int32 if requant_shift < 0 else torch.int8
    bp = _dev_ptr(beams, bdt, "beams", S * C * T * K * P * 2)
    sp = _dev_ptr(n_saturated, torch.int64, "n_saturated", 1) if n_saturated is not None else 0
    _check(load().hai_beamform(ctx, vp, wp, S, C, T, K, N, P, requant_shift, bp, sp, _stream(stream)),
           "hai_beamform")


# ------------------------------------------------------------------ batched plan
class Plan:
    """Handle of a hai_plan with its buffer layout (host copies)."""

    def __init__(self, handle, S: int):
        self.handle = handle
        self.S = S
        self.volt_off = np.zeros(S, np.int64)
        self.img_off = np.zeros(S, np.int64)
        vb, nf = ctypes.c_int64(), ctypes.c_int64()
        _check(load().hai_plan_layout(handle, self.volt_off.ctypes.data, self.img_off.ctypes.data,
                                      ctypes.byref(vb), ctypes.byref(nf)), "hai_plan_layout")
        self.volt_bytes = vb.value
        self.img_floats = nf.value

    @property
    def _as_parameter_(self):
        return self.handle


def hai_plan_create(ctx, layouts, C: int, T: int, prec: int = HAI_PREC_FP16) -> Plan:
    arr = (_vp * len(layouts))(*[ly.handle for ly in layouts])
    h = _vp()
    _check(load().hai_plan_create(ctx, arr, len(layouts), C, T, prec, ctypes.byref(h)), "hai_plan_create")
    return Plan(h, len(layouts))


def hai_plan_destroy(plan: Plan):
    load().hai_plan_destroy(plan.handle)


def hai_plan_layout(plan: Plan):
    """(volt_off[S] bytes, img_off[S] floats, volt_bytes, img_floats)."""
    return plan.volt_off, plan.img_off, plan.volt_bytes, plan.img_floats


def hai_plan_run(plan: Plan, volt, img, stream=None):
    import torch
    vp = _dev_ptr(volt, torch.int8, "volt", plan.volt_bytes)
    ip = _dev_ptr(img, torch.float32, "img", plan.img_floats)
    _check(load().hai_plan_run(plan.handle, vp, ip, _stream(stream)), "hai_plan_run")


def hai_plan_autotune(plan: Plan, volt, img, rounds: int = 2, stream=None):
    import torch
    vp = _dev_ptr(volt, torch.int8, "volt", plan.volt_bytes)
    ip = _dev_ptr(img, torch.float32, "img", plan.img_floats)
    _check(load().hai_plan_autotune(plan.handle, vp, ip, rounds, _stream(stream)), "hai_plan_autotune")


def hai_plan_autotune_cached(plan: Plan, volt, img, cache_path: str, rounds: int = 2, stream=None) -> bool:
    """Autotune with a text cache; True when the shares came from the cache."""
    import torch
    vp = _dev_ptr(volt, torch.int8, "volt", plan.volt_bytes)
    ip = _dev_ptr(img, torch.float32, "img", plan.img_floats)
    hit = _int()
    _check(load().hai_plan_autotune_cached(plan.handle, vp, ip, rounds, cache_path.encode(), ctypes.byref(hit),
                                           _stream(stream)), "hai_plan_autotune_cached")
    return bool(hit.value)


def hai_plan_schedule(plan: Plan):
    """[(grid side, CTAs, measured ms alone)] per grid group."""
    n = _int()
    g = (_int * 3)()
    c = (_int * 3)()
    m = (ctypes.c_double * 3)()
    _check(load().hai_plan_schedule(plan.handle, ctypes.byref(n), g, c, m), "hai_plan_schedule")
    return [(g[k], c[k], m[k]) for k in range(n.value)]


def hai_plan_set_hierarchy(plan: Plan, n_beam: int, weights, weight_off, requant_shift: int, xfft=None,
                           epic=None, epic_prec: int = HAI_PREC_FP16):
    """Attach the second level: station beams (weights: device int8 holding
    station s's [K][2][N_e,s][2] at byte weight_off[s], re-packed by the
    plan) imaged by the inter-station XFFT (a VisLayout) and/or EPIC (K
    Layouts).  The plan keeps references to the layouts."""
    import torch
    if not (isinstance(weights, torch.Tensor) and weights.is_cuda and weights.dtype == torch.int8):
        raise ValueError("weights must be a CUDA int8 tensor")
    off = np.ascontiguousarray(weight_off, np.int64)
    if off.shape != (plan.S,):
        raise ValueError("weight_off must hold one offset per station")
    arr = None
    if epic is not None:
        if len(epic) != n_beam:
            raise ValueError("one EPIC layout per beam")
        arr = (_vp * n_beam)(*[ly.handle for ly in epic])
    desc = _PlanHierDesc(n_beam, weights.data_ptr(), off.ctypes.data, requant_shift,
                         None if xfft is None else xfft.handle, None if arr is None else ctypes.addressof(arr),
                         epic_prec)
    _check(load().hai_plan_set_hierarchy(plan.handle, ctypes.byref(desc)), "hai_plan_set_hierarchy")
    plan.hier = (xfft, list(epic) if epic is not None else None)   # keep the layouts alive


def hai_plan_hier_sizes(plan: Plan):
    """(beam bytes, visibility int32s, XFFT image floats, EPIC image floats)."""
    v = [ctypes.c_int64() for _ in range(4)]
    _check(load().hai_plan_hier_sizes(plan.handle, *[ctypes.byref(x) for x in v]), "hai_plan_hier_sizes")
    return tuple(x.value for x in v)


def hai_plan_run_hier(plan: Plan, volt, img, beams, corr, vis=None, xfft_img=None, epic_img=None,
                      n_saturated=None, stream=None):
    import torch
    nb, nv, nx, ne = hai_plan_hier_sizes(plan)
    bufs = _PlanHierBuffers(
        _dev_ptr(beams, torch.int8, "beams", nb), _dev_ptr(corr, torch.int8, "corr", nb),
        _dev_ptr(vis, torch.int32, "vis", nv) if vis is not None else None,
        _dev_ptr(xfft_img, torch.float32, "xfft_img", nx) if xfft_img is not None else None,
        _dev_ptr(epic_img, torch.float32, "epic_img", ne) if epic_img is not None else None,
        _dev_ptr(n_saturated, torch.int64, "n_saturated", 1) if n_saturated is not None else None)
    vp = _dev_ptr(volt, torch.int8, "volt", plan.volt_bytes)
    ip = _dev_ptr(img, torch.float32, "img", plan.img_floats)
    _check(load().hai_plan_run_hier(plan.handle, vp, ip, ctypes.byref(bufs), _stream(stream)), "hai_plan_run_hier")


# ------------------------------------------------------------------ inter-station stage
def hai_beams_to_corr(ctx, beams, S: int, C: int, T: int, K: int, P: int, out, stream=None):
    import torch
    bp = _dev_ptr(beams, torch.int8, "beams", S * C * T * K * P * 2)
    op = _dev_ptr(out, torch.int8, "out", S * C * T * K * P * 2)
    _check(load().hai_beams_to_corr(ctx, bp, S, C, T, K, P, op, _stream(stream)), "hai_beams_to_corr")


class VisLayout:
    """Handle of a hai_vis_layout with its sizes."""

    def __init__(self, handle, S, N, K):
        self.handle, self.S, self.N, self.K = handle, S, N, K

    @property
    def n_baselines(self):
        return self.S * (self.S + 1) // 2


def hai_vis_layout_create(ctx, pos_m, lambda_m: float, cell_m: float, grid_n: int, dirs=None,
                          n_pol: int = 2) -> VisLayout:
    pos = np.ascontiguousarray(pos_m, np.float64)
    S = pos.shape[0]
    if pos.shape != (S, 2):
        raise ValueError("pos_m must be [S][2]")
    d = None if dirs is None else np.ascontiguousarray(dirs, np.float64)
    K = 1 if d is None else d.shape[0]
    desc = _VisLayoutDesc(S, pos.ctypes.data, lambda_m, cell_m, grid_n, n_pol, K,
                          None if d is None else d.ctypes.data)
    h = _vp()
    _check(load().hai_vis_layout_create(ctx, ctypes.byref(desc), ctypes.byref(h)), "hai_vis_layout_create")
    return VisLayout(h, S, grid_n, K)


def hai_station_epic_layout_create(ctx, pos_m, lambda_m: float, cell_m: float, grid_n: int, dirs=None, k: int = 0,
                                   n_pol: int = 2):
    """Layout of the inter-station EPIC for beam direction k (stations as the
    elements, FP64 steering weights).  Returns (Layout, stations dropped)."""
    pos = np.ascontiguousarray(pos_m, np.float64)
    S = pos.shape[0]
    if pos.shape != (S, 2):
        raise ValueError("pos_m must be [S][2]")
    d = None if dirs is None else np.ascontiguousarray(dirs, np.float64)
    K = 1 if d is None else d.shape[0]
    desc = _VisLayoutDesc(S, pos.ctypes.data, lambda_m, cell_m, grid_n, n_pol, K,
                          None if d is None else d.ctypes.data)
    h = _vp()
    dropped = ctypes.c_longlong()
    _check(load().hai_station_epic_layout_create(ctx, ctypes.byref(desc), k, ctypes.byref(h), ctypes.byref(dropped)),
           "hai_station_epic_layout_create")
    return Layout(h, S, grid_n, 1, n_pol), dropped.value


HAI_XBF_ALL_PAIRS = 0
HAI_XBF_OFFGRID_PAIRS = 1


class XbfLayout:
    """Handle of a hai_xbf_layout with its sizes."""

    def __init__(self, handle, S, N, K, max_channels):
        self.handle, self.S, self.N, self.K, self.max_channels = handle, S, N, K, max_channels


def hai_xbf_layout_create(ctx, pos_m, lambda_m: float, cell_m: float, grid_n: int, dirs=None,
                          pair_set: int = HAI_XBF_ALL_PAIRS, max_channels: int = 1,
                          prec: int = HAI_PREC_FP16) -> XbfLayout:
    pos = np.ascontiguousarray(pos_m, np.float64)
    S = pos.shape[0]
    if pos.shape != (S, 2):
        raise ValueError("pos_m must be [S][2]")
    d = None if dirs is None else np.ascontiguousarray(dirs, np.float64)
    K = 1 if d is None else d.shape[0]
    desc = _VisLayoutDesc(S, pos.ctypes.data, lambda_m, cell_m, grid_n, 2, K, None if d is None else d.ctypes.data)
    h = _vp()
    _check(load().hai_xbf_layout_create(ctx, ctypes.byref(desc), pair_set, max_channels, prec, ctypes.byref(h)),
           "hai_xbf_layout_create")
    return XbfLayout(h, S, grid_n, K, max_channels)


def hai_xbf_layout_destroy(layout: XbfLayout):
    load().hai_xbf_layout_destroy(layout.handle)


def hai_xbf_layout_info(layout: XbfLayout):
    """(pairs in the set, device bytes of the phase and coefficient buffers)."""
    n, b = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().hai_xbf_layout_info(layout.handle, ctypes.byref(n), ctypes.byref(b)), "hai_xbf_layout_info")
    return n.value, b.value


def hai_xbf_station_image(ctx, layout: XbfLayout, vis, C: int, img, accumulate: int = 0, stream=None):
    import torch
    S, N, K = layout.S, layout.N, layout.K
    vp = _dev_ptr(vis, torch.int32, "vis", K * C * (S * (S + 1) // 2) * 8) if C > 0 else 0
    ip = _dev_ptr(img, torch.float32, "img", K * C * 4 * N * N) if C > 0 else 0
    _check(load().hai_xbf_station_image(ctx, layout.handle, vp, C, ip, accumulate, _stream(stream)),
           "hai_xbf_station_image")


def hai_vis_layout_destroy(layout: VisLayout):
    load().hai_vis_layout_destroy(layout.handle)


def hai_vis_layout_offgrid(layout: VisLayout) -> int:
    n = ctypes.c_longlong()
    _check(load().hai_vis_layout_offgrid(layout.handle, ctypes.byref(n)), "hai_vis_layout_offgrid")
    return n.value


def hai_xfft_station_image(ctx, layout: VisLayout, vis, C: int, img, stream=None):
    import torch
    vp = _dev_ptr(vis, torch.int32, "vis", layout.K * C * layout.n_baselines * 8)
    ip = _dev_ptr(img, torch.float32, "img", layout.K * C * 4 * layout.N * layout.N)
    _check(load().hai_xfft_station_image(ctx, layout.handle, vp, C, ip, _stream(stream)), "hai_xfft_station_image")
