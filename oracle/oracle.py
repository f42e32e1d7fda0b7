"""NumPy front of the FP64 CPU oracle in hai_oracle.c.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg.  The product package never imports it.

Each function states the equation of the paper it computes; the arithmetic
itself lives in hai_oracle.c as plain FP64 / int64 loops.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hai_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile hai_oracle.c with gcc (IEEE FP64, OpenMP) into oracle/_lib."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            c_int, c_long = ctypes.c_int, ctypes.c_long
            L.orc_num_threads.restype = c_int
            L.orc_set_threads.argtypes = [c_int]
            L.orc_set_threads.restype = c_int
            L.orc_fft1d.argtypes = [c_int, _f64p, _f64p, c_long]
            L.orc_fft2d.argtypes = [c_int, _f64p, _f64p]
            L.orc_grid.argtypes = [c_int, c_int, c_int, _i32p, _f32p, _i8p, _f64p, _f64p]
            L.orc_grid.restype = None
            L.orc_efield_image.argtypes = [c_int, c_int, c_int, _i32p, _f32p, _i8p, _f64p, _f64p]
            L.orc_epic_image.argtypes = [c_int, c_int, c_int, _i32p, _f32p, _i8p, c_int, c_int,
                                         c_int, _f64p]
            L.orc_correlate.argtypes = [_i8p, c_int, c_int, c_int, c_int, _i64p]
            L.orc_beamform.argtypes = [_i8p, _i8p, c_int, c_int, c_int, c_int, c_int, c_int, _i64p]
            L.orc_requant_array.argtypes = [_i64p, c_long, c_int, _i8p,
                                            ctypes.POINTER(ctypes.c_int64)]
            L.orc_requant_array.restype = None
            L.orc_vis_kernel.argtypes = [c_int, _i32p, _f32p, c_int, c_int, _f64p]
            L.orc_vis_kernel.restype = None
            L.orc_xfft_image.argtypes = [c_int, c_int, c_int, _i32p, _f32p, _i64p, c_int, c_int,
                                         _f64p]
            L.orc_xfft_grid.argtypes = [c_int, c_int, c_int, _i32p, _f32p, _i64p, c_int, c_int,
                                        _f64p]
            L.orc_fft_correlate.argtypes = [c_int, c_int, c_int, _f64p, _f64p]
            L.orc_station_xfft.argtypes = [c_int, c_int, _f64p, ctypes.c_double, ctypes.c_double, c_int,
                                           _f64p, _i64p, c_int, c_int, _f64p,
                                           ctypes.POINTER(ctypes.c_int64)]
            L.orc_station_xbf.argtypes = [c_int, c_int, _f64p, ctypes.c_double, ctypes.c_double, c_int,
                                          _f64p, _i64p, c_int, c_int, c_int, _f64p]
            L.orc_dft2d_brute.argtypes = [c_int, _f64p, _f64p, _f64p, _f64p]
            L.orc_dft2d_brute.restype = None
            _lib = L
    return _lib


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's later calls (n <= 0: unchanged);
    returns the count in force."""
    return lib().orc_set_threads(n)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def _layout(anchors, taps):
    anchors = np.ascontiguousarray(anchors, np.int32)
    taps = np.ascontiguousarray(taps, np.float32)
    return anchors, taps, len(anchors), taps.shape[1]


def fft1d(x: np.ndarray) -> np.ndarray:
    """X[k] = sum_n x[n] exp(+2 pi i n k / N) by the radix-2 FFT."""
    re = np.ascontiguousarray(np.real(x), np.float64)
    im = np.ascontiguousarray(np.imag(x), np.float64)
    _check(lib().orc_fft1d(len(re), re, im, 1), "fft1d")
    return re + 1j * im


def fft2d(g: np.ndarray) -> np.ndarray:
    """F[ly][lx] = sum_j g[jy][jx] exp(+2 pi i (lx jx + ly jy)/N), radix-2."""
    n = g.shape[0]
    re = np.ascontiguousarray(np.real(g), np.float64)
    im = np.ascontiguousarray(np.imag(g), np.float64)
    _check(lib().orc_fft2d(n, re, im), "fft2d")
    return re + 1j * im


def dft2d_brute(g: np.ndarray) -> np.ndarray:
    """The same transform as fft2d by the O(N^4) direct sum."""
    n = g.shape[0]
    re = np.ascontiguousarray(np.real(g), np.float64)
    im = np.ascontiguousarray(np.imag(g), np.float64)
    ore, oim = np.empty_like(re), np.empty_like(im)
    lib().orc_dft2d_brute(n, re, im, ore, oim)
    return ore + 1j * oim


def grid(n: int, anchors, taps, e: np.ndarray) -> np.ndarray:
    """Gridded field of one (channel, sample, pol): the bracket of
    Eq. (intra-station EPIC), sum_a conj(W~_a(r_j - r_a)) E_a, [n][n] complex."""
    anchors, taps, ne, k = _layout(anchors, taps)
    e = np.ascontiguousarray(e, np.int8).reshape(ne, 2)
    gr, gi = np.empty((n, n)), np.empty((n, n))
    lib().orc_grid(n, ne, k, anchors, taps, e, gr, gi)
    return gr + 1j * gi


def efield_image(n: int, anchors, taps, e: np.ndarray) -> np.ndarray:
    """Synthesised field of Eq. (intra-station EPIC) at every pixel, with the
    phase centre at pixel (N/2, N/2)."""
    anchors, taps, ne, k = _layout(anchors, taps)
    e = np.ascontiguousarray(e, np.int8).reshape(ne, 2)
    fr, fi = np.empty((n, n)), np.empty((n, n))
    _check(lib().orc_efield_image(n, ne, k, anchors, taps, e, fr, fi), "efield_image")
    return fr + 1j * fi


def epic_image(n: int, anchors, taps, volt: np.ndarray) -> np.ndarray:
    """EPIC image (Eq. intra-station EPIC, then the squaring and temporal sum
    of Eq. intra-station squaring).  volt int8 [C][T][P][N_e][2]; returns
    float64 [C][Q][n][n] with Q = 1 (XX) for P = 1 and Q = 4 (XX, YY, Re XY,
    Im XY) for P = 2."""
    anchors, taps, ne, k = _layout(anchors, taps)
    volt = np.ascontiguousarray(volt, np.int8)
    C, T, P, ne2, _ = volt.shape
    assert ne2 == ne
    Q = 4 if P == 2 else 1
    img = np.empty((C, Q, n, n))
    _check(lib().orc_epic_image(n, ne, k, anchors, taps, volt, C, T, P, img), "epic_image")
    return img


def correlate(volt: np.ndarray) -> np.ndarray:
    """Visibilities of Eq. (intra-station visibilities) summed over T:
    int64 [C][N(N+1)/2][P][P][2], baseline a(a+1)/2 + b for a >= b."""
    volt = np.ascontiguousarray(volt, np.int8)
    C, T, P, ne, _ = volt.shape
    vis = np.empty((C, ne * (ne + 1) // 2, P, P, 2), np.int64)
    _check(lib().orc_correlate(volt, C, T, ne, P, vis), "correlate")
    return vis


def beamform(volt: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Voltage beams of Eq. (intra-station BF), diagonal polarisation:
    volt [S][C][T][P][N_e][2], w [S][K][P][N_e][2] -> int64 [S][C][T][K][P][2]."""
    volt = np.ascontiguousarray(volt, np.int8)
    w = np.ascontiguousarray(w, np.int8)
    S, C, T, P, ne, _ = volt.shape
    K = w.shape[1]
    out = np.empty((S, C, T, K, P, 2), np.int64)
    _check(lib().orc_beamform(volt, w, S, C, T, K, ne, P, out), "beamform")
    return out


def requant(x: np.ndarray, shift: int):
    """int8 beams: x / 2^shift rounded half away from zero, clamped to
    [-127, 127]; returns (values, number of clamped components)."""
    x = np.ascontiguousarray(x, np.int64)
    out = np.empty(x.shape, np.int8)
    sat = ctypes.c_int64(0)
    lib().orc_requant_array(x.reshape(-1), x.size, shift, out.reshape(-1), ctypes.byref(sat))
    return out, int(sat.value)


def vis_kernel(anchors, taps, a: int, b: int):
    """Autocorrelation gridding kernel K_ab[d] = sum_j g_a[j+d] conj(g_b[j])
    of Eq. (intra-station XFFT).  Returns (complex [(2K-1)][(2K-1)] indexed
    [ey+K-1][ex+K-1], base lag (dx0, dy0)); the lag is base + (ex, ey)."""
    anchors, taps, ne, k = _layout(anchors, taps)
    w2 = 2 * k - 1
    out = np.empty((w2, w2, 2))
    lib().orc_vis_kernel(k, anchors, taps, a, b, out)
    base = (int(anchors[a, 0] - anchors[b, 0]), int(anchors[a, 1] - anchors[b, 1]))
    return out[..., 0] + 1j * out[..., 1], base


def xfft_image(n: int, anchors, taps, vis: np.ndarray) -> np.ndarray:
    """Dirty image of Eq. (intra-station XFFT) from int64 visibilities
    [C][N_e(N_e+1)/2][P][P][2]: complex [C][P][P][n][n] for every
    polarisation pair."""
    anchors, taps, ne, k = _layout(anchors, taps)
    vis = np.ascontiguousarray(vis, np.int64)
    C, nbl, P, _, _ = vis.shape
    assert nbl == ne * (ne + 1) // 2
    img = np.empty((C, P, P, n, n, 2))
    _check(lib().orc_xfft_image(n, ne, k, anchors, taps, vis, C, P, img), "xfft_image")
    return img[..., 0] + 1j * img[..., 1]


def xfft_grid(n: int, anchors, taps, vis: np.ndarray) -> np.ndarray:
    """Gridded visibilities of Eq. (intra-station XFFT), the bracket before
    the transform: sum over all ordered pairs of V^{alpha beta}_{ab} K_ab[d]
    on the circular n grid (lag d at cell (d_x mod n, d_y mod n)).  Returns
    complex [C][P][P][n][n]."""
    anchors, taps, ne, k = _layout(anchors, taps)
    vis = np.ascontiguousarray(vis, np.int64)
    C, nbl, P, _, _ = vis.shape
    assert nbl == ne * (ne + 1) // 2
    g = np.empty((C, P, P, n, n, 2))
    _check(lib().orc_xfft_grid(n, ne, k, anchors, taps, vis, C, P, g), "xfft_grid")
    return g[..., 0] + 1j * g[..., 1]


def fft_correlate(planes: np.ndarray) -> np.ndarray:
    """FFT correlator (Section 4.1.2, Section 5.2.2): inverse DFT, normalised
    by 1/n^2 and multiplied by (-1)^(dx+dy), of accumulated EPIC image planes
    [C][Q][n][n] (Q = 1: XX; Q = 4: XX, YY, Re XY, Im XY).  Returns the
    gridded visibilities, complex [C][P][P][n][n] with the zero lag at cell
    (0, 0)."""
    planes = np.ascontiguousarray(planes, np.float64)
    C, Q, n, _ = planes.shape
    P = 2 if Q == 4 else 1
    g = np.empty((C, P, P, n, n, 2))
    _check(lib().orc_fft_correlate(n, C, P, planes, g), "fft_correlate")
    return g[..., 0] + 1j * g[..., 1]


def station_xfft(n: int, pos_m, lam_m: float, cell_m: float, dirs, vis: np.ndarray):
    """Dirty images of Eq. (inter-station XFFT): station visibilities int64
    [K][C][S(S+1)/2][P][P][2] phased towards dirs [K][2] (direction cosines)
    in FP64, gridded bilinearly at (r_m - r_n) / cell on an n x n grid.
    Returns (complex [K][C][P][P][n][n], pairs dropped off the grid)."""
    pos = np.ascontiguousarray(pos_m, np.float64)
    dirs = np.ascontiguousarray(dirs, np.float64)
    vis = np.ascontiguousarray(vis, np.int64)
    K, C, nbl, P, _, _ = vis.shape
    S = pos.shape[0]
    assert nbl == S * (S + 1) // 2 and dirs.shape == (K, 2)
    img = np.empty((K, C, P, P, n, n, 2))
    dropped = ctypes.c_int64()
    _check(lib().orc_station_xfft(n, S, pos, lam_m, cell_m, K, dirs, vis, C, P, img, ctypes.byref(dropped)),
           "station_xfft")
    return img[..., 0] + 1j * img[..., 1], dropped.value


def station_epic_layout(n: int, pos_m, lam_m: float, cell_m: float, direction):
    """Gridding kernel of Eq. (inter-station EPIC) with N_ks = 1 cell: station
    m sits at its nearest cell j_m = floor(r_m / cell + n/2 + 1/2) with the
    weight conj(W~_m) = exp(+2 pi i s_k . r_m / lambda) (FP64), which brings
    the beam direction s_k to the phase-centre pixel.  The padding factor
    gamma_A = 2 per dimension (Section 5.2.2) leaves the array the central
    half of the grid: a station whose cell lies outside [n/4, 3n/4)^2 is
    dropped (zero weight, parked on the centre cell).
    Returns (anchors int32 [S][2], taps float32 [S][1][1][2] holding W~_m as
    the EPIC gridding expects, stations dropped)."""
    pos = np.asarray(pos_m, np.float64)
    d = np.asarray(direction, np.float64)
    cells = np.floor(pos / cell_m + n / 2.0 + 0.5).astype(np.int64)
    on = np.all((cells >= n // 4) & (cells < n - n // 4), axis=1)
    anchors = np.where(on[:, None], cells, n // 2).astype(np.int32)
    turns = (pos @ d) / lam_m
    taps = np.zeros((len(pos), 1, 1, 2), np.float32)
    taps[:, 0, 0, 0] = np.where(on, np.cos(2 * np.pi * turns), 0.0)
    taps[:, 0, 0, 1] = np.where(on, -np.sin(2 * np.pi * turns), 0.0)
    return anchors, taps, int(np.count_nonzero(~on))


def station_epic(n: int, pos_m, lam_m: float, cell_m: float, dirs, beams: np.ndarray):
    """Images of Eq. (inter-station EPIC) then the squaring and temporal sum
    of Eq. (inter-station squaring): for every beam direction s_k the station
    beams E_m(s_k) int8 [K][C][T][P][S][2] gridded with station_epic_layout,
    transformed and squared as intra-station EPIC.  Returns (float64
    [K][C][Q][n][n], stations dropped)."""
    beams = np.asarray(beams)
    K = beams.shape[0]
    out, dropped = [], 0
    for k in range(K):
        anchors, taps, dropped = station_epic_layout(n, pos_m, lam_m, cell_m, dirs[k])
        out.append(epic_image(n, anchors, taps, np.ascontiguousarray(beams[k])))
    return np.stack(out), dropped


def station_xbf(n: int, pos_m, lam_m: float, cell_m: float, dirs, vis: np.ndarray, offgrid_only=False):
    """Images of Eq. (inter-station XBF): the direct FP64 DFT of station
    visibilities int64 [K][C][S(S+1)/2][P][P][2] over every ordered station
    pair (autos once) at the pixels sigma = s_k + (l - n/2) lambda / (n cell),
    or (offgrid_only) over the pairs the inter-station XFFT grid drops.
    Returns complex [K][C][P][P][n][n]."""
    pos = np.ascontiguousarray(pos_m, np.float64)
    dirs = np.ascontiguousarray(dirs, np.float64)
    vis = np.ascontiguousarray(vis, np.int64)
    K, C, nbl, P, _, _ = vis.shape
    S = pos.shape[0]
    assert nbl == S * (S + 1) // 2 and dirs.shape == (K, 2)
    img = np.empty((K, C, P, P, n, n, 2))
    _check(lib().orc_station_xbf(n, S, pos, lam_m, cell_m, K, dirs, vis, C, P, 1 if offgrid_only else 0, img),
           "station_xbf")
    return img[..., 0] + 1j * img[..., 1]


def xfft_as_epic_planes(ximg: np.ndarray) -> np.ndarray:
    """Pick the stored planes (XX, YY, Re XY, Im XY) out of a full complex
    polarisation-pair image [C][P][P][n][n]."""
    C, P = ximg.shape[:2]
    if P == 1:
        return ximg[:, 0, 0].real[:, None]
    return np.stack([ximg[:, 0, 0].real, ximg[:, 1, 1].real,
                     ximg[:, 0, 1].real, ximg[:, 0, 1].imag], axis=1)
