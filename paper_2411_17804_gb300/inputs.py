"""Seeded synthetic inputs shaped like the paper's aperture arrays.

This module holds no step of the imaging method.  It draws what the method
takes as given:

* element layouts inside a station (Section 2, Table 1: stations of N_eps
  elements of size D_e inside a station of size D_s), and station layouts;
* the gridding kernel of every element -- the paper leaves the illumination
  kernel W~ of Eq. (intra-station EPIC) to the user, so it is an input: an
  anchor cell plus K x K complex taps per element;
* sky sources and the calibrated, quantised complex int8 voltages E^p_a(t)
  of Eq. (intra-station BF) / Eq. (intra-station EPIC);
* the int8 directional weights of the voltage beamformer (Eq. intra-station BF).

Both the CUDA library and the CPU oracle receive these arrays; nothing here
calls either of them.  Small cases are drawn with NumPy, large voltage sets
with a seeded torch generator on any device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED0 = 20241127


# ----------------------------------------------------------------------------
# workload descriptions
# ----------------------------------------------------------------------------
@dataclass
class StationConfig:
    """One imaging workload (sizes only; arrays come from the draw functions)."""
    name: str
    n_elem: int            # N_eps
    diameter_m: float      # station diameter D_s
    min_spacing_m: float
    lam_m: float           # wavelength lambda
    n_chan: int            # C
    n_pol: int             # P (n_p input polarisations)
    n_time: int            # T samples per cadence (t_acc / delta t)
    grid_n: int            # padded grid side N
    cell_lambda: float     # grid cell in wavelengths
    ksize: int             # gridding kernel side K
    n_src: int = 20
    fluxes: tuple = ()     # explicit source fluxes (else power law)
    lattice: bool = False  # regular lattice instead of random disk
    seed: int = SEED0

    @property
    def units_per_cadence(self) -> int:
        """Imaged pixel x channel x pol x sample count of one cadence."""
        return self.grid_n * self.grid_n * self.n_chan * self.n_pol * self.n_time


# Five workloads of the hot path; the sizes follow the paper's arrays
# (SKA-low station of 256 elements, Table 1) and a dense all-sky lattice.
SINGLE_STATION_64 = StationConfig(
    name="station64_grid32", n_elem=64, diameter_m=8.0, min_spacing_m=0.75,
    lam_m=2.0, n_chan=1, n_pol=1, n_time=1024, grid_n=32, cell_lambda=0.5,
    ksize=3, n_src=3, fluxes=(1.0, 0.5, 0.25), seed=SEED0 + 1)

SKA_LOW_STATION_256 = StationConfig(
    name="ska_low_station256_grid64", n_elem=256, diameter_m=38.0,
    min_spacing_m=1.5, lam_m=3.0, n_chan=64, n_pol=2, n_time=2048, grid_n=64,
    cell_lambda=0.5, ksize=3, n_src=20, seed=SEED0 + 2)

DENSE_ALLSKY_16384 = StationConfig(
    name="dense_allsky16384_grid512", n_elem=128 * 128, diameter_m=64.0,
    min_spacing_m=1.0, lam_m=2.0, n_chan=16, n_pol=2, n_time=100, grid_n=512,
    cell_lambda=0.5, ksize=1, n_src=20, lattice=True, seed=SEED0 + 5)


@dataclass
class HierarchyConfig:
    """Two-level array: stations of elements (hierarchical hybrid workload)."""
    name: str = "hier256x256_beams16_grid256"
    n_station: int = 256
    station: StationConfig = field(default_factory=lambda: SKA_LOW_STATION_256)
    core_diameter_m: float = 1000.0
    tail_radius_m: float = 65000.0
    n_tail: int = 32
    n_beam: int = 16
    n_chan: int = 32
    n_pol: int = 2
    n_time: int = 1000
    grid_n: int = 256         # station-level (inter-station) grid
    cell_m: float = 19.0      # its uv cell: half a station diameter (padding 2)
    requant_shift: int = 11   # beams / 2^11: noise-dominated beam rms ~ 18 counts
    seed: int = SEED0 + 3


@dataclass
class UnevenConfig:
    """Batched uneven hierarchy: stations of log-uniform element counts."""
    name: str = "uneven512_grid32to256"
    n_station: int = 512
    n_min: int = 16
    n_max: int = 1024
    n_chan: int = 128
    n_pol: int = 2
    n_time: int = 64
    lam_m: float = 3.0
    cell_lambda: float = 0.5
    ksize: int = 3
    ref_diameter_m: float = 38.0   # diameter of a 256-element station
    # second level: the stations in a compact core, K beams each, imaged
    # between stations (XFFT on an N_A grid, EPIC on an N_E grid)
    core_diameter_m: float = 3000.0
    n_beam: int = 4
    requant_shift: int = 12
    xfft_grid_n: int = 256
    xfft_cell_m: float = 38.0
    epic_grid_n: int = 128
    epic_cell_m: float = 76.0
    seed: int = SEED0 + 4


# ----------------------------------------------------------------------------
# layouts
# ----------------------------------------------------------------------------
def disk_layout(n: int, diameter_m: float, min_spacing_m: float,
                rng: np.random.Generator, max_tries: int = 2_000_000) -> np.ndarray:
    """n positions (metres, station frame) uniform in area inside a disk of the
    given diameter, no two closer than min_spacing_m (rejection sampling)."""
    r = diameter_m / 2.0
    pts = np.zeros((0, 2))
    tries = 0
    while len(pts) < n:
        cand = rng.uniform(-r, r, size=(4096, 2))
        cand = cand[np.hypot(cand[:, 0], cand[:, 1]) <= r]
        for c in cand:
            tries += 1
            if tries > max_tries:
                raise RuntimeError("disk layout infeasible for these spacings")
            if len(pts) == 0 or np.min(np.hypot(*(pts - c).T)) >= min_spacing_m:
                pts = np.vstack([pts, c])
                if len(pts) == n:
                    break
    return pts


def lattice_layout(n_side: int, spacing_m: float) -> np.ndarray:
    """Square n_side x n_side lattice centred on the station origin."""
    k = (np.arange(n_side) - n_side // 2) * spacing_m
    xx, yy = np.meshgrid(k, k)
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def station_layout(cfg: StationConfig, seed: int | None = None) -> np.ndarray:
    rng = np.random.default_rng(cfg.seed if seed is None else seed)
    if cfg.lattice:
        side = int(round(math.sqrt(cfg.n_elem)))
        return lattice_layout(side, cfg.cell_lambda * cfg.lam_m)
    return disk_layout(cfg.n_elem, cfg.diameter_m, cfg.min_spacing_m, rng)


# ----------------------------------------------------------------------------
# gridding kernel (user input of the method)
# ----------------------------------------------------------------------------
def gaussian_kernel(pos_m: np.ndarray, lam_m: float, cell_lambda: float,
                    grid_n: int, ksize: int, sigma_cells: float = 0.5):
    """Default illumination kernel: a real Gaussian of sigma_cells evaluated at
    the K x K cells around each element, normalised to unit sum.

    Returns (anchors int32 [n][2] = (x, y) of the window's first cell,
    taps float32 [n][K][K][2] indexed [v (y)][u (x)][re, im]).  Tap (u, v)
    belongs to cell (x0 + u, y0 + v) of the row-major [y][x] grid whose cell
    (N/2, N/2) holds the station origin."""
    g = pos_m / (lam_m * cell_lambda) + grid_n / 2.0          # cell coords
    centre = np.floor(g + 0.5).astype(np.int64)
    anchors = (centre - (ksize - 1) // 2).astype(np.int32)
    n = len(pos_m)
    taps = np.zeros((n, ksize, ksize, 2), np.float32)
    off = np.arange(ksize)
    for a in range(n):
        cx = anchors[a, 0] + off - g[a, 0]
        cy = anchors[a, 1] + off - g[a, 1]
        w = np.exp(-(cy[:, None] ** 2 + cx[None, :] ** 2) / (2 * sigma_cells ** 2))
        taps[a, :, :, 0] = (w / w.sum()).astype(np.float32)
    return anchors, taps


def unit_kernel(pos_m: np.ndarray, lam_m: float, cell_lambda: float,
                grid_n: int):
    """1 x 1 kernel of weight 1 at the nearest cell (elements on cells)."""
    return gaussian_kernel(pos_m, lam_m, cell_lambda, grid_n, 1)


def station_kernel(cfg: StationConfig, pos_m: np.ndarray):
    if cfg.ksize == 1:
        return unit_kernel(pos_m, cfg.lam_m, cfg.cell_lambda, cfg.grid_n)
    return gaussian_kernel(pos_m, cfg.lam_m, cfg.cell_lambda, cfg.grid_n, cfg.ksize)


# ----------------------------------------------------------------------------
# sky and voltages
# ----------------------------------------------------------------------------
def draw_sources(n_src: int, rng: np.random.Generator, fluxes=(),
                 max_dircos: float = 0.8):
    """Directions (l, m) uniform in area inside |s| <= max_dircos and fluxes
    (given, else dN/dS ~ S^-2 on [0.05, 1])."""
    rad = max_dircos * np.sqrt(rng.uniform(0, 1, n_src))
    ang = rng.uniform(0, 2 * np.pi, n_src)
    dirs = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    if len(fluxes):
        flux = np.asarray(fluxes, np.float64)
    else:
        u = rng.uniform(0, 1, n_src)
        smin, smax = 0.05, 1.0        # inverse CDF of S^-2 on [smin, smax]
        flux = 1.0 / (1.0 / smin - u * (1.0 / smin - 1.0 / smax))
    return dirs, flux


def voltages(pos_m: np.ndarray, lam_m: float, dirs: np.ndarray, flux: np.ndarray,
             n_chan: int, n_time: int, n_pol: int, seed: int,
             device="cpu", scale: float = 16.0, chan0: int = 0):
    """Quantised complex int8 voltages, torch tensor [C][T][P][N_e][2].

    Each source contributes amplitude A ~ CN(0, S/P) per (c, t, p) times
    exp(-2 pi i s.r/lambda) (so beamforming with exp(+2 pi i s.r/lambda)
    peaks on it); every element adds unit complex noise CN(0, 1).  Values are
    scale * x rounded half-to-even and clamped to [-127, 127]."""
    import torch

    gen = torch.Generator(device=device)
    ne = len(pos_m)
    out = torch.empty((n_chan, n_time, n_pol, ne, 2), dtype=torch.int8, device=device)
    ph = -2.0 * np.pi * (dirs @ pos_m.T) / lam_m                  # [src][ne]
    steer = torch.tensor(np.exp(1j * ph), dtype=torch.complex64, device=device)
    sd = torch.tensor(np.sqrt(flux / n_pol / 2.0), dtype=torch.float32, device=device)
    for c in range(n_chan):
        gen.manual_seed(int(seed) * 1000003 + chan0 + c)
        rows = n_time * n_pol
        a = torch.randn((rows, len(flux), 2), generator=gen, device=device) * sd[None, :, None]
        amp = torch.complex(a[..., 0], a[..., 1])
        sig = amp @ steer                                          # [rows][ne]
        nz = torch.randn((rows, ne, 2), generator=gen, device=device) * math.sqrt(0.5)
        x = torch.stack([sig.real, sig.imag], dim=-1) + nz
        q = torch.clamp(torch.round(x * scale), -127, 127).to(torch.int8)
        out[c] = q.view(n_time, n_pol, ne, 2)
    return out


def station_voltages(cfg: StationConfig, pos_m: np.ndarray, device="cpu",
                     n_chan: int | None = None, n_time: int | None = None,
                     chan0: int = 0):
    rng = np.random.default_rng(cfg.seed + 7)
    dirs, flux = draw_sources(cfg.n_src, rng, cfg.fluxes)
    return voltages(pos_m, cfg.lam_m, dirs, flux,
                    cfg.n_chan if n_chan is None else n_chan,
                    cfg.n_time if n_time is None else n_time,
                    cfg.n_pol, cfg.seed, device=device, chan0=chan0)


def random_voltages(shape, seed: int, device="cpu", lo: int = -128, hi: int = 127):
    """Uniform int8 values in [lo, hi] (adversarial / edge-case inputs)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    return torch.randint(lo, hi + 1, shape, generator=gen, device=device,
                         dtype=torch.int16).to(torch.int8)


# ----------------------------------------------------------------------------
# beamformer weights and hierarchical layouts
# ----------------------------------------------------------------------------
def round_half_away(x: np.ndarray) -> np.ndarray:
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def beam_directions(n_beam: int, lam_m: float, diameter_m: float) -> np.ndarray:
    """n_beam = s*s directions on a square lattice of spacing lambda/D_s
    centred on zenith."""
    s = int(round(math.sqrt(n_beam)))
    k = (np.arange(s) - (s - 1) / 2.0) * lam_m / diameter_m
    xx, yy = np.meshgrid(k, k)
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def bf_weights(pos_m: np.ndarray, lam_m: float, beam_dirs: np.ndarray,
               n_pol: int) -> np.ndarray:
    """int8 complex weights [K][P][N_e][2]: w = round(127 exp(-i phi)),
    phi = 2 pi s_k.r_a / lambda, so that conj(w) E steers as the BF sum does
    (same weights for both polarisations)."""
    ph = 2.0 * np.pi * (beam_dirs @ pos_m.T) / lam_m                 # [K][ne]
    w = np.stack([round_half_away(127 * np.cos(ph)),
                  round_half_away(-127 * np.sin(ph))], axis=-1)     # [K][ne][2]
    w = np.repeat(w[:, None], n_pol, axis=1)
    return np.clip(w, -127, 127).astype(np.int8)


def station_centres(cfg: HierarchyConfig) -> np.ndarray:
    """Stations in a compact core plus a sparse tail (log-uniform radius)."""
    rng = np.random.default_rng(cfg.seed)
    n_core = cfg.n_station - cfg.n_tail
    core = disk_layout(n_core, cfg.core_diameter_m, cfg.station.diameter_m, rng)
    rad = np.exp(rng.uniform(np.log(cfg.core_diameter_m / 2), np.log(cfg.tail_radius_m),
                             cfg.n_tail))
    ang = rng.uniform(0, 2 * np.pi, cfg.n_tail)
    tail = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    return np.vstack([core, tail])


def hierarchy_voltages(cfg: HierarchyConfig, centres_m: np.ndarray, elem_m: np.ndarray,
                       dirs: np.ndarray, flux: np.ndarray, n_station: int, n_chan: int,
                       n_time: int, device="cpu", scale: float = 16.0):
    """int8 voltages [S][C][T][P][N_e][2] of the first n_station stations: one
    sky per (channel, sample, pol) seen by every element at r_m + r_a with
    phase exp(-2 pi i s.(r_m + r_a) / lambda), plus independent unit complex
    noise per (station, element); quantised as `voltages`."""
    import torch

    P, ne, lam = cfg.n_pol, len(elem_m), cfg.station.lam_m
    out = torch.empty((n_station, n_chan, n_time, P, ne, 2), dtype=torch.int8, device=device)
    sd = torch.tensor(np.sqrt(flux / P / 2.0), dtype=torch.float32, device=device)
    gen = torch.Generator(device=device)
    rows = n_time * P
    for c in range(n_chan):
        gen.manual_seed(int(cfg.seed) * 1000003 + c)
        a = torch.randn((rows, len(flux), 2), generator=gen, device=device) * sd[None, :, None]
        amp = torch.complex(a[..., 0], a[..., 1])
        for m in range(n_station):
            ph = -2.0 * np.pi * (dirs @ (elem_m + centres_m[m]).T) / lam
            steer = torch.tensor(np.exp(1j * ph), dtype=torch.complex64, device=device)
            sig = amp @ steer
            gen.manual_seed(int(cfg.seed) * 1000003 + 7919 * (m + 1) + c)
            nz = torch.randn((rows, ne, 2), generator=gen, device=device) * math.sqrt(0.5)
            x = torch.stack([sig.real, sig.imag], dim=-1) + nz
            out[m, c] = torch.clamp(torch.round(x * scale), -127, 127).to(torch.int8).view(n_time, P, ne, 2)
    return out


def uneven_station_sizes(cfg: UnevenConfig) -> np.ndarray:
    rng = np.random.default_rng(cfg.seed)
    return np.exp(rng.uniform(np.log(cfg.n_min), np.log(cfg.n_max), cfg.n_station)
                  ).astype(np.int64)


def uneven_diameter(n_elem: int, cfg: UnevenConfig) -> float:
    """Station diameter: the 256-element station's, scaled with sqrt(N_e) so
    the element density stays that of the SKA-low station."""
    return cfg.ref_diameter_m * math.sqrt(n_elem / 256.0)


def uneven_grid_side(n_elem: int, cfg: UnevenConfig) -> int:
    """Padded grid side of a station: the next power of two >= 2 x (diameter
    in cells + K), i.e. padding factor 2 on the kernel's full support, clamped
    to [32, 256]."""
    need = 2.0 * (uneven_diameter(n_elem, cfg) / (cfg.lam_m * cfg.cell_lambda) + cfg.ksize)
    n = 32
    while n < need and n < 256:
        n *= 2
    return n


def uneven_station(cfg: UnevenConfig, index: int, n_elem: int | None = None) -> StationConfig:
    """StationConfig of station `index` of the uneven array (its own seed)."""
    ne = int(uneven_station_sizes(cfg)[index]) if n_elem is None else int(n_elem)
    return StationConfig(
        name=f"{cfg.name}_s{index}", n_elem=ne, diameter_m=uneven_diameter(ne, cfg),
        min_spacing_m=1.5, lam_m=cfg.lam_m, n_chan=cfg.n_chan, n_pol=cfg.n_pol,
        n_time=cfg.n_time, grid_n=uneven_grid_side(ne, cfg), cell_lambda=cfg.cell_lambda,
        ksize=cfg.ksize, n_src=20, seed=cfg.seed * 7919 + index)


def uneven_centres(cfg: UnevenConfig, n_station: int | None = None) -> np.ndarray:
    """Station centres of the uneven array: a disk of the core diameter with
    a minimum spacing of the largest station's diameter."""
    S = cfg.n_station if n_station is None else n_station
    rng = np.random.default_rng(cfg.seed + 17)
    return disk_layout(S, cfg.core_diameter_m, uneven_diameter(cfg.n_max, cfg), rng)


def uneven_beam_weights(cfg: UnevenConfig, positions, dirs: np.ndarray):
    """Beam weights of every station (bf_weights towards dirs, both pols)
    packed one station after another; returns (int8 buffer, byte offsets)."""
    blocks = [bf_weights(np.asarray(pos), cfg.lam_m, dirs, 2).reshape(-1) for pos in positions]
    off = np.zeros(len(blocks), np.int64)
    o = 0
    for s, b in enumerate(blocks):
        off[s] = o
        o += (b.size + 15) & ~15
    buf = np.zeros(max(o, 16), np.int8)
    for s, b in enumerate(blocks):
        buf[off[s]:off[s] + b.size] = b
    return buf, off

