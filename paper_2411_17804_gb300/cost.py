"""FLOP-cost model of the imaging architectures (Table 2) with the array
parameters of Table 1.

Every Table 2 entry is a FLOP count per station (intra-station) or per
station beam (inter-station) per voxel, one spectral channel times one
independent pixel, incurred once per timescale: per sample delta t
(25 us, Section 3) or per imaging cadence t_acc.  The cost density in FLOP
per second per voxel is each entry divided by its timescale, summed over the
architecture's components (Section 2's cost metric: a complex multiply is 6
FLOP, a complex add 2, a CMAC 8).

Host-side context for the measured throughputs; no part of the imaging path
uses it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

DELTA_T = 25e-6                 # nominal sample interval delta t (Section 3)
CADENCES = (1e-4, 1e-3, 1e-1, 10.0)   # the t_acc columns of Table 3
ARCHS = ("BF", "EPIC", "XBF", "XFFT")


@dataclass(frozen=True)
class ArrayParams:
    """One row of Table 1 (lengths in wavelengths)."""
    name: str
    lam_m: float
    DA: float        # array diameter D_A / lambda
    Ns: int          # stations
    Ds: float        # station diameter D_s / lambda
    Neps: int        # elements per station
    De: float        # element diameter D_e / lambda

    @property
    def f_A(self) -> float:
        """Array filling factor N_s (D_s / D_A)^2."""
        return self.Ns * (self.Ds / self.DA) ** 2

    @property
    def f_s(self) -> float:
        """Station filling factor N_eps (D_e / D_s)^2."""
        return self.Neps * (self.De / self.Ds) ** 2


ARRAYS = {
    "LAMBDA-I": ArrayParams("LAMBDA-I", 2.0, 3.9e6, 4, 17.5, 256, 1.0),
    "SKA-low-core": ArrayParams("SKA-low-core", 2.0, 5.25e2, 256, 17.5, 256, 1.0),
    "SKA-low": ArrayParams("SKA-low", 2.0, 3.5e4, 512, 17.5, 256, 1.0),
    # CASPA as printed (D_e / lambda = 0.5).  The station filling factor printed
    # beside it (0.996 = 65 (1 / 8.08)^2) and the station-level EPIC / XFFT
    # crossover of a few ms (Section 6, Table 3) both need D_e = lambda, which
    # CASPA_DE1 holds: Table 1 is inconsistent with itself on this row.
    "CASPA": ArrayParams("CASPA", 0.25, 4.6e4, 3, 8.08, 65, 0.5),
    "FarView-core": ArrayParams("FarView-core", 10.0, 6.77e2, 81, 38.5, 625, 1.0),
}


# The reading of CASPA that the printed f_s and Section 6 imply (D_e = lambda).
CASPA_DE1 = ArrayParams("CASPA (D_e = lambda)", 0.25, 4.6e4, 3, 8.08, 65, 1.0)


@dataclass(frozen=True)
class Term:
    component: str
    flop: float          # per voxel, per occurrence
    per: str             # "sample" (delta t) or "cadence" (t_acc)


def components(arch: str, n: int, ratio: float, n_p: int = 2, n_k: int = 1, gamma: float = 2.0,
               radix: int = 2) -> list[Term]:
    """Table 2 terms of one architecture.

    n      elements per station (intra-station) or stations (inter-station)
    ratio  D_s / D_e (intra) or D_A / D_s (inter): ratio^2 independent pixels
           per station (beam)
    n_k    gridding-kernel cells of EPIC (N_ke, N_ks); XFFT grids with 2^2 n_k
    gamma  EPIC padding factor per dimension (gamma_s, gamma_A)
    radix  FFT radix r."""
    pix = ratio * ratio
    pairs = n * (n - 1) / 2.0
    rl = radix / math.log2(radix)
    if arch == "BF":
        return [Term("beamforming", 8 * n_p ** 2 * n, "sample"),
                Term("squaring", 6 * n_p ** 2, "sample"),
                Term("accumulation", 2 * n_p ** 2, "sample")]
    if arch == "EPIC":
        return [Term("gridding", 6 * n_p ** 2 * n * n_k / pix, "sample"),
                Term("fft", 8 * n_p * rl * gamma ** 2 * math.log2((gamma * ratio) ** 2), "sample"),
                Term("squaring", 6 * n_p ** 2 * gamma ** 2, "sample"),
                Term("accumulation", 2 * n_p ** 2 * gamma ** 2, "sample")]
    corr = [Term("correlator", 6 * n_p ** 2 * pairs / pix, "sample"),
            Term("accumulation", 2 * n_p ** 2 * pairs / pix, "sample")]
    if arch == "XBF":
        return corr + [Term("dft", 8 * n_p ** 2 * pairs, "cadence")]
    if arch == "XFFT":
        return corr + [Term("gridding", 8 * n_p ** 4 * (4 * n_k) * pairs / pix, "cadence"),
                       Term("fft", 8 * n_p ** 2 * rl * math.log2(pix), "cadence")]
    raise ValueError(f"unknown architecture {arch}")


def density(arch: str, n: int, ratio: float, t_acc: float, **kw) -> float:
    """Cost density in FLOP/s per voxel at cadence t_acc."""
    return sum(t.flop / (DELTA_T if t.per == "sample" else t_acc) for t in components(arch, n, ratio, **kw))


def level_args(a: ArrayParams, level: str) -> tuple[int, float]:
    """(n, ratio) of the intra-station ("intra") or inter-station ("inter")
    stage of an array."""
    if level == "intra":
        return a.Neps, a.Ds / a.De
    if level == "inter":
        return a.Ns, a.DA / a.Ds
    raise ValueError(level)


def ranking(array, level: str, t_acc: float) -> list[tuple[str, float]]:
    """Architectures of one stage sorted by cost density (cheapest first);
    `array` is a Table 1 name or an ArrayParams."""
    n, ratio = level_args(ARRAYS[array] if isinstance(array, str) else array, level)
    return sorted(((x, density(x, n, ratio, t_acc)) for x in ARCHS), key=lambda p: p[1])


def flop_per_cadence(arch: str, n: int, ratio: float, channels: int, samples: int, **kw) -> float:
    """Table 2 FLOP of one station (or station beam) over one cadence of
    `samples` samples and `channels` channels: per-sample terms times the
    samples, per-cadence terms once, times ratio^2 voxels per channel."""
    terms = components(arch, n, ratio, **kw)
    per_voxel = sum(t.flop * (samples if t.per == "sample" else 1) for t in terms)
    return per_voxel * ratio * ratio * channels
