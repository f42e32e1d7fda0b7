"""Shared helpers of the GPU parity tests (inputs from the seeded generators,
expected values from the oracle only)."""
import numpy as np

from paper_2411_17804_gb300 import inputs as I

FP32_TOL = 1e-5     # per image plane, FP32 path
REDUCED_TOL = 2e-3  # per image plane, fp16 / bf16 tensor-core paths
# Split hi/lo tensor-core products are a reduced-precision path (fp16 / bf16
# operands), bound by REDUCED_TOL; the tests hold them to the FP32 level
# instead: Frobenius error < FP32_TOL and every pixel within SPLIT_PIXEL_TOL of
# the plane's peak.  Per pixel the FP32 accumulation of K products (in TMEM,
# K up to ~5,000 for the XBF) leaves about sqrt(K) 2^-24 of the sum of |terms|
# (~4e-6), and the dropped lo*lo term 2^-22 per product, on pixels where the
# terms cancel, so the per-pixel bound is twice the FP32 one.
SPLIT_PIXEL_TOL = 2e-5
# BF16 operands (unit roundoff u = 2^-8 against FP16's 2^-11).  The FP16 bound
# above comes from three roundings to the operand type (gridded values,
# stage-1 results, DFT operand) entering |F|^2 at about 2 sqrt(3) u; with
# bf16's u that is 1.35e-2, outside the 2e-3 reduced-precision tolerance, so
# plain BF16 is held to its own derived bound and the split form is the usable
# one.  Split into hi + lo parts, each rounded quantity keeps an error <= u^2
# and the dropped lo*lo product <= u^2, so |F|^2 is within about 8 u^2:
# 1.2e-4 for BF16 (inside 2e-3), 1.9e-6 for FP16 (the FP32 level).
BF16_TOL = 1.4e-2
BF16_SPLIT_TOL = 1.2e-4


def _plane_scales(want):
    """Per-(channel, plane) Frobenius norm and peak of the expected image, with
    the cross-polarisation planes (which may be near zero) measured against the
    auto planes' scale: floor at 1e-3 x the larger auto plane."""
    C, Q = want.shape[:2]
    w = want.reshape(C, Q, -1)
    den = np.linalg.norm(w, axis=-1)
    peak = np.abs(w).max(axis=-1)
    na = min(2, Q)
    den = np.maximum(den, 1e-3 * den[:, :na].max(axis=1, keepdims=True))
    peak = np.maximum(peak, 1e-3 * peak[:, :na].max(axis=1, keepdims=True))
    return den, peak


def frob_err_planes(got, want):
    """Relative Frobenius error per (channel, plane): [C][Q] (the reported
    image-error metric)."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    C, Q = want.shape[:2]
    num = np.linalg.norm((got - want).reshape(C, Q, -1), axis=-1)
    den, _ = _plane_scales(want)
    return num / den


def pixel_err_planes(got, want):
    """Element-by-element error per (channel, plane): max over pixels of
    |I_gpu - I_ref| / max |I_ref|: [C][Q]."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    C, Q = want.shape[:2]
    num = np.abs(got - want).reshape(C, Q, -1).max(axis=-1)
    _, peak = _plane_scales(want)
    return num / peak


def rel_err_planes(got, want):
    """Per (channel, plane) the larger of the relative Frobenius error and the
    per-pixel error |I_gpu - I_ref| / max |I_ref|, so that a test asserting
    `rel_err_planes(...) < tol` holds every pixel to the tolerance as well as
    the plane's norm.  NaN anywhere fails."""
    got = np.asarray(got, np.float64)
    if not np.all(np.isfinite(got)):
        return np.full(np.asarray(want).shape[:2], np.inf)
    return np.maximum(frob_err_planes(got, want), pixel_err_planes(got, want))


def station(cfg, seed=None):
    pos = I.station_layout(cfg, seed)
    anchors, taps = I.station_kernel(cfg, pos)
    return pos, anchors, taps
