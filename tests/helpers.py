"""Shared helpers of the GPU parity tests (inputs from the seeded generators,
expected values from the oracle only)."""
import numpy as np

from paper_2411_17804_gb300 import inputs as I

FP32_TOL = 1e-5     # relative Frobenius error per image plane, FP32 path
REDUCED_TOL = 2e-3  # relative error per image plane, FP16 tensor-core path


def rel_err_planes(got, want):
    """Relative Frobenius error per (channel, plane): [C][Q] array."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    num = np.linalg.norm((got - want).reshape(got.shape[0], got.shape[1], -1), axis=-1)
    den = np.linalg.norm(want.reshape(want.shape[0], want.shape[1], -1), axis=-1)
    # cross-pol planes may be tiny; measure them against the auto planes' scale
    auto = np.max(den[:, : min(2, want.shape[1])], axis=1, keepdims=True)
    return num / np.maximum(den, 1e-3 * auto)


def station(cfg, seed=None):
    pos = I.station_layout(cfg, seed)
    anchors, taps = I.station_kernel(cfg, pos)
    return pos, anchors, taps
