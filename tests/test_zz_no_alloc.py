"""The allocation-free EPIC entry point against the regular one and the oracle.

hai_epic_image_fp32_static is for callers that cannot call cudaMalloc (it
keeps its gather table and partial images in a static device array inside
the library).  Through the C ABI it must give the image of hai_epic_image's
FP32 path on the same inputs, on consecutive calls that reuse the shared
array, and the FP64 oracle's image within the FP32 tolerance.  This file is
collected last so that a run stopping at the first failure has run every
other test first."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import FP32_TOL, rel_err_planes, station

pytestmark = pytest.mark.gpu


def reference_image(hai, anchors, taps, n, volt):
    C, T, P = volt.shape[:3]
    ctx = hai.hai_create(0)
    lay = hai.hai_layout_create(ctx, anchors, taps, n, P)
    img = torch.empty((C, lay.n_planes, n, n), device="cuda")
    hai.hai_epic_image(ctx, lay, volt, C, T, hai.HAI_PREC_FP32, img, 0)
    hai.hai_sync(ctx)
    hai.hai_layout_destroy(lay)
    hai.hai_destroy(ctx)
    return img.cpu().numpy()


def static_image(hai, anchors, taps, n, volt, accumulate=0, img=None):
    """Call the C entry point directly with a host layout description."""
    C, T, P, ne, _ = volt.shape
    anchors = np.ascontiguousarray(anchors, np.int32)
    taps = np.ascontiguousarray(taps, np.float32)
    desc = hai._LayoutDesc(ne, n, taps.shape[1], P, anchors.ctypes.data, taps.ctypes.data)
    if img is None:
        img = torch.full((C, 4 if P == 2 else 1, n, n), float("nan"), device="cuda")
    stream = torch.cuda.current_stream()
    rc = hai.load().hai_epic_image_fp32_static(0, ctypes.byref(desc), volt.data_ptr(), C, T,
                                               img.data_ptr(), accumulate, stream.cuda_stream)
    assert rc == 0, hai.hai_last_error()
    torch.cuda.synchronize()
    return img


def test_static_entry_matches_regular_entry_on_consecutive_calls(hai):
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    v1 = I.station_voltages(cfg, pos, n_chan=3, n_time=77, device="cuda")
    v2 = I.station_voltages(cfg, pos, n_chan=5, n_time=40, device="cuda", chan0=9)
    # two calls in a row on different cadences share (and overwrite) the array
    got1 = static_image(hai, anchors, taps, cfg.grid_n, v1).cpu().numpy()
    got2 = static_image(hai, anchors, taps, cfg.grid_n, v2).cpu().numpy()
    assert rel_err_planes(got1, reference_image(hai, anchors, taps, cfg.grid_n, v1)).max() < FP32_TOL
    assert rel_err_planes(got2, reference_image(hai, anchors, taps, cfg.grid_n, v2)).max() < FP32_TOL
    # and the oracle's images directly
    assert rel_err_planes(got1, O.epic_image(cfg.grid_n, anchors, taps, v1.cpu().numpy())).max() < FP32_TOL
    assert rel_err_planes(got2, O.epic_image(cfg.grid_n, anchors, taps, v2.cpu().numpy())).max() < FP32_TOL


def test_static_entry_other_layouts_and_accumulate(hai):
    cfg = I.SINGLE_STATION_64
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, n_time=300, device="cuda")
    want = reference_image(hai, anchors, taps, cfg.grid_n, volt)
    img = static_image(hai, anchors, taps, cfg.grid_n, volt)
    assert rel_err_planes(img.cpu().numpy(), want).max() < FP32_TOL
    img = static_image(hai, anchors, taps, cfg.grid_n, volt, accumulate=1, img=img)
    assert rel_err_planes(img.cpu().numpy(), 2 * want).max() < FP32_TOL
    assert rel_err_planes(img.cpu().numpy(), 2 * O.epic_image(cfg.grid_n, anchors, taps, volt.cpu().numpy())).max() \
        < FP32_TOL


def test_static_entry_direct_path_many_channels(hai):
    """64 channels: one CTA per channel writes the image in place (no partial
    images, no reduction), with and without accumulate."""
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, n_chan=64, n_time=6, device="cuda")
    want = O.epic_image(cfg.grid_n, anchors, taps, volt.cpu().numpy())
    img = static_image(hai, anchors, taps, cfg.grid_n, volt)
    assert rel_err_planes(img.cpu().numpy(), want).max() < FP32_TOL
    assert rel_err_planes(img.cpu().numpy(), reference_image(hai, anchors, taps, cfg.grid_n, volt)).max() < FP32_TOL
    img = static_image(hai, anchors, taps, cfg.grid_n, volt, accumulate=1, img=img)
    assert rel_err_planes(img.cpu().numpy(), 2 * want).max() < FP32_TOL


def test_static_entry_refuses_taps_off_the_grid(hai):
    cfg = I.SINGLE_STATION_64
    _, anchors, taps = station(cfg)
    anchors = anchors.copy()
    anchors[7] = (cfg.grid_n - 1, 3)                  # a 3x3 window starting on the last column
    volt = torch.zeros((1, 2, 1, len(anchors), 2), dtype=torch.int8, device="cuda")
    img = torch.zeros((1, 1, cfg.grid_n, cfg.grid_n), device="cuda")
    with pytest.raises(hai.HaiError) as e:
        hai.hai_epic_image_fp32_static(0, anchors, taps, cfg.grid_n, 1, volt, 1, 2, img)
    assert e.value.status == 2


def test_static_entry_rejects_sizes_beyond_its_maximum(hai):
    ne, k = 5000, 5                                   # 125000 gather entries > 102400
    anchors = np.zeros((ne, 2), np.int32)
    taps = np.zeros((ne, k, k, 2), np.float32)
    volt = torch.zeros((1, 1, 1, ne, 2), dtype=torch.int8, device="cuda")
    img = torch.zeros((1, 1, 64, 64), device="cuda")
    with pytest.raises(hai.HaiError) as e:
        hai.hai_epic_image_fp32_static(0, anchors, taps, 64, 1, volt, 1, 1, img)
    assert e.value.status == 4 and "maximum" in e.value.message
