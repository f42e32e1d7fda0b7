"""hai_epic_image_host (EPIC on host buffers, channels streamed through the
GPU in chunks with the copies overlapping the imaging) against
hai_epic_image on device buffers, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2411_17804_gb300 import inputs as I
from tests.helpers import FP32_TOL, rel_err_planes, station

pytestmark = pytest.mark.gpu
CFG = I.SKA_LOW_STATION_256


@pytest.fixture(scope="module")
def ctx(hai):
    c = hai.hai_create(0)
    yield c
    hai.hai_destroy(c)


@pytest.fixture(scope="module")
def lay(hai, ctx):
    _, anchors, taps = station(CFG)
    L = hai.hai_layout_create(ctx, anchors, taps, CFG.grid_n, 2)
    yield L
    hai.hai_layout_destroy(L)


def device_image(hai, ctx, lay, volt, C, T, prec):
    img = torch.empty((C, 4, CFG.grid_n, CFG.grid_n), device="cuda")
    hai.hai_epic_image(ctx, lay, volt.cuda(), C, T, prec, img, 0)
    hai.hai_sync(ctx)
    return img.cpu().numpy()


def host_image(hai, ctx, lay, volt, C, T, prec, chunk, pin=True, accumulate=0, img=None):
    vh = volt.pin_memory() if pin else volt.clone()
    if img is None:
        img = torch.full((C, 4, CFG.grid_n, CFG.grid_n), float("nan"))
    ih = img.pin_memory() if pin else img
    hai.hai_epic_image_host(ctx, lay, vh, C, T, prec, ih, accumulate, chunk)
    hai.hai_sync(ctx)
    return ih.numpy()


@pytest.mark.parametrize("chunk", [0, 1, 2, 5, 7])
def test_host_path_matches_device_path_fp16(hai, ctx, lay, chunk):
    C, T = 5, 300
    volt = I.random_voltages((C, T, 2, CFG.n_elem, 2), seed=11)
    want = device_image(hai, ctx, lay, volt, C, T, hai.HAI_PREC_FP16)
    got = host_image(hai, ctx, lay, volt, C, T, hai.HAI_PREC_FP16, chunk)
    assert rel_err_planes(got, want).max() < FP32_TOL


def test_host_path_fp32_pageable_and_accumulate(hai, ctx, lay):
    C, T = 3, 64
    volt = I.random_voltages((C, T, 2, CFG.n_elem, 2), seed=12)
    want = device_image(hai, ctx, lay, volt, C, T, hai.HAI_PREC_FP32)
    got = host_image(hai, ctx, lay, volt, C, T, hai.HAI_PREC_FP32, 2, pin=False)
    assert rel_err_planes(got, want).max() < FP32_TOL
    # accumulate: the host image is copied in and added to
    acc = host_image(hai, ctx, lay, volt, C, T, hai.HAI_PREC_FP32, 2, accumulate=1,
                     img=torch.from_numpy(want.copy()))
    assert rel_err_planes(acc, 2 * want).max() < FP32_TOL


def test_host_path_empty_cadence_and_bad_arguments(hai, ctx, lay):
    C = 2
    img = host_image(hai, ctx, lay, torch.zeros((C, 0, 2, CFG.n_elem, 2), dtype=torch.int8), C, 0,
                     hai.HAI_PREC_FP16, 0)
    assert not np.isnan(img).any() and np.count_nonzero(img) == 0
    volt = torch.zeros((C, 4, 2, CFG.n_elem, 2), dtype=torch.int8)
    with pytest.raises(ValueError):        # device tensors are refused by the binding
        hai.hai_epic_image_host(ctx, lay, volt.cuda(), C, 4, hai.HAI_PREC_FP16,
                                torch.zeros((C, 4, CFG.grid_n, CFG.grid_n)))
    with pytest.raises(hai.HaiError) as e:
        hai.hai_epic_image_host(ctx, lay, volt, C, 4, hai.HAI_PREC_FP16,
                                torch.zeros((C, 4, CFG.grid_n, CFG.grid_n)), 0, -1)
    assert e.value.status == 1
