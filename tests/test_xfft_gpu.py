"""GPU parity of the correlator + FFT imager against the oracle, and the
EPIC == XFFT invariant on the GPU (both device paths, same voltages)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import FP32_TOL, REDUCED_TOL, rel_err_planes, station

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(hai):
    c = hai.hai_create(0)
    yield c
    hai.hai_destroy(c)


def xfft_gpu(hai, ctx, anchors, taps, n, volt, accumulate=0, img=None):
    C, T, P, ne, _ = volt.shape
    lay = hai.hai_layout_create(ctx, anchors, taps, n, P)
    vis = torch.empty((C, ne * (ne + 1) // 2, P, P, 2), dtype=torch.int32, device="cuda")
    hai.hai_correlate(ctx, volt.cuda().contiguous(), C, T, ne, P, vis, 0)
    if img is None:
        img = torch.full((C, lay.n_planes, n, n), float("nan"), device="cuda")
    hai.hai_xfft_image(ctx, lay, vis, C, img, accumulate)
    hai.hai_sync(ctx)
    hai.hai_layout_destroy(lay)
    return img.cpu().numpy(), vis.cpu().numpy()


@pytest.mark.parametrize("n,P,ne,cplx", [(16, 1, 12, False), (16, 2, 20, True), (32, 2, 40, False)])
def test_xfft_matches_oracle(hai, ctx, n, P, ne, cplx):
    rng = np.random.default_rng(n * 7 + ne)
    k = 3
    anchors = rng.integers(0, n - k + 1, (ne, 2)).astype(np.int32)
    taps = rng.standard_normal((ne, k, k, 2)).astype(np.float32)
    if not cplx:
        taps[..., 1] = 0
    volt = I.random_voltages((2, 11, P, ne, 2), seed=ne)
    got, vis = xfft_gpu(hai, ctx, anchors, taps, n, volt)
    want = O.xfft_as_epic_planes(O.xfft_image(n, anchors, taps, vis.astype(np.int64)))
    assert rel_err_planes(got, want).max() < FP32_TOL


def test_epic_equals_xfft_on_gpu(hai, ctx):
    """Direct imaging (EPIC, FP32 and FP16 tensor-core paths) and the
    correlator + FFT imager give the same image from the same voltages."""
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, n_chan=2, n_time=96)
    n = cfg.grid_n
    ximg, _ = xfft_gpu(hai, ctx, anchors, taps, n, volt)
    lay = hai.hai_layout_create(ctx, anchors, taps, n, 2)
    for prec, tol in ((hai.HAI_PREC_FP32, FP32_TOL), (hai.HAI_PREC_FP16, REDUCED_TOL)):
        img = torch.empty((2, 4, n, n), device="cuda")
        hai.hai_epic_image(ctx, lay, volt.cuda(), 2, 96, prec, img, 0)
        hai.hai_sync(ctx)
        assert rel_err_planes(img.cpu().numpy(), ximg).max() < tol
    hai.hai_layout_destroy(lay)
    want = O.epic_image(n, anchors, taps, volt.numpy())
    assert rel_err_planes(ximg, want).max() < FP32_TOL


def test_xfft_accumulate(hai, ctx):
    cfg = I.SINGLE_STATION_64
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, n_time=64)
    n = cfg.grid_n
    first, vis = xfft_gpu(hai, ctx, anchors, taps, n, volt)
    img = torch.tensor(first, device="cuda")
    again, _ = xfft_gpu(hai, ctx, anchors, taps, n, volt, accumulate=1, img=img)
    assert rel_err_planes(again, 2 * first).max() < FP32_TOL


def test_xfft_is_deterministic(hai, ctx):
    """Each grid cell sums its contributions in a fixed order: repeated calls
    agree to the bit (the layout's gridding list is built by the first)."""
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, n_chan=3, n_time=64)
    n = cfg.grid_n
    lay = hai.hai_layout_create(ctx, anchors, taps, n, 2)
    vis = torch.empty((3, cfg.n_elem * (cfg.n_elem + 1) // 2, 2, 2, 2), dtype=torch.int32, device="cuda")
    hai.hai_correlate(ctx, volt.cuda(), 3, 64, cfg.n_elem, 2, vis, 0)
    a = torch.empty((3, 4, n, n), device="cuda")
    b = torch.full((3, 4, n, n), float("nan"), device="cuda")
    hai.hai_xfft_image(ctx, lay, vis, 3, a)
    hai.hai_xfft_image(ctx, lay, vis, 3, b)
    hai.hai_sync(ctx)
    assert torch.equal(a, b)
    hai.hai_layout_destroy(lay)
