"""Layouts built by the library from element positions, the anchors and taps
it exports for the oracle, and the workspace-size queries."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import FP32_TOL, REDUCED_TOL, rel_err_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(hai):
    c = hai.hai_create(0)
    yield c
    hai.hai_destroy(c)


@pytest.mark.parametrize("cfg,k,sigma", [(I.SKA_LOW_STATION_256, 3, 0.5), (I.SINGLE_STATION_64, 3, 0.7),
                                         (I.SKA_LOW_STATION_256, 5, 1.0), (I.DENSE_ALLSKY_16384, 1, 0.5)])
def test_default_kernel_from_positions(hai, ctx, cfg, k, sigma):
    """The library's Gaussian illumination kernel from positions equals the
    seeded generator's (same reading: nearest cell, K x K window, unit sum)."""
    pos = I.station_layout(cfg)
    lay = hai.hai_layout_create_from_positions(ctx, pos, cfg.lam_m, cfg.cell_lambda, cfg.grid_n, k, sigma, cfg.n_pol)
    try:
        anchors, taps = hai.hai_layout_anchors(lay)
        want_a, want_t = I.gaussian_kernel(pos, cfg.lam_m, cfg.cell_lambda, cfg.grid_n, k, sigma)
        assert np.array_equal(anchors, want_a)
        np.testing.assert_allclose(taps, want_t, rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(taps[..., 0].sum(axis=(1, 2)), 1.0, rtol=1e-6)
        assert np.all(taps[..., 1] == 0)
    finally:
        hai.hai_layout_destroy(lay)


def test_image_of_a_position_layout_matches_oracle(hai, ctx):
    """EPIC on a layout from positions against the oracle fed with the anchors
    and taps the library exports (inputs shared, not code)."""
    cfg = I.SKA_LOW_STATION_256
    pos = I.station_layout(cfg)
    lay = hai.hai_layout_create_from_positions(ctx, pos, cfg.lam_m, cfg.cell_lambda, cfg.grid_n, 3, 0.5, 2)
    try:
        anchors, taps = hai.hai_layout_anchors(lay)
        volt = I.station_voltages(cfg, pos, n_chan=2, n_time=33)
        want = O.epic_image(cfg.grid_n, anchors, taps, volt.numpy())
        for prec, tol in ((hai.HAI_PREC_FP32, FP32_TOL), (hai.HAI_PREC_FP16, REDUCED_TOL)):
            img = torch.full((2, 4, cfg.grid_n, cfg.grid_n), float("nan"), device="cuda")
            hai.hai_epic_image(ctx, lay, volt.cuda(), 2, 33, prec, img, 0)
            hai.hai_sync(ctx)
            assert rel_err_planes(img.cpu().numpy(), want).max() < tol
    finally:
        hai.hai_layout_destroy(lay)


def test_positions_off_the_grid_are_refused(hai, ctx):
    pos = np.array([[0.0, 0.0], [200.0, 0.0]])          # 200 m at 1.5 m cells: far outside a 64^2 grid
    with pytest.raises(hai.HaiError) as e:
        hai.hai_layout_create_from_positions(ctx, pos, 3.0, 0.5, 64, 3, 0.5, 2)
    assert e.value.status == 2
    with pytest.raises(hai.HaiError) as e:
        hai.hai_layout_create_from_positions(ctx, pos[:1], 3.0, 0.5, 64, 3, 0.0, 2)
    assert e.value.status == 1


def test_workspace_sizes(hai, ctx):
    """Layouts report the device memory they hold: more for a large grid (its
    tensor-core batch scratch and the FP32 path's two 1 GB row scratches)
    than for a small one; a plan reports its tables
    and schedule; a context its status words and DFT operands."""
    small = I.SKA_LOW_STATION_256
    pos = I.station_layout(small)
    an, tp = I.station_kernel(small, pos)
    l64 = hai.hai_layout_create(ctx, an, tp, 64, 2)
    dense = I.DENSE_ALLSKY_16384
    dpos = I.station_layout(dense)
    dan, dtp = I.station_kernel(dense, dpos)
    l512 = hai.hai_layout_create(ctx, dan, dtp, 512, 2)
    try:
        b64, b512 = hai.hai_layout_workspace_size(l64), hai.hai_layout_workspace_size(l512)
        assert 0 < b64 < 64 << 20
        assert b512 > 2 << 30
        assert hai.hai_ctx_workspace_size(ctx) > 0
        plan = hai.hai_plan_create(ctx, [l64, l64], 2, 8)
        try:
            assert hai.hai_workspace_size(plan) > 0
        finally:
            hai.hai_plan_destroy(plan)
    finally:
        hai.hai_layout_destroy(l64)
        hai.hai_layout_destroy(l512)
