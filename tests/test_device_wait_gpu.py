"""Failure detection on the device: a bounded mbarrier wait that runs out.

Every pipelined kernel of the library waits on mbarrier phases through one
bounded wait.  hai_check_device_wait makes that wait run out on purpose (one
CTA waits on a phase that nothing completes, no copy or MMA in flight, a limit
of a few thousand cycles): the kernel must end by itself, hai_sync must report
HAI_ERR_TIMEOUT once and clear the status word, and the context must stay
usable (an EPIC image after it still matches the oracle)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import FP32_TOL, rel_err_planes, station

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit", [1024, 4096, 1 << 20])
def test_wait_gives_up_and_context_survives(hai, limit):
    ctx = hai.hai_create(0)
    try:
        hai.hai_sync(ctx)                                   # clean start
        hai.hai_check_device_wait(ctx, limit)
        with pytest.raises(hai.HaiError) as e:
            hai.hai_sync(ctx)
        assert e.value.status == 6                          # HAI_ERR_TIMEOUT
        assert hai.hai_check_device_wait_result(ctx) == 1   # the wait itself gave up
        hai.hai_sync(ctx)                                   # the word was cleared
        # the context still images correctly after the timeout
        cfg = I.SINGLE_STATION_64
        pos, anchors, taps = station(cfg)
        volt = I.station_voltages(cfg, pos, n_time=64)
        lay = hai.hai_layout_create(ctx, anchors, taps, cfg.grid_n, cfg.n_pol)
        img = torch.zeros((1, 1, cfg.grid_n, cfg.grid_n), device="cuda")
        hai.hai_epic_image(ctx, lay, volt.cuda(), 1, 64, hai.HAI_PREC_FP32, img, 0)
        hai.hai_sync(ctx)
        hai.hai_layout_destroy(lay)
        want = O.epic_image(cfg.grid_n, anchors, taps, volt.numpy())
        assert rel_err_planes(img.cpu().numpy().astype(np.float64), want).max() < FP32_TOL
    finally:
        hai.hai_destroy(ctx)


def test_wait_limit_out_of_range_is_refused(hai):
    ctx = hai.hai_create(0)
    try:
        for bad in (0, 1023, (1 << 24) + 1):
            with pytest.raises(hai.HaiError) as e:
                hai.hai_check_device_wait(ctx, bad)
            assert e.value.status == 1
        hai.hai_sync(ctx)
    finally:
        hai.hai_destroy(ctx)
