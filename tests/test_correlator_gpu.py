"""GPU parity of the int8 correlator against the int64 oracle: bit-exact."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import station

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(hai):
    c = hai.hai_create(0)
    yield c
    hai.hai_destroy(c)


def run_corr(hai, ctx, volt, accumulate=0, vis=None):
    C, T, P, N, _ = volt.shape
    if vis is None:
        vis = torch.full((C, N * (N + 1) // 2, P, P, 2), -7, dtype=torch.int32, device="cuda")
    hai.hai_correlate(ctx, volt.cuda().contiguous(), C, T, N, P, vis, accumulate)
    hai.hai_sync(ctx)
    return vis.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("C,T,N,P", [
    (2, 40, 64, 2),      # one stage, several tiles
    (1, 100, 37, 1),     # ragged element count, ragged stage
    (3, 1, 16, 2),       # single sample
    (1, 600, 96, 2),     # crosses the 512-sample exact block
    (2, 1030, 130, 1),   # three blocks, ragged everything
    (1, 64, 256, 2),     # SKA-low station size
    (1, 96, 700, 2),     # several pack groups, the last one partial
])
def test_correlator_bit_exact(hai, ctx, C, T, N, P):
    volt = I.random_voltages((C, T, P, N, 2), seed=C * 1000 + T + N)
    got = run_corr(hai, ctx, volt)
    want = O.correlate(volt.numpy())
    assert np.array_equal(got, want)


def test_correlator_unaligned_voltages(hai, ctx):
    """A voltage pointer 2 bytes past a 16-byte boundary (N a multiple of 8):
    the pack takes its element-wise loads instead of 16-byte vectors."""
    C, T, N, P = 2, 77, 64, 2
    volt = I.random_voltages((C, T, P, N, 2), seed=9)
    flat = torch.zeros(volt.numel() + 16, dtype=torch.int8, device="cuda")
    flat[2:2 + volt.numel()] = volt.flatten().cuda()
    vis = torch.zeros((C, N * (N + 1) // 2, P, P, 2), dtype=torch.int32, device="cuda")
    hai.hai_correlate(ctx, flat[2:2 + volt.numel()], C, T, N, P, vis, 0)
    hai.hai_sync(ctx)
    assert np.array_equal(vis.cpu().numpy().astype(np.int64), O.correlate(volt.numpy()))


def test_correlator_adversarial_extremes(hai, ctx):
    """All -128 for 1024 samples: each 512-sample block sums to exactly 2^24."""
    C, T, N, P = 1, 1024, 64, 2
    volt = torch.full((C, T, P, N, 2), -128, dtype=torch.int8)
    got = run_corr(hai, ctx, volt)
    assert np.array_equal(got, O.correlate(volt.numpy()))
    assert got[0, 0, 0, 0, 0] == T * 2 * 128 * 128
    volt[:, ::3, :, ::2, 1] = 127
    volt[:, 1::5, 1, :, 0] = 127
    assert np.array_equal(run_corr(hai, ctx, volt), O.correlate(volt.numpy()))


def test_correlator_accumulate_and_limits(hai, ctx):
    C, T, N, P = 2, 70, 48, 2
    volt = I.random_voltages((C, T, P, N, 2), seed=5)
    vis = torch.zeros((C, N * (N + 1) // 2, P, P, 2), dtype=torch.int32, device="cuda")
    v = volt.cuda()
    hai.hai_correlate(ctx, v[:, :30].contiguous(), C, 30, N, P, vis, 0)
    hai.hai_correlate(ctx, v[:, 30:].contiguous(), C, 40, N, P, vis, 1)
    hai.hai_sync(ctx)
    assert np.array_equal(vis.cpu().numpy(), O.correlate(volt.numpy()))
    # T above the int32 bound: refused by the C ABI before anything launches
    rc = hai.load().hai_correlate(ctx, v.data_ptr(), C, 65536, N, P, vis.data_ptr(), 0, None)
    assert rc == 3 and "65535" in hai.hai_last_error()


def test_correlator_full_size_sampled_channels(hai, ctx):
    """The SKA-low cadence (64 channels x 2048 samples x 256 elements x 2 pols)
    in one launch; the oracle recomputes two channels."""
    cfg = I.SKA_LOW_STATION_256
    pos, _, _ = station(cfg)
    volt = I.station_voltages(cfg, pos, device="cuda")
    C, T, P, N = cfg.n_chan, cfg.n_time, cfg.n_pol, cfg.n_elem
    vis = torch.empty((C, N * (N + 1) // 2, P, P, 2), dtype=torch.int32, device="cuda")
    hai.hai_correlate(ctx, volt, C, T, N, P, vis, 0)
    hai.hai_sync(ctx)
    for c in (0, 45):
        want = O.correlate(volt[c:c + 1].cpu().numpy())
        assert np.array_equal(vis[c:c + 1].cpu().numpy().astype(np.int64), want)
