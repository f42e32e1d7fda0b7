"""GPU parity of the int8 voltage beamformer against the int64 oracle:
bit-exact int32 beams and int8 requantisation with the same saturation count."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(hai):
    c = hai.hai_create(0)
    yield c
    hai.hai_destroy(c)


def run_bf(hai, ctx, volt, w, shift=-1):
    S, C, T, P, N, _ = volt.shape
    K = w.shape[1]
    dt = torch.int32 if shift < 0 else torch.int8
    beams = torch.full((S, C, T, K, P, 2), 99, dtype=dt, device="cuda")
    sat = torch.zeros(1, dtype=torch.int64, device="cuda")
    hai.hai_beamform(ctx, volt.cuda().contiguous(), w.cuda().contiguous(), S, C, T, K, N, P, shift, beams, sat)
    hai.hai_sync(ctx)
    return beams.cpu().numpy(), int(sat.item())


@pytest.mark.parametrize("S,C,T,K,N,P", [
    (2, 2, 200, 16, 256, 2),   # station-shaped, ragged sample tile
    (3, 1, 128, 8, 64, 1),
    (1, 3, 50, 16, 40, 2),     # ragged element chunk
    (2, 1, 300, 24, 136, 2),
])
def test_beamformer_bit_exact(hai, ctx, S, C, T, K, N, P):
    volt = I.random_voltages((S, C, T, P, N, 2), seed=S + C + T + N)
    w = I.random_voltages((S, K, P, N, 2), seed=K + N, lo=-127)
    got, _ = run_bf(hai, ctx, volt, w)
    want = O.beamform(volt.numpy(), w.numpy())
    assert np.array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("S,C,T,K,N,P", [(2, 2, 130, 16, 256, 2), (1, 2, 70, 8, 64, 1), (2, 1, 260, 24, 96, 2)])
def test_beamformer_requantised(hai, ctx, S, C, T, K, N, P):
    volt = I.random_voltages((S, C, T, P, N, 2), seed=1)
    w = I.random_voltages((S, K, P, N, 2), seed=2, lo=-127)
    want = O.beamform(volt.numpy(), w.numpy())
    for shift in (0, 9, 12):
        got, sat = run_bf(hai, ctx, volt, w, shift)
        q, nsat = O.requant(want, shift)
        assert np.array_equal(got, q)
        assert sat == nsat


def test_beamformer_extremes_and_steering(hai, ctx):
    S, C, T, K, N, P = 1, 1, 64, 8, 512, 2
    volt = torch.full((S, C, T, P, N, 2), -128, dtype=torch.int8)
    w = torch.full((S, K, P, N, 2), -128, dtype=torch.int8)
    got, _ = run_bf(hai, ctx, volt, w)
    assert np.array_equal(got.astype(np.int64), O.beamform(volt.numpy(), w.numpy()))
    # station weights built for beam directions steer onto a plane wave
    rng = np.random.default_rng(3)
    pos = I.disk_layout(64, 12.0, 1.0, rng)
    dirs = I.beam_directions(16, 2.0, 12.0)
    wt = torch.tensor(I.bf_weights(pos, 2.0, dirs, 2))[None]
    ph = -2 * np.pi * (dirs[5] @ pos.T) / 2.0
    e = np.stack([np.round(90 * np.cos(ph)), np.round(90 * np.sin(ph))], -1).astype(np.int8)
    volt = torch.tensor(np.broadcast_to(e, (1, 1, 8, 2, 64, 2)).copy())
    got, _ = run_bf(hai, ctx, volt, wt)
    mag = np.hypot(got[0, 0, :, :, 0, 0], got[0, 0, :, :, 0, 1])
    assert np.all(np.argmax(mag, axis=1) == 5)
    assert np.array_equal(got.astype(np.int64), O.beamform(volt.numpy(), wt.numpy()))
