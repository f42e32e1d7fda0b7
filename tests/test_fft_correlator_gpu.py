"""GPU parity of the FFT correlator (visibilities from accumulated EPIC images
by an inverse FFT) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import FP32_TOL, REDUCED_TOL, station

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(hai):
    c = hai.hai_create(0)
    yield c
    hai.hai_destroy(c)


def grid_err(got, want):
    """Error per (channel, alpha, beta) grid relative to the largest
    auto-polarisation grid of the channel, [C][P][P]: the larger of the
    Frobenius error (against that grid's norm) and the largest per-lag error
    (against that grid's largest |value|), so every lag is held to the
    tolerance."""
    C, P = want.shape[:2]
    if not np.all(np.isfinite(got)):
        return np.full((C, P, P), np.inf)
    num = np.linalg.norm((got - want).reshape(C, P, P, -1), axis=-1)
    auto = np.max([np.linalg.norm(want[:, p, p].reshape(C, -1), axis=-1) for p in range(P)], axis=0)
    pix = np.abs(got - want).reshape(C, P, P, -1).max(axis=-1)
    peak = np.max([np.abs(want[:, p, p]).reshape(C, -1).max(axis=-1) for p in range(P)], axis=0)
    return np.maximum(num / auto[:, None, None], pix / peak[:, None, None])


def fft_correlate(hai, ctx, img, N, P):
    C = img.shape[0]
    out = torch.full((C, P, P, N, N, 2), float("nan"), device="cuda")
    hai.hai_fft_correlate(ctx, img, C, N, P, out)
    hai.hai_sync(ctx)
    a = out.cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def epic(hai, ctx, anchors, taps, n, volt, prec):
    C, T, P = volt.shape[:3]
    lay = hai.hai_layout_create(ctx, anchors, taps, n, P)
    img = torch.empty((C, lay.n_planes, n, n), device="cuda")
    hai.hai_epic_image(ctx, lay, volt.cuda().contiguous(), C, T, prec, img, 0)
    hai.hai_sync(ctx)
    hai.hai_layout_destroy(lay)
    return img


@pytest.mark.parametrize("N,P,C", [(16, 2, 3), (32, 1, 2), (64, 2, 2), (128, 2, 1), (256, 1, 2), (512, 2, 1), (512, 1, 2)])
def test_inverse_transform_matches_oracle(hai, ctx, N, P, C):
    Q = 4 if P == 2 else 1
    planes = torch.from_numpy(np.random.default_rng(N + P).standard_normal((C, Q, N, N)).astype(np.float32))
    got = fft_correlate(hai, ctx, planes.cuda(), N, P)
    want = O.fft_correlate(planes.numpy())
    assert grid_err(got, want).max() < FP32_TOL


@pytest.mark.parametrize("prec,tol", [("FP32", FP32_TOL), ("FP16", REDUCED_TOL), ("FP16_SPLIT", FP32_TOL * 10)])
def test_ska_station_images_give_the_gridded_visibilities(hai, ctx, prec, tol):
    """SKA-low station (256 elements, 3 x 3 taps, 64^2 grid): EPIC image on
    the GPU, inverse FFT on the GPU = the oracle's correlator visibilities
    gridded with the illumination autocorrelation kernel."""
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, n_chan=2, n_time=24)
    img = epic(hai, ctx, anchors, taps, cfg.grid_n, volt, getattr(hai, "HAI_PREC_" + prec))
    got = fft_correlate(hai, ctx, img, cfg.grid_n, 2)
    want = O.xfft_grid(cfg.grid_n, anchors, taps, O.correlate(volt.numpy()))
    assert grid_err(got, want).max() < tol


def test_large_grid_station_gives_the_gridded_visibilities(hai, ctx):
    """A 700-element station of the uneven array on a 128^2 grid (the FP32
    large-grid EPIC path), one polarisation and two."""
    sc = I.uneven_station(I.UnevenConfig(), 0, 700)
    pos, anchors, taps = station(sc)
    for P in (1, 2):
        volt = I.random_voltages((2, 5, P, len(pos), 2), seed=40 + P)
        img = epic(hai, ctx, anchors, taps, 128, volt, hai.HAI_PREC_FP32)
        got = fft_correlate(hai, ctx, img, 128, P)
        want = O.xfft_grid(128, anchors, taps, O.correlate(volt.numpy()))
        assert grid_err(got, want).max() < FP32_TOL


def test_dense_lattice_lags_are_redundant_baseline_sums(hai, ctx):
    """The dense 128 x 128 lattice (one unit tap per element, 512^2 grid):
    every lag holds the sum over the baselines separated by it.  Whole grids
    against the oracle route; sampled lags against the sum written out from
    the voltages."""
    cfg = I.DENSE_ALLSKY_16384
    pos = I.station_layout(cfg)
    anchors, taps = I.station_kernel(cfg, pos)
    C, T, P, n = 1, 3, 2, cfg.grid_n
    volt = I.random_voltages((C, T, P, len(pos), 2), seed=77)
    img = epic(hai, ctx, anchors, taps, n, volt, hai.HAI_PREC_FP32)
    got = fft_correlate(hai, ctx, img, n, P)
    want = O.fft_correlate(O.epic_image(n, anchors, taps, volt.numpy()))
    assert grid_err(got, want).max() < FP32_TOL
    side = 128
    v = volt.numpy().astype(np.float64)
    e = (v[..., 0] + 1j * v[..., 1]).reshape(C, T, P, side, side)          # [c][t][p][iy][ix]
    scale = np.abs(want[0, 0, 0, 0, 0])
    for dx, dy in [(0, 0), (1, 0), (0, 1), (5, -3), (-17, 40), (127, 127), (-127, 0)]:
        ys, xs = slice(max(0, -dy), side - max(0, dy)), slice(max(0, -dx), side - max(0, dx))
        ys2, xs2 = slice(max(0, dy), side - max(0, -dy)), slice(max(0, dx), side - max(0, -dx))
        for al in range(P):
            for be in range(P):
                # sum over a = b + d of E_a conj(E_b)
                ref = np.sum(e[0, :, al, ys2, xs2] * np.conj(e[0, :, be, ys, xs]))
                g = got[0, al, be, dy % n, dx % n]
                assert abs(g - ref) < 1e-5 * scale, (dx, dy, al, be, g, ref)


def test_edge_cases_and_bad_arguments(hai, ctx):
    img = torch.zeros((1, 4, 64, 64), device="cuda")
    out = torch.zeros((1, 2, 2, 64, 64, 2), device="cuda")
    hai.hai_fft_correlate(ctx, img[:0], 0, 64, 2, out[:0])          # empty: no-op
    lib = hai.load()
    for N, P, status in [(8, 2, 4), (48, 2, 4), (1024, 2, 4), (64, 3, 1), (64, 0, 1)]:
        assert lib.hai_fft_correlate(ctx, img.data_ptr(), 1, N, P, out.data_ptr(), None) == status
    assert lib.hai_fft_correlate(ctx, img.data_ptr(), 1, 64, 2, out.data_ptr() + 4, None) == 1
    assert "aligned" in hai.hai_last_error()
    # an impulse at the phase-centre pixel of XX is a flat XX grid 1 / N^2;
    # the other grids stay zero
    img[0, 0, 32, 32] = 1.0
    hai.hai_fft_correlate(ctx, img, 1, 64, 2, out)
    hai.hai_sync(ctx)
    g = out.cpu().numpy()
    # pixel (32, 32): exp(-2 pi i 32 (dx + dy) / 64) (-1)^(dx+dy) = 1
    assert np.abs(g[0, 0, 0, ..., 0] - 1.0 / 4096).max() < 1e-9
    assert np.abs(g[0, 0, 0, ..., 1]).max() < 1e-9
    assert np.abs(g[0, 1]).max() == 0.0 and np.abs(g[0, 0, 1]).max() == 0.0
