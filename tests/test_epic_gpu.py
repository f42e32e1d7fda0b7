"""GPU parity of the EPIC imager (FP32 path) against the FP64 oracle, through
the C ABI."""
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


def run_epic(hai, ctx, anchors, taps, n, volt, prec, accumulate=0, img=None):
    C, T, P = volt.shape[:3]
    lay = hai.hai_layout_create(ctx, anchors, taps, n, P)
    try:
        if img is None:
            img = torch.full((C, lay.n_planes, n, n), float("nan"), device="cuda")
        hai.hai_epic_image(ctx, lay, volt.cuda().contiguous(), C, T, prec, img, accumulate)
        hai.hai_sync(ctx)
        return img.cpu().numpy()
    finally:
        hai.hai_layout_destroy(lay)


def test_single_station_64_full_size(hai, ctx):
    cfg = I.SINGLE_STATION_64
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos)
    got = run_epic(hai, ctx, anchors, taps, cfg.grid_n, volt, hai.HAI_PREC_FP32)
    want = O.epic_image(cfg.grid_n, anchors, taps, volt.numpy())
    err = rel_err_planes(got, want)
    assert err.max() < FP32_TOL, err
    assert np.abs(got - want).max() / np.abs(want).max() < FP32_TOL


@pytest.mark.parametrize("C,T", [(3, 40), (1, 7), (5, 1), (2, 301)])
def test_ska_station_ragged_splits(hai, ctx, C, T):
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, n_chan=C, n_time=T)
    got = run_epic(hai, ctx, anchors, taps, cfg.grid_n, volt, hai.HAI_PREC_FP32)
    want = O.epic_image(cfg.grid_n, anchors, taps, volt.numpy())
    assert rel_err_planes(got, want).max() < FP32_TOL


@pytest.mark.parametrize("n,P,ne", [(16, 1, 5), (16, 2, 1), (32, 2, 40), (64, 1, 300)])
def test_grid_sizes_pols_and_element_counts(hai, ctx, n, P, ne):
    rng = np.random.default_rng(n + P + ne)
    k = 3
    anchors = rng.integers(0, n - k + 1, (ne, 2)).astype(np.int32)
    taps = rng.standard_normal((ne, k, k, 2)).astype(np.float32)
    volt = I.random_voltages((2, 9, P, ne, 2), seed=ne)
    got = run_epic(hai, ctx, anchors, taps, n, volt, hai.HAI_PREC_FP32)
    want = O.epic_image(n, anchors, taps, volt.numpy())
    assert rel_err_planes(got, want).max() < FP32_TOL


@pytest.mark.parametrize("P,bw,bh,ne,C,T", [
    (2, 20, 48, 64, 3, 41),     # box at most 32 cells wide, taller than 32
    (2, 48, 20, 64, 2, 17),     # wider than 32, at most 32 tall
    (2, 64, 64, 200, 2, 9),     # the whole grid
    (1, 30, 30, 7, 3, 23),      # one pol, 14-byte samples (plain voltage loads)
    (1, 50, 40, 9, 2, 10),      # one pol, box over 32 both ways
    (2, 33, 31, 5, 2, 12),      # one cell over half the grid along x; 20-byte samples
    (2, 29, 28, 256, 160, 2),   # more channels than CTAs: one CTA per channel
])
def test_fp32_64_box_forms(hai, ctx, P, bw, bh, ne, C, T):
    """The N = 64 FP32 kernel's box forms (at most 32 cells, or more, along x
    and along y), one and two pols, samples that do or do not fill whole
    16-byte copies, the time split, and one CTA per channel with accumulate."""
    n, k = 64, 3
    rng = np.random.default_rng(bw * 1000 + bh * 10 + ne)
    x0, y0 = (n - bw) // 2, n - bh
    ax = rng.integers(x0, x0 + bw - k + 1, ne)
    ay = rng.integers(y0, y0 + bh - k + 1, ne)
    ax[0], ay[0] = x0, y0
    ax[-1], ay[-1] = x0 + bw - k, y0 + bh - k
    anchors = np.stack([ax, ay], 1).astype(np.int32)
    taps = rng.standard_normal((ne, k, k, 2)).astype(np.float32)
    volt = I.random_voltages((C, T, P, ne, 2), seed=bw + bh + ne)
    lay = hai.hai_layout_create(ctx, anchors, taps, n, P)
    try:
        assert list(hai.hai_layout_box(lay)) == [x0, y0, x0 + bw, y0 + bh]
        v = volt.cuda().contiguous()
        img = torch.full((C, lay.n_planes, n, n), float("nan"), device="cuda")
        hai.hai_epic_image(ctx, lay, v, C, T, hai.HAI_PREC_FP32, img, 0)
        hai.hai_sync(ctx)
        want = O.epic_image(n, anchors, taps, volt.numpy())
        assert rel_err_planes(img.cpu().numpy(), want).max() < FP32_TOL
        hai.hai_epic_image(ctx, lay, v, C, T, hai.HAI_PREC_FP32, img, 1)
        hai.hai_sync(ctx)
        assert rel_err_planes(img.cpu().numpy(), 2 * want).max() < FP32_TOL
    finally:
        hai.hai_layout_destroy(lay)


def test_adversarial_extreme_voltages(hai, ctx):
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = torch.full((2, 16, 2, len(pos), 2), -128, dtype=torch.int8)
    volt[:, ::2, 1, :, 1] = 127
    got = run_epic(hai, ctx, anchors, taps, cfg.grid_n, volt, hai.HAI_PREC_FP32)
    want = O.epic_image(cfg.grid_n, anchors, taps, volt.numpy())
    assert rel_err_planes(got, want).max() < FP32_TOL


def test_accumulate_and_empty_cadence(hai, ctx):
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, n_chan=2, n_time=12)
    n = cfg.grid_n
    lay = hai.hai_layout_create(ctx, anchors, taps, n, 2)
    img = torch.zeros((2, 4, n, n), device="cuda")
    v = volt.cuda()
    hai.hai_epic_image(ctx, lay, v[:, :5].contiguous(), 2, 5, hai.HAI_PREC_FP32, img, 0)
    hai.hai_epic_image(ctx, lay, v[:, 5:].contiguous(), 2, 7, hai.HAI_PREC_FP32, img, 1)
    hai.hai_sync(ctx)
    want = O.epic_image(n, anchors, taps, volt.numpy())
    assert rel_err_planes(img.cpu().numpy(), want).max() < FP32_TOL
    # T = 0 zeroes the image (accumulate = 0) or leaves it (accumulate = 1)
    hai.hai_epic_image(ctx, lay, v, 2, 0, hai.HAI_PREC_FP32, img, 1)
    hai.hai_sync(ctx)
    assert rel_err_planes(img.cpu().numpy(), want).max() < FP32_TOL
    hai.hai_epic_image(ctx, lay, v, 2, 0, hai.HAI_PREC_FP32, img, 0)
    hai.hai_sync(ctx)
    assert torch.count_nonzero(img).item() == 0
    hai.hai_layout_destroy(lay)


def test_deterministic(hai, ctx):
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, n_chan=3, n_time=50)
    a = run_epic(hai, ctx, anchors, taps, cfg.grid_n, volt, hai.HAI_PREC_FP32)
    b = run_epic(hai, ctx, anchors, taps, cfg.grid_n, volt, hai.HAI_PREC_FP32)
    assert np.array_equal(a, b)


def test_off_grid_and_bad_args(hai, ctx):
    anchors = np.array([[62, 3]], np.int32)
    taps = np.ones((1, 3, 3, 2), np.float32)
    with pytest.raises(hai.HaiError) as e:
        hai.hai_layout_create(ctx, anchors, taps, 64, 1)
    assert e.value.status == 2
    with pytest.raises(hai.HaiError) as e:
        hai.hai_layout_create(ctx, np.array([[1, 1]], np.int32), taps, 48, 1)
    assert e.value.status == 1


def test_ska_station_full_size_sampled_channels(hai, ctx):
    """Full cadence (64 channels x 2048 samples) in the benchmark's launch
    configuration; the oracle recomputes three channels."""
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, device="cuda")
    n = cfg.grid_n
    lay = hai.hai_layout_create(ctx, anchors, taps, n, 2)
    img = torch.empty((cfg.n_chan, 4, n, n), device="cuda")
    hai.hai_epic_image(ctx, lay, volt, cfg.n_chan, cfg.n_time, hai.HAI_PREC_FP32, img, 0)
    hai.hai_sync(ctx)
    hai.hai_layout_destroy(lay)
    for c in (0, 37, 63):
        want = O.epic_image(n, anchors, taps, volt[c:c + 1].cpu().numpy())
        assert rel_err_planes(img[c:c + 1].cpu().numpy(), want).max() < FP32_TOL


# ------------------------------------------------------------------ FP16 tensor-core path
@pytest.mark.parametrize("C,T", [(3, 40), (1, 7), (5, 1), (2, 301), (1, 2), (4, 33)])
def test_tc_ska_station_ragged_splits(hai, ctx, C, T):
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, n_chan=C, n_time=T)
    got = run_epic(hai, ctx, anchors, taps, cfg.grid_n, volt, hai.HAI_PREC_FP16)
    want = O.epic_image(cfg.grid_n, anchors, taps, volt.numpy())
    err = rel_err_planes(got, want)
    assert err.max() < REDUCED_TOL, err


def test_tc_full_size_sampled_channels(hai, ctx):
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, device="cuda")
    n = cfg.grid_n
    lay = hai.hai_layout_create(ctx, anchors, taps, n, 2)
    img = torch.empty((cfg.n_chan, 4, n, n), device="cuda")
    hai.hai_epic_image(ctx, lay, volt, cfg.n_chan, cfg.n_time, hai.HAI_PREC_FP16, img, 0)
    hai.hai_sync(ctx)
    hai.hai_layout_destroy(lay)
    for c in (0, 31, 63):
        want = O.epic_image(n, anchors, taps, volt[c:c + 1].cpu().numpy())
        err = rel_err_planes(img[c:c + 1].cpu().numpy(), want)
        assert err.max() < REDUCED_TOL, (c, err)


def test_tc_adversarial_and_random_taps(hai, ctx):
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = torch.full((2, 16, 2, len(pos), 2), -128, dtype=torch.int8)
    volt[:, ::2, 1, :, 1] = 127
    got = run_epic(hai, ctx, anchors, taps, cfg.grid_n, volt, hai.HAI_PREC_FP16)
    want = O.epic_image(cfg.grid_n, anchors, taps, volt.numpy())
    assert rel_err_planes(got, want).max() < REDUCED_TOL
    # complex taps, uniform random voltages
    rng = np.random.default_rng(3)
    ctaps = taps.copy()
    ctaps[..., 1] = 0.3 * rng.standard_normal(taps.shape[:-1]).astype(np.float32)
    volt = I.random_voltages((2, 24, 2, len(pos), 2), seed=77)
    got = run_epic(hai, ctx, anchors, ctaps, cfg.grid_n, volt, hai.HAI_PREC_FP16)
    want = O.epic_image(cfg.grid_n, anchors, ctaps, volt.numpy())
    assert rel_err_planes(got, want).max() < REDUCED_TOL


def test_tc_accumulate_and_deterministic(hai, ctx):
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    volt = I.station_voltages(cfg, pos, n_chan=2, n_time=20)
    n = cfg.grid_n
    lay = hai.hai_layout_create(ctx, anchors, taps, n, 2)
    img = torch.zeros((2, 4, n, n), device="cuda")
    v = volt.cuda()
    hai.hai_epic_image(ctx, lay, v[:, :9].contiguous(), 2, 9, hai.HAI_PREC_FP16, img, 0)
    hai.hai_epic_image(ctx, lay, v[:, 9:].contiguous(), 2, 11, hai.HAI_PREC_FP16, img, 1)
    hai.hai_sync(ctx)
    want = O.epic_image(n, anchors, taps, volt.numpy())
    assert rel_err_planes(img.cpu().numpy(), want).max() < REDUCED_TOL
    a = run_epic(hai, ctx, anchors, taps, n, volt, hai.HAI_PREC_FP16)
    b = run_epic(hai, ctx, anchors, taps, n, volt, hai.HAI_PREC_FP16)
    assert np.array_equal(a, b)
    hai.hai_layout_destroy(lay)


@pytest.mark.parametrize("n_elem,C,T", [
    (40, 3, 37),      # N = 32: time split over CTAs, ragged 4-sample steps
    (40, 160, 5),     # N = 32: one CTA per channel
    (60, 1, 1),       # N = 32: a single sample
    (300, 2, 9),      # N = 64 station of the uneven array
    (700, 2, 13),     # N = 128: time split over 4-CTA clusters
    (1000, 40, 3),    # N = 128: one cluster per channel, largest station
    (500, 1, 2),      # N = 128: fewer samples than clusters
])
def test_tc_uneven_station_grid_sides(hai, ctx, n_elem, C, T):
    """Stations of the uneven array at their own grid side (32, 64, 128):
    voltages of the seeded sky, then complex taps with uniform voltages; both
    also accumulated a second time onto the first result."""
    sc = I.uneven_station(I.UnevenConfig(), 0, n_elem)
    pos, anchors, taps = station(sc)
    n = sc.grid_n
    rng = np.random.default_rng(n_elem)
    ctaps = taps.copy()
    ctaps[..., 1] = 0.3 * rng.standard_normal(taps.shape[:-1]).astype(np.float32)
    cases = [(taps, I.station_voltages(sc, pos, n_chan=C, n_time=T)),
             (ctaps, I.random_voltages((C, T, 2, len(pos), 2), seed=n_elem + C + T))]
    for tp, volt in cases:
        lay = hai.hai_layout_create(ctx, anchors, tp, n, 2)
        img = torch.full((C, 4, n, n), float("nan"), device="cuda")
        v = volt.cuda()
        hai.hai_epic_image(ctx, lay, v, C, T, hai.HAI_PREC_FP16, img, 0)
        hai.hai_sync(ctx)
        want = O.epic_image(n, anchors, tp, volt.numpy())
        got = img.cpu().numpy()
        assert rel_err_planes(got, want).max() < REDUCED_TOL, (n, rel_err_planes(got, want).max())
        hai.hai_epic_image(ctx, lay, v, C, T, hai.HAI_PREC_FP16, img, 1)
        hai.hai_sync(ctx)
        assert rel_err_planes(img.cpu().numpy(), 2 * want).max() < REDUCED_TOL
        hai.hai_layout_destroy(lay)


def test_tc_unsupported_layout_is_reported(hai, ctx):
    cfg = I.SINGLE_STATION_64
    pos, anchors, taps = station(cfg)
    lay = hai.hai_layout_create(ctx, anchors, taps, cfg.grid_n, 1)
    img = torch.zeros((1, 1, cfg.grid_n, cfg.grid_n), device="cuda")
    volt = torch.zeros((1, 4, 1, len(pos), 2), dtype=torch.int8, device="cuda")
    with pytest.raises(hai.HaiError) as e:
        hai.hai_epic_image(ctx, lay, volt, 1, 4, hai.HAI_PREC_FP16, img, 0)
    assert e.value.status == 4
    hai.hai_layout_destroy(lay)


# ------------------------------------------------------------------ FP32, large grids (N = 128 .. 512)
def _dense(n_side=128):
    cfg = I.DENSE_ALLSKY_16384
    pos = I.station_layout(cfg)
    anchors, taps = I.station_kernel(cfg, pos)
    return cfg, pos, anchors, taps


@pytest.mark.parametrize("case,C,T,P", [
    ("n128", 2, 5, 2),        # a 700-element station of the uneven array
    ("n256", 3, 7, 2),        # the SKA station on a 256^2 grid
    ("n512", 2, 3, 2),        # the dense lattice, 128 x 128 box
    ("n512", 1, 2, 1),        # one polarisation
    ("n512", 9, 9, 2),        # two sample batches and two channel blocks of the row scratch
    ("n512_cplx", 3, 4, 2),   # 3 x 3 complex taps, random anchors: several entries per cell, box < 128
    ("n512_wide", 2, 3, 2),   # a box wider than 128 cells (the general transforms)
    ("n512_tall", 2, 3, 2),   # a box taller than 128 cells
])
def test_large_grid_fp32_matches_oracle(hai, ctx, case, C, T, P):
    if case.startswith("n512_"):
        rng = np.random.default_rng(len(case))
        n, ne, k = 512, 150, 3
        wx, wy = {"n512_cplx": (100, 120), "n512_wide": (200, 90), "n512_tall": (90, 200)}[case]
        anchors = np.stack([rng.integers(5, 5 + wx - k, ne), rng.integers(7, 7 + wy - k, ne)], axis=1).astype(np.int32)
        taps = rng.standard_normal((ne, k, k, 2)).astype(np.float32)
        volt = I.random_voltages((C, T, P, ne, 2), seed=C + 3 * T)
    elif case == "n128":
        sc = I.uneven_station(I.UnevenConfig(), 0, 700)
        pos, anchors, taps = station(sc)
        n = 128
        volt = I.random_voltages((C, T, P, len(pos), 2), seed=C + T)
    elif case == "n256":
        pos, anchors, taps = station(I.SKA_LOW_STATION_256)
        n = 256
        volt = I.random_voltages((C, T, P, len(pos), 2), seed=C * T)
    else:
        cfg, pos, anchors, taps = _dense()
        n = 512
        volt = I.random_voltages((C, T, P, len(pos), 2), seed=C + 2 * T)
    got = run_epic(hai, ctx, anchors, taps, n, volt, hai.HAI_PREC_FP32)
    want = O.epic_image(n, anchors, taps, volt.numpy())
    assert rel_err_planes(got, want).max() < FP32_TOL
    # accumulate onto the first result
    lay = hai.hai_layout_create(ctx, anchors, taps, n, P)
    img = torch.from_numpy(got).cuda()
    hai.hai_epic_image(ctx, lay, volt.cuda(), C, T, hai.HAI_PREC_FP32, img, 1)
    hai.hai_sync(ctx)
    assert rel_err_planes(img.cpu().numpy(), 2 * want).max() < FP32_TOL
    hai.hai_layout_destroy(lay)


def test_dense_allsky_full_cadence_sampled_channel(hai, ctx):
    """The dense all-sky lattice at full size (16,384 elements, 512^2 grid,
    16 channels, 2 pols, 100 samples of the seeded sky) in one call; the
    oracle recomputes channel 0."""
    cfg, pos, anchors, taps = _dense()
    volt = I.station_voltages(cfg, pos, device="cuda")
    n, C, T = cfg.grid_n, cfg.n_chan, cfg.n_time
    lay = hai.hai_layout_create(ctx, anchors, taps, n, 2)
    img = torch.empty((C, 4, n, n), device="cuda")
    hai.hai_epic_image(ctx, lay, volt, C, T, hai.HAI_PREC_FP32, img, 0)
    hai.hai_sync(ctx)
    hai.hai_layout_destroy(lay)
    want = O.epic_image(n, anchors, taps, volt[:1].cpu().numpy())
    assert rel_err_planes(img[:1].cpu().numpy(), want).max() < FP32_TOL


@pytest.mark.parametrize("case,C,T", [
    ("n512", 2, 3),           # the dense lattice: 128 x 128 box, 1 x 1 unit taps
    ("n512", 3, 5),
    ("n256", 2, 7),           # the SKA station (3 x 3 Gaussian taps) on a 256^2 grid
    ("n256_cplx", 1, 4),      # random complex taps, random anchors over a 100 x 120 box
])
def test_large_grid_tensor_cores_match_oracle(hai, ctx, case, C, T):
    """FP16 tensor-core path of the large grids (gridding, stage-1 GEMM into
    an HBM operand, stage-2 GEMM with the squaring) against the oracle."""
    if case == "n512":
        cfg, pos, anchors, taps = _dense()
        n = 512
    elif case == "n256":
        pos, anchors, taps = station(I.SKA_LOW_STATION_256)
        n = 256
    else:
        rng = np.random.default_rng(3)
        n, ne, k = 256, 150, 3
        anchors = np.stack([rng.integers(40, 138, ne), rng.integers(30, 148, ne)], axis=1).astype(np.int32)
        taps = rng.standard_normal((ne, k, k, 2)).astype(np.float32)
        pos = anchors
    volt = I.random_voltages((C, T, 2, len(anchors), 2), seed=C * 7 + T)
    got = run_epic(hai, ctx, anchors, taps, n, volt, hai.HAI_PREC_FP16)
    want = O.epic_image(n, anchors, taps, volt.numpy())
    assert rel_err_planes(got, want).max() < REDUCED_TOL
    # accumulate onto the first result
    lay = hai.hai_layout_create(ctx, anchors, taps, n, 2)
    img = torch.from_numpy(got).cuda()
    hai.hai_epic_image(ctx, lay, volt.cuda(), C, T, hai.HAI_PREC_FP16, img, 1)
    hai.hai_sync(ctx)
    assert rel_err_planes(img.cpu().numpy(), 2 * want).max() < REDUCED_TOL
    hai.hai_layout_destroy(lay)


def test_large_grid_tensor_cores_full_dense_cadence_sampled_channel(hai, ctx):
    """The dense all-sky lattice's full cadence (16 channels x 100 samples,
    two scratch batches) in one call; the oracle recomputes two channels,
    one of them split across the batches."""
    cfg, pos, anchors, taps = _dense()
    volt = I.station_voltages(cfg, pos, device="cuda")
    n, C, T = cfg.grid_n, cfg.n_chan, cfg.n_time
    lay = hai.hai_layout_create(ctx, anchors, taps, n, 2)
    img = torch.empty((C, 4, n, n), device="cuda")
    hai.hai_epic_image(ctx, lay, volt, C, T, hai.HAI_PREC_FP16, img, 0)
    hai.hai_sync(ctx)
    for c in (0, 8):
        want = O.epic_image(n, anchors, taps, volt[c:c + 1].cpu().numpy())
        assert rel_err_planes(img[c:c + 1].cpu().numpy(), want).max() < REDUCED_TOL, c
    hai.hai_layout_destroy(lay)


def test_large_grid_fp16_tall_box_is_reported_unsupported(hai, ctx):
    """Boxes taller than 128 cells at N = 512 keep to the FP32 path."""
    anchors = np.array([[10, 10], [40, 200]], np.int32)
    taps = np.ones((2, 1, 1, 2), np.float32)
    lay = hai.hai_layout_create(ctx, anchors, taps, 512, 2)
    volt = torch.zeros((1, 2, 2, 2, 2), dtype=torch.int8, device="cuda")
    img = torch.zeros((1, 4, 512, 512), device="cuda")
    with pytest.raises(hai.HaiError) as e:
        hai.hai_epic_image(ctx, lay, volt, 1, 2, hai.HAI_PREC_FP16, img, 0)
    assert e.value.status == 4
    hai.hai_layout_destroy(lay)


# ------------------------------------------------------------------ FP16 split hi/lo
@pytest.mark.parametrize("n_elem,C,T,cplx", [(256, 3, 40, False), (256, 2, 301, True), (50, 5, 9, False),
                                              (300, 1, 1, True)])
def test_tc_split_recovers_fp32_accuracy(hai, ctx, n_elem, C, T, cplx):
    """Every operand as hi + lo fp16 and the products hi*hi + hi*lo + lo*hi:
    the images meet the FP32 bound and are far closer to the oracle than the
    plain FP16 path's."""
    if n_elem == 256:
        sc = I.SKA_LOW_STATION_256
    else:
        sc = I.uneven_station(I.UnevenConfig(), 0, n_elem)
    pos, anchors, taps = station(sc)
    if cplx:
        taps = taps.copy()
        taps[..., 1] = 0.3 * np.random.default_rng(n_elem).standard_normal(taps.shape[:-1]).astype(np.float32)
    volt = I.station_voltages(sc, pos, n_chan=C, n_time=T) if not cplx else \
        I.random_voltages((C, T, 2, len(pos), 2), seed=C + T)
    want = O.epic_image(sc.grid_n, anchors, taps, volt.numpy())
    split = run_epic(hai, ctx, anchors, taps, sc.grid_n, volt, hai.HAI_PREC_FP16_SPLIT)
    plain = run_epic(hai, ctx, anchors, taps, sc.grid_n, volt, hai.HAI_PREC_FP16)
    e_split, e_plain = rel_err_planes(split, want).max(), rel_err_planes(plain, want).max()
    assert e_split < FP32_TOL, e_split
    assert e_split < e_plain / 20, (e_split, e_plain)


def test_tc_box_wider_than_half_grid_at_128_is_refused(hai, ctx):
    """Every tensor-core precision needs the kernel box within N/2 x N/2
    cells; a 93-cell box at N = 128 is refused (FP32 still images it)."""
    anchors = np.array([[10, 10], [100, 100], [60, 20]], np.int32)
    taps = np.zeros((3, 3, 3, 2), np.float32)
    taps[:, 1, 1, 0] = 1.0
    lay = hai.hai_layout_create(ctx, anchors, taps, 128, 2)
    try:
        volt = I.random_voltages((1, 2, 2, 3, 2), seed=23, device="cuda")
        img = torch.zeros((1, 4, 128, 128), device="cuda")
        for prec in (hai.HAI_PREC_FP16, hai.HAI_PREC_BF16, hai.HAI_PREC_FP16_SPLIT, hai.HAI_PREC_BF16_SPLIT):
            with pytest.raises(hai.HaiError) as e:
                hai.hai_epic_image(ctx, lay, volt, 1, 2, prec, img, 0)
            assert e.value.status == 4
        hai.hai_epic_image(ctx, lay, volt, 1, 2, hai.HAI_PREC_FP32, img, 0)
        hai.hai_sync(ctx)
        want = O.epic_image(128, anchors, taps, volt.cpu().numpy())
        assert rel_err_planes(img.cpu().numpy(), want).max() < FP32_TOL
    finally:
        hai.hai_layout_destroy(lay)


def test_misaligned_buffers_are_refused(hai, ctx):
    """A voltage pointer on an odd byte (half a complex value) or an image
    pointer off 4 bytes is refused before any launch."""
    cfg = I.SKA_LOW_STATION_256
    pos, anchors, taps = station(cfg)
    lay = hai.hai_layout_create(ctx, anchors, taps, cfg.grid_n, 2)
    try:
        ne, n = len(pos), cfg.grid_n
        raw = torch.zeros(2 * 2 * ne * 2 + 16, dtype=torch.int8, device="cuda")
        img = torch.zeros((1, 4, n, n), device="cuda")
        L = hai.load()
        for prec in (hai.HAI_PREC_FP32, hai.HAI_PREC_FP16):
            rc = L.hai_epic_image(ctx, lay.handle, raw.data_ptr() + 1, 1, 2, prec, img.data_ptr(), 0, None)
            assert rc == 1 and "aligned" in hai.hai_last_error()
            rc = L.hai_epic_image(ctx, lay.handle, raw.data_ptr(), 1, 2, prec, img.data_ptr() + 2, 0, None)
            assert rc == 1
        vis = torch.zeros((1, ne * (ne + 1) // 2, 2, 2, 2), dtype=torch.int32, device="cuda")
        rc = L.hai_correlate(ctx, raw.data_ptr() + 1, 1, 2, ne, 2, vis.data_ptr(), 0, None)
        assert rc == 1 and "aligned" in hai.hai_last_error()
    finally:
        hai.hai_layout_destroy(lay)
