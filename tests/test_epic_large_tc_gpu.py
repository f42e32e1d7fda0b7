"""Tensor-core EPIC on the large grids (N = 256, 512, and 128) in every
operand form: FP16, BF16 and their hi/lo splits, against the FP64 oracle.

The dense all-sky lattice (128 x 128 elements at 0.5 lambda on a 512^2 grid,
1 x 1 unit taps) and the SKA-shaped station on a 256^2 grid.  The cases cover
several sample batches per call, channel chunks (more channels than the batch
scratch holds pairs), (item, sample) ranges that split items between CTAs
(the partial tiles and their fixup), accumulate, determinism and the full
cadence of 10^4 samples on a sampled channel."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import (BF16_SPLIT_TOL, BF16_TOL, FP32_TOL, REDUCED_TOL, SPLIT_PIXEL_TOL, frob_err_planes,
                           pixel_err_planes, rel_err_planes, station)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(hai):
    c = hai.hai_create(0)
    yield c
    hai.hai_destroy(c)


def dense():
    cfg = I.DENSE_ALLSKY_16384
    pos, anchors, taps = station(cfg)
    return cfg, pos, anchors, taps


def check(hai, prec, got, want):
    """Each precision against the oracle at its bound (helpers: derivations)."""
    if prec == hai.HAI_PREC_FP16:
        assert rel_err_planes(got, want).max() < REDUCED_TOL
    elif prec == hai.HAI_PREC_BF16:
        assert rel_err_planes(got, want).max() < BF16_TOL
    elif prec == hai.HAI_PREC_FP16_SPLIT:
        assert frob_err_planes(got, want).max() < FP32_TOL
        assert pixel_err_planes(got, want).max() < SPLIT_PIXEL_TOL
    elif prec == hai.HAI_PREC_BF16_SPLIT:
        assert rel_err_planes(got, want).max() < BF16_SPLIT_TOL
    else:
        assert rel_err_planes(got, want).max() < FP32_TOL


def image(hai, ctx, lay, volt, C, T, prec, n, img=None, accumulate=0):
    if img is None:
        img = torch.full((C, 4, n, n), float("nan"), device="cuda")
    hai.hai_epic_image(ctx, lay, volt, C, T, prec, img, accumulate)
    hai.hai_sync(ctx)
    return img


PRECS = ["FP16", "BF16", "FP16_SPLIT", "BF16_SPLIT"]


@pytest.mark.parametrize("pname", PRECS)
@pytest.mark.parametrize("case,C,T", [
    ("n512", 2, 3),           # 64 items x 3 samples on 152 CTAs: items split between CTAs
    ("n512", 3, 40),
    ("n256", 2, 7),           # the SKA station (3 x 3 Gaussian taps) on a 256^2 grid
    ("n256_cplx", 1, 4),      # random complex taps, random anchors over a 100 x 120 box
])
def test_every_operand_form_matches_oracle(hai, ctx, pname, case, C, T):
    prec = getattr(hai, f"HAI_PREC_{pname}")
    if case == "n512":
        _, pos, anchors, taps = dense()
        n = 512
    elif case == "n256":
        pos, anchors, taps = station(I.SKA_LOW_STATION_256)
        n = 256
    else:
        rng = np.random.default_rng(3)
        n, ne, k = 256, 150, 3
        anchors = np.stack([rng.integers(40, 138, ne), rng.integers(30, 148, ne)], axis=1).astype(np.int32)
        taps = rng.standard_normal((ne, k, k, 2)).astype(np.float32)
    volt = I.random_voltages((C, T, 2, len(anchors), 2), seed=C * 7 + T)
    want = O.epic_image(n, anchors, taps, volt.numpy())
    lay = hai.hai_layout_create(ctx, anchors, taps, n, 2)
    try:
        img = image(hai, ctx, lay, volt.cuda(), C, T, prec, n)
        got = img.cpu().numpy()
        check(hai, prec, got, want)
        # accumulate onto the first result
        image(hai, ctx, lay, volt.cuda(), C, T, prec, n, img, 1)
        check(hai, prec, img.cpu().numpy(), 2 * want)
    finally:
        hai.hai_layout_destroy(lay)


@pytest.mark.parametrize("pname", ["FP16", "BF16_SPLIT"])
def test_many_channels_go_in_chunks(hai, ctx, pname):
    """More channels than the batch scratch holds (channel, sample) pairs (819
    plain, 409 split at 512^2): the channels go in chunks; sampled channels on
    both sides of every chunk boundary against the oracle."""
    prec = getattr(hai, f"HAI_PREC_{pname}")
    _, pos, anchors, taps = dense()
    C, T, n = 830, 1, 512
    volt = I.random_voltages((C, T, 2, len(pos), 2), seed=11, device="cuda")
    lay = hai.hai_layout_create(ctx, anchors, taps, n, 2)
    try:
        img = image(hai, ctx, lay, volt, C, T, prec, n)
        for c in (0, 408, 409, 818, 819, 829):
            want = O.epic_image(n, anchors, taps, volt[c:c + 1].cpu().numpy())
            check(hai, prec, img[c:c + 1].cpu().numpy(), want)
    finally:
        hai.hai_layout_destroy(lay)


def test_results_are_bit_identical_on_repeat(hai, ctx):
    """Partial tiles are added in a fixed CTA order: repeated calls agree to
    the bit."""
    _, pos, anchors, taps = dense()
    volt = I.random_voltages((3, 17, 2, len(pos), 2), seed=5, device="cuda")
    lay = hai.hai_layout_create(ctx, anchors, taps, 512, 2)
    try:
        for prec in (hai.HAI_PREC_FP16, hai.HAI_PREC_BF16_SPLIT):
            a = image(hai, ctx, lay, volt, 3, 17, prec, 512).cpu()
            b = image(hai, ctx, lay, volt, 3, 17, prec, 512).cpu()
            assert torch.equal(a, b)
    finally:
        hai.hai_layout_destroy(lay)


@pytest.fixture(scope="module")
def long_cadence(hai):
    """The dense all-sky lattice over a cadence of 10^4 samples (the longest of
    the workload), one sampled channel of the seeded sky: voltages and the
    oracle's image (FP64, all host cores)."""
    cfg, pos, anchors, taps = dense()
    volt = I.station_voltages(cfg, pos, device="cuda", n_chan=1, n_time=10000, chan0=5)
    want = O.epic_image(cfg.grid_n, anchors, taps, volt.cpu().numpy())
    return cfg, anchors, taps, volt, want


@pytest.mark.parametrize("pname", ["FP32", "FP16", "FP16_SPLIT", "BF16_SPLIT", "BF16"])
def test_long_cadence_of_ten_thousand_samples(hai, ctx, long_cadence, pname):
    """T = 10^4: FP32 accumulation over the whole cadence stays within each
    path's bound (the FP32 path <= 1e-5, the reduced-precision ones within
    theirs)."""
    cfg, anchors, taps, volt, want = long_cadence
    prec = getattr(hai, f"HAI_PREC_{pname}")
    lay = hai.hai_layout_create(ctx, anchors, taps, cfg.grid_n, 2)
    try:
        img = image(hai, ctx, lay, volt, 1, 10000, prec, cfg.grid_n)
        check(hai, prec, img.cpu().numpy(), want)
    finally:
        hai.hai_layout_destroy(lay)


# ------------------------------------------------------------------ N = 32, 64
@pytest.mark.parametrize("pname", ["BF16", "BF16_SPLIT", "FP16_SPLIT", "FP16"])
@pytest.mark.parametrize("n_elem,C,T,cplx", [(256, 3, 40, False), (256, 2, 301, True), (50, 5, 9, False),
                                              (300, 1, 1, True)])
def test_small_grids_every_operand_form(hai, ctx, pname, n_elem, C, T, cplx):
    """The N = 32 / 64 tensor-core kernel with FP16 or BF16 operands, plain or
    split, against the oracle at each form's bound; the SKA station (64^2)
    and stations of the uneven array (32^2), real and complex taps."""
    prec = getattr(hai, f"HAI_PREC_{pname}")
    sc = I.SKA_LOW_STATION_256 if n_elem == 256 else I.uneven_station(I.UnevenConfig(), 0, n_elem)
    pos, anchors, taps = station(sc)
    if cplx:
        taps = taps.copy()
        taps[..., 1] = 0.3 * np.random.default_rng(n_elem).standard_normal(taps.shape[:-1]).astype(np.float32)
    volt = I.station_voltages(sc, pos, n_chan=C, n_time=T) if not cplx else \
        I.random_voltages((C, T, 2, len(pos), 2), seed=C + T)
    want = O.epic_image(sc.grid_n, anchors, taps, volt.numpy())
    lay = hai.hai_layout_create(ctx, anchors, taps, sc.grid_n, 2)
    try:
        img = image(hai, ctx, lay, volt.cuda(), C, T, prec, sc.grid_n)
        check(hai, prec, img.cpu().numpy(), want)
        image(hai, ctx, lay, volt.cuda(), C, T, prec, sc.grid_n, img, 1)
        check(hai, prec, img.cpu().numpy(), 2 * want)
    finally:
        hai.hai_layout_destroy(lay)


def test_every_form_at_128(hai, ctx):
    """N = 128: FP16 and BF16 on the 4-CTA cluster kernel, the two splits on
    the large-grid kernels (64 MB scratch: 170 split (channel, sample) pairs
    per batch, so 3 x 70 samples take two batches), each against the oracle
    at its bound, and accumulate."""
    sc = I.uneven_station(I.UnevenConfig(), 0, 700)
    pos, anchors, taps = station(sc)
    lay = hai.hai_layout_create(ctx, anchors, taps, 128, 2)
    try:
        C, T = 3, 70
        volt = I.random_voltages((C, T, 2, len(pos), 2), seed=17)
        want = O.epic_image(128, anchors, taps, volt.numpy())
        for pname in PRECS:
            prec = getattr(hai, f"HAI_PREC_{pname}")
            img = image(hai, ctx, lay, volt.cuda(), C, T, prec, 128)
            check(hai, prec, img.cpu().numpy(), want)
            if "SPLIT" in pname:
                image(hai, ctx, lay, volt.cuda(), C, T, prec, 128, img, 1)
                check(hai, prec, img.cpu().numpy(), 2 * want)
    finally:
        hai.hai_layout_destroy(lay)


def test_split_at_128_channel_chunks(hai, ctx):
    """More channels than a split batch at N = 128 holds pairs (170): sampled
    channels on both sides of the chunk boundary against the oracle."""
    sc = I.uneven_station(I.UnevenConfig(), 0, 700)
    pos, anchors, taps = station(sc)
    lay = hai.hai_layout_create(ctx, anchors, taps, 128, 2)
    try:
        C = 180
        volt = I.random_voltages((C, 1, 2, len(pos), 2), seed=19, device="cuda")
        img = image(hai, ctx, lay, volt, C, 1, hai.HAI_PREC_FP16_SPLIT, 128)
        for c in (0, 169, 170, 179):
            want = O.epic_image(128, anchors, taps, volt[c:c + 1].cpu().numpy())
            check(hai, hai.HAI_PREC_FP16_SPLIT, img[c:c + 1].cpu().numpy(), want)
    finally:
        hai.hai_layout_destroy(lay)


def test_autotune_choice_cache_and_parity(hai, ctx, tmp_path):
    """hai_autotune picks the channels per chunk of the large-grid tensor path
    by timing, writes it to the cache, applies a cached choice without
    timing, and the tuned layout still matches the oracle."""
    _, pos, anchors, taps = dense()
    lay = hai.hai_layout_create(ctx, anchors, taps, 512, 2)
    cache = str(tmp_path / "tune.txt")
    try:
        c1 = hai.hai_autotune(ctx, lay, 16, 200, hai.HAI_PREC_FP16, cache)
        assert c1 in (1, 2, 4, 8, 16)
        text = open(cache).read()
        assert f"| chunk {c1} |" in text and " N512 " in text
        # a cached line is applied as written (here a different, valid choice)
        key = text.split(" | ")[0]
        with open(cache, "a") as f:
            f.write(f"{key} | chunk 3 | 0 ms\n")
        assert hai.hai_autotune(ctx, lay, 16, 200, hai.HAI_PREC_FP16, cache) == 3
        volt = I.random_voltages((5, 30, 2, len(pos), 2), seed=9, device="cuda")
        img = image(hai, ctx, lay, volt, 5, 30, hai.HAI_PREC_FP16, 512)
        want = O.epic_image(512, anchors, taps, volt.cpu().numpy())
        check(hai, hai.HAI_PREC_FP16, img.cpu().numpy(), want)
        assert hai.hai_autotune(ctx, lay, 16, 200, hai.HAI_PREC_FP32, cache) == 0
    finally:
        hai.hai_layout_destroy(lay)
