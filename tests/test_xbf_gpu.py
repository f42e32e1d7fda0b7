"""GPU parity of the inter-station XBF (direct DFT of station visibilities as
one tensor-core GEMM against FP64-built geometry phases) with the oracle,
through the C ABI: all pairs, the pairs the XFFT grid drops, the
XFFT + XBF hybrid image, and the hierarchical array at full grid size."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import FP32_TOL, REDUCED_TOL, SPLIT_PIXEL_TOL, frob_err_planes, pixel_err_planes, rel_err_planes

pytestmark = pytest.mark.gpu
H = I.HierarchyConfig()


@pytest.fixture(scope="module")
def ctx(hai):
    c = hai.hai_create(0)
    yield c
    hai.hai_destroy(c)


def planes(img_pq):
    """[K][C][P][P][n][n] complex -> [K*C][4][n][n]: XX, YY, Re XY, Im XY."""
    K, C = img_pq.shape[:2]
    x = img_pq.reshape(K * C, 2, 2, *img_pq.shape[-2:])
    return np.stack([x[:, 0, 0].real, x[:, 1, 1].real, x[:, 0, 1].real, x[:, 0, 1].imag], axis=1)


def hermitian_vis(rng, K, C, S, lo=-2**20, hi=2**20):
    vis = rng.integers(lo, hi, (K, C, S * (S + 1) // 2, 2, 2, 2)).astype(np.int32)
    for m in range(S):
        bl = m * (m + 1) // 2 + m
        vis[..., bl, 0, 0, 1] = 0
        vis[..., bl, 1, 1, 1] = 0
        vis[..., bl, 1, 0, 0] = vis[..., bl, 0, 1, 0]
        vis[..., bl, 1, 0, 1] = -vis[..., bl, 0, 1, 1]
    return vis


def run_xbf(hai, ctx, pos, lam, cell, n, dirs, vis, pair_set, img=None, accumulate=0, prec=None):
    K, C = vis.shape[:2]
    prec = hai.HAI_PREC_FP16 if prec is None else prec
    lay = hai.hai_xbf_layout_create(ctx, pos, lam, cell, n, dirs, pair_set, C, prec)
    if img is None:
        img = torch.full((K * C, 4, n, n), float("nan"), device="cuda")
    hai.hai_xbf_station_image(ctx, lay, torch.from_numpy(vis).cuda(), C, img, accumulate)
    hai.hai_sync(ctx)
    info = hai.hai_xbf_layout_info(lay)
    hai.hai_xbf_layout_destroy(lay)
    return img.cpu().numpy(), info


@pytest.mark.parametrize("S,K,C,n", [(12, 2, 2, 32), (5, 1, 3, 16), (40, 3, 1, 64)])
def test_all_pairs_match_oracle(hai, ctx, S, K, C, n):
    rng = np.random.default_rng(S * n)
    cell, lam = 19.0, 3.0
    pos = rng.uniform(-n * cell / 3, n * cell / 3, (S, 2))
    dirs = rng.uniform(-0.1, 0.1, (K, 2))
    vis = hermitian_vis(rng, K, C, S)
    got, (npairs, _) = run_xbf(hai, ctx, pos, lam, cell, n, dirs, vis, hai.HAI_XBF_ALL_PAIRS)
    assert npairs == S * (S + 1) // 2
    want = O.station_xbf(n, pos, lam, cell, dirs, vis.astype(np.int64))
    assert rel_err_planes(got, planes(want)).max() < REDUCED_TOL


def test_offgrid_pairs_and_the_hybrid_image(hai, ctx):
    """A core plus a 4-station tail: XBF over the dropped pairs matches the
    oracle, and XFFT then XBF with accumulate = 1 gives the image of every
    pair (XFFT part gridded, XBF part exact), against the oracle's sum."""
    rng = np.random.default_rng(7)
    S, K, C, n, cell, lam = 24, 2, 2, 32, 19.0, 3.0
    pos = rng.uniform(-n * cell / 6, n * cell / 6, (S, 2))
    pos[-4:] = rng.uniform(2 * n * cell, 6 * n * cell, (4, 2))
    dirs = rng.uniform(-0.05, 0.05, (K, 2))
    vis = hermitian_vis(rng, K, C, S)
    part, (npairs, _) = run_xbf(hai, ctx, pos, lam, cell, n, dirs, vis, hai.HAI_XBF_OFFGRID_PAIRS)
    want_part = O.station_xbf(n, pos, lam, cell, dirs, vis.astype(np.int64), offgrid_only=True)
    assert rel_err_planes(part, planes(want_part)).max() < REDUCED_TOL
    want_xfft, dropped = O.station_xfft(n, pos, lam, cell, dirs, vis.astype(np.int64))
    assert npairs == dropped >= 4 * (S - 4)
    vl = hai.hai_vis_layout_create(ctx, pos, lam, cell, n, dirs)
    img = torch.empty((K * C, 4, n, n), device="cuda")
    hai.hai_xfft_station_image(ctx, vl, torch.from_numpy(vis).cuda(), C, img)
    hai.hai_sync(ctx)
    hai.hai_vis_layout_destroy(vl)
    hyb, _ = run_xbf(hai, ctx, pos, lam, cell, n, dirs, vis, hai.HAI_XBF_OFFGRID_PAIRS, img=img, accumulate=1)
    assert rel_err_planes(hyb, planes(want_xfft + want_part)).max() < REDUCED_TOL


def test_hierarchical_array_full_grid(hai, ctx):
    """The hierarchical array (256 stations, 19 m cell, 256^2 grid): the
    pairs the station grid drops (the 65 km tail), one beam, one channel, in
    the benchmark's configuration, against the oracle's direct sum."""
    centres = I.station_centres(H)
    S, n = len(centres), H.grid_n
    dirs = I.beam_directions(H.n_beam, H.station.lam_m, H.station.diameter_m)[5:6]
    vis = hermitian_vis(np.random.default_rng(11), 1, 1, S, -2**24, 2**24)
    got, (npairs, nbytes) = run_xbf(hai, ctx, centres, H.station.lam_m, H.cell_m, n, dirs, vis,
                                    hai.HAI_XBF_OFFGRID_PAIRS)
    want = O.station_xbf(n, centres, H.station.lam_m, H.cell_m, dirs, vis.astype(np.int64), offgrid_only=True)
    assert npairs > 5000 and nbytes > npairs * 4 * n * n
    assert rel_err_planes(got, planes(want)).max() < REDUCED_TOL


@pytest.mark.parametrize("S,K,C,n,offgrid", [(12, 2, 2, 32, False), (40, 1, 2, 64, False), (24, 2, 1, 32, True)])
def test_split_products_reach_fp32_accuracy(hai, ctx, S, K, C, n, offgrid):
    """HAI_PREC_FP16_SPLIT (hi*hi + hi*lo + lo*hi through the same GEMM):
    FP32-level image error, far below the plain fp16 one."""
    rng = np.random.default_rng(S + n)
    cell, lam = 19.0, 3.0
    pos = rng.uniform(-n * cell / 3, n * cell / 3, (S, 2))
    if offgrid:
        pos[-4:] = rng.uniform(2 * n * cell, 6 * n * cell, (4, 2))
    dirs = rng.uniform(-0.1, 0.1, (K, 2))
    vis = hermitian_vis(rng, K, C, S)
    ps = hai.HAI_XBF_OFFGRID_PAIRS if offgrid else hai.HAI_XBF_ALL_PAIRS
    want = planes(O.station_xbf(n, pos, lam, cell, dirs, vis.astype(np.int64), offgrid_only=offgrid))
    split, (_, nbytes) = run_xbf(hai, ctx, pos, lam, cell, n, dirs, vis, ps, prec=hai.HAI_PREC_FP16_SPLIT)
    plain, (_, nbytes1) = run_xbf(hai, ctx, pos, lam, cell, n, dirs, vis, ps)
    e_split, e_plain = rel_err_planes(split, want).max(), rel_err_planes(plain, want).max()
    assert frob_err_planes(split, want).max() < FP32_TOL
    assert pixel_err_planes(split, want).max() < SPLIT_PIXEL_TOL, e_split
    assert e_split < e_plain / 20, (e_split, e_plain)
    assert nbytes > 2.5 * nbytes1


def test_no_pairs_and_bad_arguments(hai, ctx):
    pos = np.array([[0.0, 0.0], [10.0, 5.0], [-7.0, 3.0]])
    vis = hermitian_vis(np.random.default_rng(1), 1, 1, 3)
    # every pair on the grid: the off-grid set is empty and the image zero
    got, (npairs, _) = run_xbf(hai, ctx, pos, 3.0, 19.0, 32, None, vis, hai.HAI_XBF_OFFGRID_PAIRS)
    assert npairs == 0 and np.all(got == 0.0)
    with pytest.raises(hai.HaiError) as e:
        hai.hai_xbf_layout_create(ctx, pos, 3.0, 19.0, 48, None, 0, 1)
    assert e.value.status == 1
    with pytest.raises(hai.HaiError) as e:
        hai.hai_xbf_layout_create(ctx, pos, 3.0, 19.0, 32, None, 0, 1, hai.HAI_PREC_FP32)
    assert e.value.status == 4
    lay = hai.hai_xbf_layout_create(ctx, pos, 3.0, 19.0, 32, None, 0, 1)
    img = torch.zeros((2, 4, 32, 32), device="cuda")
    with pytest.raises(hai.HaiError) as e:       # more channels than the layout holds
        hai.hai_xbf_station_image(ctx, lay, torch.zeros((2 * 6 * 8,), dtype=torch.int32, device="cuda"), 2, img)
    assert e.value.status == 1
    hai.hai_xbf_layout_destroy(lay)
