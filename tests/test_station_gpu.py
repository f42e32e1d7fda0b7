"""GPU parity of the inter-station stage of the hierarchical array: beams to
correlator layout (bit-exact), the inter-station XFFT with FP64 steering
against the oracle, and the whole chain beamformer -> requantise -> station
correlator -> steered XFFT against the oracle chain."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import FP32_TOL, rel_err_planes

pytestmark = pytest.mark.gpu
H = I.HierarchyConfig()


@pytest.fixture(scope="module")
def ctx(hai):
    c = hai.hai_create(0)
    yield c
    hai.hai_destroy(c)


def planes(img_pq):
    """[K][C][P][P][n][n] complex -> [K*C][4][n][n] planes XX, YY, Re XY, Im XY."""
    K, C = img_pq.shape[:2]
    x = img_pq.reshape(K * C, 2, 2, *img_pq.shape[-2:])
    return np.stack([x[:, 0, 0].real, x[:, 1, 1].real, x[:, 0, 1].real, x[:, 0, 1].imag], axis=1)


@pytest.mark.parametrize("S,C,T,K,P", [(5, 2, 3, 4, 2), (37, 1, 9, 16, 2), (256, 2, 2, 16, 2), (3, 3, 1, 1, 1)])
def test_beams_to_corr_is_the_transpose(hai, ctx, S, C, T, K, P):
    beams = I.random_voltages((S, C, T, K, P, 2), seed=S + T)
    out = torch.full((K, C, T, P, S, 2), 99, dtype=torch.int8, device="cuda")
    hai.hai_beams_to_corr(ctx, beams.cuda(), S, C, T, K, P, out)
    torch.cuda.synchronize()
    assert torch.equal(out.cpu(), beams.permute(3, 1, 2, 4, 0, 5).contiguous())


def hermitian_autos(vis, S):
    """Make the autos what a correlator gives: XX, YY real, YX = conj(XY)."""
    for m in range(S):
        bl = m * (m + 1) // 2 + m
        vis[..., bl, 0, 0, 1] = 0
        vis[..., bl, 1, 1, 1] = 0
        vis[..., bl, 1, 0, 0] = vis[..., bl, 0, 1, 0]
        vis[..., bl, 1, 0, 1] = -vis[..., bl, 0, 1, 1]
    return vis


def station_case(S, n, cell, seed, tail=0):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-n * cell / 5, n * cell / 5, (S, 2))
    if tail:
        pos[-tail:] = rng.uniform(4 * n * cell, 9 * n * cell, (tail, 2))
    return pos


@pytest.mark.parametrize("S,K,C,n,tail", [(12, 2, 3, 32, 0), (30, 3, 2, 64, 4), (9, 1, 1, 16, 2), (40, 2, 2, 256, 0)])
def test_station_xfft_matches_oracle(hai, ctx, S, K, C, n, tail):
    """The last case's uv window (~200 cells) takes two gridding tiles per
    axis, the last one narrower than the first."""
    cell, lam = 19.0, 3.0
    pos = station_case(S, n, cell, S * n, tail)
    dirs = np.random.default_rng(K).uniform(-0.1, 0.1, (K, 2))
    nbl = S * (S + 1) // 2
    vis = np.random.default_rng(C).integers(-2**20, 2**20, (K, C, nbl, 2, 2, 2)).astype(np.int32)
    vis = hermitian_autos(vis, S)
    lay = hai.hai_vis_layout_create(ctx, pos, lam, cell, n, dirs)
    img = torch.full((K * C, 4, n, n), float("nan"), device="cuda")
    hai.hai_xfft_station_image(ctx, lay, torch.from_numpy(vis).cuda(), C, img)
    hai.hai_sync(ctx)
    want, dropped = O.station_xfft(n, pos, lam, cell, dirs, vis.astype(np.int64))
    assert hai.hai_vis_layout_offgrid(lay) == dropped
    if tail:
        assert dropped > 0
    assert rel_err_planes(img.cpu().numpy(), planes(want)).max() < FP32_TOL
    hai.hai_vis_layout_destroy(lay)


def test_station_xfft_long_baselines_need_fp64_phase(hai, ctx):
    """Stations 20-65 km out on whole cells of a coarse grid: the steering
    phase reaches ~10^5 rad; the FP64 phase keeps the images at FP32
    accuracy (an FP32 phase would be off by ~10^-2 rad per pair)."""
    lam, n = 3.0, 32
    cell = 4000.0
    rng = np.random.default_rng(3)
    cells = rng.integers(-3, 4, (10, 2)) + np.array([12, 0])
    pos = cells * cell + rng.uniform(-0.4, 0.4, (10, 2)) * cell
    dirs = np.array([[0.0137, -0.0091], [0.05, 0.02]])
    nbl = 10 * 11 // 2
    vis = hermitian_autos(rng.integers(-1000, 1000, (2, 1, nbl, 2, 2, 2)).astype(np.int32), 10)
    lay = hai.hai_vis_layout_create(ctx, pos, lam, cell, n, dirs)
    img = torch.empty((2, 4, n, n), device="cuda")
    hai.hai_xfft_station_image(ctx, lay, torch.from_numpy(vis).cuda(), 1, img)
    hai.hai_sync(ctx)
    want, _ = O.station_xfft(n, pos, lam, cell, dirs, vis.astype(np.int64))
    assert np.abs(pos).max() > 2e4
    assert rel_err_planes(img.cpu().numpy(), planes(want)).max() < FP32_TOL
    hai.hai_vis_layout_destroy(lay)


def run_chain(hai, ctx, volt, w, S, C, T, K, P, ne, shift, lay):
    """beamformer (requantised) -> beams_to_corr -> correlator -> steered XFFT."""
    beams = torch.empty((S, C, T, K, P, 2), dtype=torch.int8, device="cuda")
    sat = torch.zeros(1, dtype=torch.int64, device="cuda")
    hai.hai_beamform(ctx, volt, w, S, C, T, K, ne, P, shift, beams, sat)
    cin = torch.empty((K, C, T, P, S, 2), dtype=torch.int8, device="cuda")
    hai.hai_beams_to_corr(ctx, beams, S, C, T, K, P, cin)
    vis = torch.empty((K * C, S * (S + 1) // 2, P, P, 2), dtype=torch.int32, device="cuda")
    hai.hai_correlate(ctx, cin.view(K * C, T, P, S, 2), K * C, T, S, P, vis, 0)
    img = torch.empty((K * C, 4, H.grid_n, H.grid_n), device="cuda")
    hai.hai_xfft_station_image(ctx, lay, vis, C, img)
    hai.hai_sync(ctx)
    return beams, sat, vis, img


def test_hierarchical_chain_matches_oracle_chain(hai, ctx):
    """A reduced hierarchical array (24 stations of 64 elements from the
    seeded station layout and array layout, 16 beams, 2 channels, 48 samples)
    through the whole GPU chain; every stage against the oracle chain."""
    S, C, T, K, P = 24, 2, 48, 16, 2
    st = I.StationConfig(name="st64", n_elem=64, diameter_m=19.0, min_spacing_m=1.5, lam_m=3.0, n_chan=C,
                         n_pol=P, n_time=T, grid_n=32, cell_lambda=0.5, ksize=3, seed=I.SEED0 + 9)
    elem = I.station_layout(st)
    centres = I.station_centres(H)[:S]
    dirs = I.beam_directions(K, st.lam_m, st.diameter_m)
    rng = np.random.default_rng(H.seed)
    src = np.vstack([dirs[:2] + 0.01, rng.uniform(-0.05, 0.05, (3, 2))])
    flux = np.array([1.0, 0.8, 0.5, 0.3, 0.2])
    volt = I.hierarchy_voltages(H, centres, elem, src, flux, S, C, T, device="cuda")
    w1 = I.bf_weights(elem, st.lam_m, dirs, P)
    w = torch.from_numpy(np.repeat(w1[None], S, axis=0)).cuda()
    shift = 9
    lay = hai.hai_vis_layout_create(ctx, centres, st.lam_m, H.cell_m, H.grid_n, dirs)
    beams, sat, vis, img = run_chain(hai, ctx, volt, w, S, C, T, K, P, len(elem), shift, lay)
    # integer stages bit-exact
    b64 = O.beamform(volt.cpu().numpy(), w.cpu().numpy())
    bq, nsat = O.requant(b64, shift)
    assert np.array_equal(beams.cpu().numpy(), bq) and sat.item() == nsat
    cin = np.ascontiguousarray(bq.transpose(3, 1, 2, 4, 0, 5)).reshape(K * C, T, P, S, 2)
    v64 = O.correlate(cin)
    assert np.array_equal(vis.cpu().numpy().astype(np.int64), v64)
    # steered inter-station images
    want, dropped = O.station_xfft(H.grid_n, centres, st.lam_m, H.cell_m, dirs,
                                   v64.reshape(K, C, *v64.shape[1:]))
    assert hai.hai_vis_layout_offgrid(lay) == dropped
    assert rel_err_planes(img.cpu().numpy(), planes(want)).max() < FP32_TOL
    hai.hai_vis_layout_destroy(lay)


def test_hierarchical_full_size_sampled(hai, ctx):
    """The hierarchical workload's full cadence (256 stations x 256 elements,
    32 channels, 2 pols, 1000 samples, 16 beams, 256^2 station grid) in the
    launch configuration of the benchmark, uniform int8 voltages; the oracle
    recomputes two stations' beams, two (beam, channel) correlations and two
    images."""
    S, C, T, K, P, ne = H.n_station, H.n_chan, H.n_time, H.n_beam, H.n_pol, H.station.n_elem
    g = torch.Generator(device="cuda").manual_seed(5)
    volt = torch.randint(-128, 128, (S, C, T, P, ne, 2), dtype=torch.int8, device="cuda", generator=g)
    elem = I.station_layout(H.station)
    centres = I.station_centres(H)
    dirs = I.beam_directions(K, H.station.lam_m, H.station.diameter_m)
    w1 = I.bf_weights(elem, H.station.lam_m, dirs, P)
    w = torch.from_numpy(np.repeat(w1[None], S, axis=0)).cuda()
    lay = hai.hai_vis_layout_create(ctx, centres, H.station.lam_m, H.cell_m, H.grid_n, dirs)
    beams, sat, vis, img = run_chain(hai, ctx, volt, w, S, C, T, K, P, ne, H.requant_shift, lay)
    del volt
    # beams of two stations (voltages regenerated from the same seed)
    g2 = torch.Generator(device="cuda").manual_seed(5)
    vfull = torch.randint(-128, 128, (S, C, T, P, ne, 2), dtype=torch.int8, device="cuda", generator=g2)
    for s in (0, 200):
        b64 = O.beamform(vfull[s:s + 1].cpu().numpy(), w[s:s + 1].cpu().numpy())
        bq, _ = O.requant(b64, H.requant_shift)
        assert np.array_equal(beams[s:s + 1].cpu().numpy(), bq)
    del vfull
    bcpu = beams.cpu().numpy()
    for kc in (0, 333):
        k, c = divmod(kc, C)
        cin = np.ascontiguousarray(bcpu[:, c, :, k].transpose(1, 2, 0, 3))[None]   # [1][T][P][S][2]
        v64 = O.correlate(cin)
        assert np.array_equal(vis[kc:kc + 1].cpu().numpy().astype(np.int64), v64)
        want, dropped = O.station_xfft(H.grid_n, centres, H.station.lam_m, H.cell_m, dirs[k:k + 1], v64[None])
        assert rel_err_planes(img[kc:kc + 1].cpu().numpy(), planes(want)).max() < FP32_TOL
        assert hai.hai_vis_layout_offgrid(lay) == dropped > 0
    hai.hai_vis_layout_destroy(lay)
