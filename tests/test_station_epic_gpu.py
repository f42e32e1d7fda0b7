"""GPU parity of the inter-station EPIC (station beams gridded at the station
positions with FP64 steering weights, then the EPIC kernels) against the
oracle, through the C ABI: the hierarchical array's geometry, both
precisions, and the chain beamformer -> requantise -> beams_to_corr ->
inter-station EPIC."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import FP32_TOL, REDUCED_TOL, rel_err_planes

pytestmark = pytest.mark.gpu
H = I.HierarchyConfig()
N_EPIC = 128          # padding 2 on the 1 km core at a 19 m cell


@pytest.fixture(scope="module")
def ctx(hai):
    c = hai.hai_create(0)
    yield c
    hai.hai_destroy(c)


def station_epic(hai, ctx, centres, lam, cell, n, dirs, cin, prec):
    """cin: device int8 [K][C][T][P][S][2].  Returns images [K][C][Q][n][n]
    and the stations dropped."""
    K, C, T, P, S = cin.shape[:5]
    out = torch.full((K, C, 4 if P == 2 else 1, n, n), float("nan"), device="cuda")
    dropped = None
    for k in range(K):
        lay, dropped = hai.hai_station_epic_layout_create(ctx, centres, lam, cell, n, dirs, k, P)
        hai.hai_epic_image(ctx, lay, cin[k].contiguous(), C, T, prec, out[k], 0)
        hai.hai_sync(ctx)
        hai.hai_layout_destroy(lay)
    return out.cpu().numpy(), dropped


@pytest.mark.parametrize("prec,tol", [("FP32", FP32_TOL), ("FP16", REDUCED_TOL)])
def test_hierarchical_geometry_matches_oracle(hai, ctx, prec, tol):
    """All 256 stations of the hierarchical array (core and tail) on the
    128^2 array grid, three beam directions, random int8 beams."""
    centres = I.station_centres(H)
    lam = H.station.lam_m
    dirs = np.array([[0.0, 0.0], [0.031, -0.057], [-0.12, 0.08]])
    K, C, T, P, S = 3, 2, 11, 2, len(centres)
    cin = I.random_voltages((K, C, T, P, S, 2), seed=5)
    got, dropped = station_epic(hai, ctx, centres, lam, H.cell_m, N_EPIC, dirs, cin.cuda(),
                                getattr(hai, "HAI_PREC_" + prec))
    want, wdrop = O.station_epic(N_EPIC, centres, lam, H.cell_m, dirs, cin.numpy())
    assert dropped == wdrop and 0 < dropped < H.n_tail + 1
    for k in range(K):
        assert rel_err_planes(got[k], want[k]).max() < tol, k


@pytest.mark.parametrize("n,P", [(32, 2), (64, 1), (64, 2)])
def test_small_arrays_and_one_polarisation(hai, ctx, n, P):
    rng = np.random.default_rng(n + P)
    cell, lam = 19.0, 3.0
    S = 40
    centres = rng.uniform(-n * cell / 4, n * cell / 4, (S, 2))
    centres[:3] = rng.uniform(n * cell, 2 * n * cell, (3, 2))        # dropped
    dirs = rng.uniform(-0.2, 0.2, (2, 2))
    cin = I.random_voltages((2, 3, 7, P, S, 2), seed=n * P)
    got, dropped = station_epic(hai, ctx, centres, lam, cell, n, dirs, cin.cuda(), hai.HAI_PREC_FP32)
    want, wdrop = O.station_epic(n, centres, lam, cell, dirs, cin.numpy())
    assert dropped == wdrop >= 3
    for k in range(2):
        assert rel_err_planes(got[k], want[k]).max() < FP32_TOL


def test_chain_beamformer_to_station_epic(hai, ctx):
    """Reduced hierarchical array (32 stations of 64 elements, 16 beams, 2
    channels, 16 samples): int8 beamformer with requantisation, beams to the
    station-major layout, inter-station EPIC on tensor cores; the oracle runs
    the same chain from the same seeded voltages."""
    S, C, T, K, P = 32, 2, 16, 16, 2
    st = I.StationConfig(name="st64", n_elem=64, diameter_m=19.0, min_spacing_m=1.5, lam_m=3.0, n_chan=C,
                         n_pol=P, n_time=T, grid_n=32, cell_lambda=0.5, ksize=3, seed=I.SEED0 + 9)
    elem = I.station_layout(st)
    centres = I.station_centres(H)[:S]
    dirs = I.beam_directions(K, st.lam_m, st.diameter_m)
    src = dirs[:2] + 0.004
    volt = I.hierarchy_voltages(H, centres, elem, src, np.array([1.0, 0.6]), S, C, T, device="cuda")
    w = torch.from_numpy(np.repeat(I.bf_weights(elem, st.lam_m, dirs, P)[None], S, axis=0)).cuda()
    shift = 9
    beams = torch.empty((S, C, T, K, P, 2), dtype=torch.int8, device="cuda")
    sat = torch.zeros(1, dtype=torch.int64, device="cuda")
    hai.hai_beamform(ctx, volt, w, S, C, T, K, len(elem), P, shift, beams, sat)
    cin = torch.empty((K, C, T, P, S, 2), dtype=torch.int8, device="cuda")
    hai.hai_beams_to_corr(ctx, beams, S, C, T, K, P, cin)
    got, dropped = station_epic(hai, ctx, centres, st.lam_m, H.cell_m, N_EPIC, dirs, cin, hai.HAI_PREC_FP16)
    bq, _ = O.requant(O.beamform(volt.cpu().numpy(), w.cpu().numpy()), shift)
    want, wdrop = O.station_epic(N_EPIC, centres, st.lam_m, H.cell_m, dirs,
                                 np.ascontiguousarray(bq.transpose(3, 1, 2, 4, 0, 5)))
    assert dropped == wdrop
    for k in range(K):
        assert rel_err_planes(got[k], want[k]).max() < REDUCED_TOL


def test_layout_arguments(hai, ctx):
    pos = np.zeros((4, 2))
    with pytest.raises(hai.HaiError) as e:
        hai.hai_station_epic_layout_create(ctx, pos, 3.0, 19.0, 64, np.zeros((2, 2)), 2)
    assert e.value.status == 1
    with pytest.raises(hai.HaiError) as e:
        hai.hai_station_epic_layout_create(ctx, pos, -1.0, 19.0, 64, None, 0)
    assert e.value.status == 1
    with pytest.raises(hai.HaiError) as e:
        hai.hai_station_epic_layout_create(ctx, pos, 3.0, 19.0, 1024, None, 0)
    assert e.value.status in (1, 4)
    lay, dropped = hai.hai_station_epic_layout_create(ctx, pos, 3.0, 19.0, 64, None, 0)
    assert dropped == 0 and lay.n_elem == 4 and lay.ksize == 1
    assert hai.hai_layout_box(lay) == (32, 32, 33, 33)
    hai.hai_layout_destroy(lay)
