"""The second level of the hierarchy in the batched plan's graph launch:
station beams of uneven stations (bit-exact against the oracle beamformer
and requantisation), their inter-station order, the inter-station
correlator (bit-exact) + XFFT and the inter-station EPIC of every beam
against the oracle chain, and the station images of the same launch against
the plan's own run."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import FP32_TOL, REDUCED_TOL, rel_err_planes, station

pytestmark = pytest.mark.gpu

U = I.UnevenConfig()


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


def build(hai, ctx, S, C, T, K, sizes=None, xfft=True, epic=True, epic_prec=None, vrange=8):
    stations = [I.uneven_station(U, i, None if sizes is None else sizes[i]) for i in range(S)]
    pos, lays = [], []
    for sc in stations:
        p, anchors, taps = station(sc)
        pos.append(p)
        lays.append(hai.hai_layout_create(ctx, anchors, taps, sc.grid_n, 2))
    plan = hai.hai_plan_create(ctx, lays, C, T)
    for ly in lays:
        hai.hai_layout_destroy(ly)
    volt = I.random_voltages((plan.volt_bytes,), seed=S + C + T, lo=-vrange, hi=vrange)
    dirs = I.beam_directions(K, U.lam_m, U.ref_diameter_m)
    wbuf, woff = I.uneven_beam_weights(U, pos, dirs)
    centres = I.uneven_centres(U, S)
    vl = hai.hai_vis_layout_create(ctx, centres, U.lam_m, U.xfft_cell_m, U.xfft_grid_n, dirs) if xfft else None
    el = [hai.hai_station_epic_layout_create(ctx, centres, U.lam_m, U.epic_cell_m, U.epic_grid_n, dirs, k)[0]
          for k in range(K)] if epic else None
    w = torch.from_numpy(wbuf).cuda()
    hai.hai_plan_set_hierarchy(plan, K, w, woff, U.requant_shift, xfft=vl, epic=el,
                               epic_prec=hai.HAI_PREC_FP32 if epic_prec is None else epic_prec)
    return plan, stations, volt, wbuf, woff, dirs, centres, vl, el


def release(hai, plan, vl, el):
    hai.hai_plan_destroy(plan)
    if vl is not None:
        hai.hai_vis_layout_destroy(vl)
    for ly in el or []:
        hai.hai_layout_destroy(ly)


def oracle_beams(plan, stations, volt, wbuf, woff, C, T, K):
    """Requantised beams [S][C][T][K][2][2] and the clamp count, per station
    through the oracle beamformer."""
    v = volt.numpy()
    out, nsat = [], 0
    for s, sc in enumerate(stations):
        ne = sc.n_elem
        vs = v[plan.volt_off[s]: plan.volt_off[s] + C * T * 2 * ne * 2].reshape(1, C, T, 2, ne, 2)
        ws = wbuf[woff[s]: woff[s] + K * 2 * ne * 2].reshape(1, K, 2, ne, 2)
        q, sat = O.requant(O.beamform(vs, ws), U.requant_shift)
        out.append(q[0])
        nsat += sat
    return np.stack(out), nsat


@pytest.mark.parametrize("epic_prec,tol", [("FP32", FP32_TOL), ("FP16", REDUCED_TOL)])
def test_second_level_matches_oracle_chain(hai, ctx, epic_prec, tol):
    """20 uneven stations (16 .. 1024 elements: several 256-element passes
    and ragged ones), 2 channels x 20 samples (a ragged block of 16), 4 beams;
    both inter-station stages in one launch."""
    S, C, T, K = 20, 2, 20, 4
    plan, stations, volt, wbuf, woff, dirs, centres, vl, el = build(
        hai, ctx, S, C, T, K, epic_prec=getattr(hai, "HAI_PREC_" + epic_prec))
    try:
        assert max(sc.n_elem for sc in stations) > 512
        nb, nv, nx, ne = hai.hai_plan_hier_sizes(plan)
        assert nb == S * C * T * K * 4 and nv == K * C * (S * (S + 1) // 2) * 8
        beams = torch.full((nb,), 99, dtype=torch.int8, device="cuda")
        corr = torch.full((nb,), 99, dtype=torch.int8, device="cuda")
        vis = torch.zeros(nv, dtype=torch.int32, device="cuda")
        ximg = torch.full((nx,), float("nan"), device="cuda")
        eimg = torch.full((ne,), float("nan"), device="cuda")
        nsat = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        img = torch.full((plan.img_floats,), float("nan"), device="cuda")
        vd = volt.cuda()
        hai.hai_plan_run_hier(plan, vd, img, beams, corr, vis, ximg, eimg, nsat)
        hai.hai_sync(ctx)
        # level 1: station images as the plan alone writes them
        img1 = torch.full((plan.img_floats,), float("nan"), device="cuda")
        hai.hai_plan_run(plan, vd, img1)
        hai.hai_sync(ctx)
        assert torch.equal(img.cpu(), img1.cpu())
        # beams, their order, visibilities: integers, bit-exact
        want_b, want_sat = oracle_beams(plan, stations, volt, wbuf, woff, C, T, K)
        got_b = beams.cpu().numpy().reshape(S, C, T, K, 2, 2)
        assert np.array_equal(got_b, want_b)
        assert int(nsat.item()) == want_sat
        cin = want_b.transpose(3, 1, 2, 4, 0, 5)                       # [K][C][T][P][S][2]
        assert np.array_equal(corr.cpu().numpy().reshape(cin.shape), cin)
        want_v = O.correlate(cin.reshape(K * C, T, 2, S, 2))
        assert np.array_equal(vis.cpu().numpy().reshape(want_v.shape), want_v)
        # inter-station images
        nbl = S * (S + 1) // 2
        want_x, dropped = O.station_xfft(U.xfft_grid_n, centres, U.lam_m, U.xfft_cell_m, dirs,
                                         want_v.reshape(K, C, nbl, 2, 2, 2))
        assert dropped == 0
        n = U.xfft_grid_n
        assert rel_err_planes(ximg.cpu().numpy().reshape(K * C, 4, n, n), planes(want_x)).max() < FP32_TOL
        want_e, _ = O.station_epic(U.epic_grid_n, centres, U.lam_m, U.epic_cell_m, dirs, cin)
        n = U.epic_grid_n
        got_e = eimg.cpu().numpy().reshape(K, C, 4, n, n)
        for k in range(K):
            assert rel_err_planes(got_e[k], want_e[k]).max() < tol, k
    finally:
        release(hai, plan, vl, el)


def test_one_stage_only_and_recapture(hai, ctx):
    """Only the inter-station EPIC set (no XFFT buffers needed); new buffers
    make the graph capture again; beams saturate at a loud input."""
    S, C, T, K = 6, 1, 16, 4
    plan, stations, volt, wbuf, woff, dirs, centres, vl, el = build(hai, ctx, S, C, T, K, xfft=False,
                                                                     vrange=127)
    try:
        nb, nv, nx, ne = hai.hai_plan_hier_sizes(plan)
        assert nv == 0 and nx == 0 and ne > 0
        vd = volt.cuda()
        want_b, want_sat = oracle_beams(plan, stations, volt, wbuf, woff, C, T, K)
        assert want_sat > 0
        for rep in range(2):
            beams = torch.zeros(nb, dtype=torch.int8, device="cuda")
            corr = torch.zeros(nb, dtype=torch.int8, device="cuda")
            eimg = torch.zeros(ne, device="cuda")
            nsat = torch.zeros(1, dtype=torch.int64, device="cuda")
            img = torch.zeros(plan.img_floats, device="cuda")
            hai.hai_plan_run_hier(plan, vd, img, beams, corr, None, None, eimg, nsat)
            hai.hai_sync(ctx)
            assert np.array_equal(beams.cpu().numpy().reshape(want_b.shape), want_b), rep
            assert int(nsat.item()) == want_sat
        cin = want_b.transpose(3, 1, 2, 4, 0, 5)
        want_e, _ = O.station_epic(U.epic_grid_n, centres, U.lam_m, U.epic_cell_m, dirs, cin)
        n = U.epic_grid_n
        got_e = eimg.cpu().numpy().reshape(K, C, 4, n, n)
        for k in range(K):
            assert rel_err_planes(got_e[k], want_e[k]).max() < FP32_TOL
    finally:
        release(hai, plan, vl, el)


@pytest.mark.parametrize("K", [9, 36])
def test_beam_counts(hai, ctx, K):
    """An odd beam count (a padded beam pair) and 18 beam pairs (32-sample
    blocks): beams bit-exact, visibilities bit-exact."""
    S, C, T = 5, 1, 40
    plan, stations, volt, wbuf, woff, dirs, centres, vl, el = build(hai, ctx, S, C, T, K, epic=False)
    try:
        nb, nv, nx, ne = hai.hai_plan_hier_sizes(plan)
        beams = torch.zeros(nb, dtype=torch.int8, device="cuda")
        corr = torch.zeros(nb, dtype=torch.int8, device="cuda")
        vis = torch.zeros(nv, dtype=torch.int32, device="cuda")
        ximg = torch.zeros(nx, device="cuda")
        img = torch.zeros(plan.img_floats, device="cuda")
        hai.hai_plan_run_hier(plan, volt.cuda(), img, beams, corr, vis, ximg)
        hai.hai_sync(ctx)
        want_b, _ = oracle_beams(plan, stations, volt, wbuf, woff, C, T, K)
        assert np.array_equal(beams.cpu().numpy().reshape(want_b.shape), want_b)
        cin = want_b.transpose(3, 1, 2, 4, 0, 5)
        want_v = O.correlate(cin.reshape(K * C, T, 2, S, 2))
        assert np.array_equal(vis.cpu().numpy().reshape(want_v.shape), want_v)
    finally:
        release(hai, plan, vl, el)


def test_beams_small_odd_and_split_stations(hai, ctx):
    """The persistent beam kernel's edge cases: stations of 1, 2 and 3
    elements, odd and even element counts (element pairs straddling 32-bit
    words, a padded last pair), and a 700-element station whose flat
    (channel, sample) rows take several items crossing channel boundaries;
    a loud input for saturations.  Beams and the clamp count bit-exact."""
    S, C, T, K = 6, 3, 13, 4
    sizes = [1, 2, 3, 17, 64, 700]
    plan, stations, volt, wbuf, woff, dirs, centres, vl, el = build(hai, ctx, S, C, T, K, sizes=sizes, epic=False,
                                                                     vrange=127)
    try:
        nb, nv, nx, ne = hai.hai_plan_hier_sizes(plan)
        beams = torch.zeros(nb, dtype=torch.int8, device="cuda")
        corr = torch.zeros(nb, dtype=torch.int8, device="cuda")
        vis = torch.zeros(nv, dtype=torch.int32, device="cuda")
        ximg = torch.zeros(nx, device="cuda")
        nsat = torch.zeros(1, dtype=torch.int64, device="cuda")
        img = torch.zeros(plan.img_floats, device="cuda")
        hai.hai_plan_run_hier(plan, volt.cuda(), img, beams, corr, vis, ximg, None, nsat)
        hai.hai_sync(ctx)
        want_b, want_sat = oracle_beams(plan, stations, volt, wbuf, woff, C, T, K)
        assert np.array_equal(beams.cpu().numpy().reshape(want_b.shape), want_b)
        assert int(nsat.item()) == want_sat
    finally:
        release(hai, plan, vl, el)


def test_hierarchy_arguments(hai, ctx):
    S, C, T, K = 3, 1, 4, 4
    plan, stations, volt, wbuf, woff, dirs, centres, vl, el = build(hai, ctx, S, C, T, K, epic=False)
    try:
        w = torch.from_numpy(wbuf).cuda()
        with pytest.raises(hai.HaiError) as e:                          # the XFFT layout has K = 4 directions
            hai.hai_plan_set_hierarchy(plan, 2, w, woff, 4, xfft=vl)
        assert e.value.status == 1
        with pytest.raises(hai.HaiError) as e:                          # no inter-station stage
            hai.hai_plan_set_hierarchy(plan, K, w, woff, 4)
        assert e.value.status == 1
        with pytest.raises(hai.HaiError) as e:
            hai.hai_plan_set_hierarchy(plan, K, w, woff, 31, xfft=vl)
        assert e.value.status == 1
    finally:
        release(hai, plan, vl, el)


def test_full_cadence_sampled(hai, ctx):
    """The uneven array at full size in the benchmark's launch configuration
    (512 stations, 128 channels x 64 samples, plan autotuned, 4 beams, both
    inter-station stages; random int8 voltages made on the device): sampled
    station images, beams of sampled stations (bit-exact), the visibilities
    and both inter-station images of sampled (beam, channel) pairs against
    the oracle."""
    C, T, K = U.n_chan, U.n_time, U.n_beam
    S = U.n_station
    stations = [I.uneven_station(U, i) for i in range(S)]
    pos, lays, kern = [], [], []
    for sc in stations:
        p, anchors, taps = station(sc)
        pos.append(p)
        kern.append((anchors, taps))
        lays.append(hai.hai_layout_create(ctx, anchors, taps, sc.grid_n, 2))
    plan = hai.hai_plan_create(ctx, lays, C, T)
    for ly in lays:
        hai.hai_layout_destroy(ly)
    g = torch.Generator(device="cuda").manual_seed(12)
    volt = torch.randint(-128, 128, (plan.volt_bytes,), dtype=torch.int8, device="cuda", generator=g)
    img = torch.empty((plan.img_floats,), device="cuda")
    hai.hai_plan_autotune(plan, volt, img, 2)
    dirs = I.beam_directions(K, U.lam_m, U.ref_diameter_m)
    wbuf, woff = I.uneven_beam_weights(U, pos, dirs)
    centres = I.uneven_centres(U)
    vl = hai.hai_vis_layout_create(ctx, centres, U.lam_m, U.xfft_cell_m, U.xfft_grid_n, dirs)
    el = [hai.hai_station_epic_layout_create(ctx, centres, U.lam_m, U.epic_cell_m, U.epic_grid_n, dirs, k)[0]
          for k in range(K)]
    try:
        hai.hai_plan_set_hierarchy(plan, K, torch.from_numpy(wbuf).cuda(), woff, U.requant_shift, xfft=vl, epic=el,
                                   epic_prec=hai.HAI_PREC_FP16)
        nb, nv, nx, ne = hai.hai_plan_hier_sizes(plan)
        beams = torch.empty(nb, dtype=torch.int8, device="cuda")
        corr = torch.empty(nb, dtype=torch.int8, device="cuda")
        vis = torch.empty(nv, dtype=torch.int32, device="cuda")
        ximg = torch.empty(nx, device="cuda")
        eimg = torch.empty(ne, device="cuda")
        hai.hai_plan_run_hier(plan, volt, img, beams, corr, vis, ximg, eimg)
        hai.hai_sync(ctx)
        v = volt.cpu().numpy()
        # station images of sampled (station, channel) blocks
        imgs = img.cpu().numpy()
        for s, c in ((0, 0), (97, 127), (255, 64), (400, 3), (511, 100)):
            sc, (anchors, taps) = stations[s], kern[s]
            n, nel = sc.grid_n, sc.n_elem
            blk = v[plan.volt_off[s]: plan.volt_off[s] + C * T * 2 * nel * 2].reshape(C, T, 2, nel, 2)
            want = O.epic_image(n, anchors, taps, blk[c:c + 1])
            got = imgs[plan.img_off[s] + c * 4 * n * n: plan.img_off[s] + (c + 1) * 4 * n * n].reshape(1, 4, n, n)
            assert rel_err_planes(got, want).max() < REDUCED_TOL, (s, c)
        # beams of sampled stations, every channel and sample: bit-exact
        got_b = beams.cpu().numpy().reshape(S, C, T, K, 2, 2)
        for s in (1, 200, 511):
            nel = stations[s].n_elem
            vs = v[plan.volt_off[s]: plan.volt_off[s] + C * T * 2 * nel * 2].reshape(1, C, T, 2, nel, 2)
            ws = wbuf[woff[s]: woff[s] + K * 2 * nel * 2].reshape(1, K, 2, nel, 2)
            q, _ = O.requant(O.beamform(vs, ws), U.requant_shift)
            assert np.array_equal(got_b[s], q[0]), s
        # second level for sampled (beam, channel) pairs, from the beams the plan made
        cin_all = corr.cpu().numpy().reshape(K, C, T, 2, S, 2)
        assert np.array_equal(cin_all, got_b.transpose(3, 1, 2, 4, 0, 5))
        nbl = S * (S + 1) // 2
        vis_all = vis.cpu().numpy().reshape(K, C, nbl, 2, 2, 2)
        x_all = ximg.cpu().numpy().reshape(K, C, 4, U.xfft_grid_n, U.xfft_grid_n)
        e_all = eimg.cpu().numpy().reshape(K, C, 4, U.epic_grid_n, U.epic_grid_n)
        for k, c in ((0, 0), (3, 127), (1, 50)):
            cin = cin_all[k:k + 1, c:c + 1]
            want_v = O.correlate(cin.reshape(1, T, 2, S, 2))
            assert np.array_equal(vis_all[k, c], want_v[0]), (k, c)
            want_x, dropped = O.station_xfft(U.xfft_grid_n, centres, U.lam_m, U.xfft_cell_m, dirs[k:k + 1],
                                             want_v.reshape(1, 1, nbl, 2, 2, 2))
            assert dropped == 0
            assert rel_err_planes(x_all[k, c][None], planes(want_x)).max() < FP32_TOL, (k, c)
            want_e, _ = O.station_epic(U.epic_grid_n, centres, U.lam_m, U.epic_cell_m, dirs[k:k + 1], cin)
            assert rel_err_planes(e_all[k, c][None], want_e[0]).max() < REDUCED_TOL, (k, c)
    finally:
        hai.hai_plan_destroy(plan)
        hai.hai_vis_layout_destroy(vl)
        for ly in el:
            hai.hai_layout_destroy(ly)
