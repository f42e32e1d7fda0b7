"""GPU parity of the batched uneven-station plan (one CUDA-graph launch per
cadence) against the FP64 oracle and against the per-station paths."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I
from tests.helpers import FP32_TOL, REDUCED_TOL, rel_err_planes, station

pytestmark = pytest.mark.gpu

UNEVEN = I.UnevenConfig()


@pytest.fixture(scope="module")
def ctx(hai):
    c = hai.hai_create(0)
    yield c
    hai.hai_destroy(c)


def make_array(hai, ctx, indices, C, T, sizes=None, random=False):
    """Layouts, voltages (host) and configs of the chosen stations."""
    out = []
    for k, i in enumerate(indices):
        sc = I.uneven_station(UNEVEN, i, None if sizes is None else sizes[k])
        pos, anchors, taps = station(sc)
        if random:
            volt = I.random_voltages((C, T, 2, len(pos), 2), seed=1000 + i)
        else:
            volt = I.station_voltages(sc, pos, n_chan=C, n_time=T)
        lay = hai.hai_layout_create(ctx, anchors, taps, sc.grid_n, 2)
        out.append((sc, anchors, taps, volt, lay))
    return out


def pack(plan, arr):
    buf = torch.zeros(plan.volt_bytes, dtype=torch.int8)
    for s, (_, _, _, volt, _) in enumerate(arr):
        flat = volt.reshape(-1)
        buf[plan.volt_off[s]: plan.volt_off[s] + flat.numel()] = flat
    return buf.cuda()


def unpack(plan, img, arr, C):
    img = img.cpu().numpy()
    res = []
    for s, (sc, *_rest) in enumerate(arr):
        n = sc.grid_n
        res.append(img[plan.img_off[s]: plan.img_off[s] + C * 4 * n * n].reshape(C, 4, n, n))
    return res


def test_plan_matches_oracle_and_per_station_paths(hai, ctx):
    C, T = 3, 10
    # three stations per grid side, smallest and largest sizes of the array included
    sizes = [16, 40, 66, 80, 200, 330, 400, 760, 1024]
    arr = make_array(hai, ctx, range(len(sizes)), C, T, sizes)
    assert sorted({a[0].grid_n for a in arr}) == [32, 64, 128]
    plan = hai.hai_plan_create(ctx, [a[4] for a in arr], C, T)
    vbuf = pack(plan, arr)
    img = torch.full((plan.img_floats,), float("nan"), device="cuda")
    hai.hai_plan_run(plan, vbuf, img)
    hai.hai_sync(ctx)
    got = unpack(plan, img, arr, C)
    for s, (sc, anchors, taps, volt, lay) in enumerate(arr):
        n = sc.grid_n
        want = O.epic_image(n, anchors, taps, volt.numpy())
        assert rel_err_planes(got[s], want).max() < REDUCED_TOL, (s, n)
        # the per-station tensor-core path
        one = torch.empty((C, 4, n, n), device="cuda")
        hai.hai_epic_image(ctx, lay, volt.cuda(), C, T, hai.HAI_PREC_FP16, one, 0)
        hai.hai_sync(ctx)
        assert rel_err_planes(got[s], one.cpu().numpy()).max() < REDUCED_TOL
        # the plain FP32 path (small-grid kernel up to 64, large-grid path at 128)
        hai.hai_epic_image(ctx, lay, volt.cuda(), C, T, hai.HAI_PREC_FP32, one, 0)
        hai.hai_sync(ctx)
        assert rel_err_planes(one.cpu().numpy(), want).max() < FP32_TOL
        assert rel_err_planes(got[s], one.cpu().numpy()).max() < REDUCED_TOL
    hai.hai_plan_destroy(plan)
    for a in arr:
        hai.hai_layout_destroy(a[4])


def test_plan_schedule_independent_and_graph_reuse(hai, ctx):
    """Every (station, channel) is summed by one CTA in sample order, so the
    images are bit-identical under any schedule: before and after autotuning,
    on repeated launches and on a second pair of buffers (new graph)."""
    C, T = 5, 7
    sizes = [20, 50, 100, 300, 600, 900]
    arr = make_array(hai, ctx, range(len(sizes)), C, T, sizes, random=True)
    plan = hai.hai_plan_create(ctx, [a[4] for a in arr], C, T)
    vbuf = pack(plan, arr)
    img = torch.empty((plan.img_floats,), device="cuda")
    hai.hai_plan_run(plan, vbuf, img)
    hai.hai_sync(ctx)
    first = img.cpu().numpy().copy()
    hai.hai_plan_run(plan, vbuf, img)
    hai.hai_sync(ctx)
    assert np.array_equal(first, img.cpu().numpy())
    before = hai.hai_plan_schedule(plan)
    hai.hai_plan_autotune(plan, vbuf, img, 2)
    after = hai.hai_plan_schedule(plan)
    assert [g for g, _, _ in after] == [g for g, _, _ in before]
    assert all(ms > 0 for _, _, ms in after)
    assert sum(c for _, c, _ in after) <= torch.cuda.get_device_properties(0).multi_processor_count
    img2 = torch.empty_like(img)
    vbuf2 = vbuf.clone()
    hai.hai_plan_run(plan, vbuf2, img2)
    hai.hai_plan_run(plan, vbuf, img)
    hai.hai_sync(ctx)
    assert np.array_equal(first, img2.cpu().numpy())
    assert np.array_equal(first, img.cpu().numpy())
    got = unpack(plan, img, arr, C)
    for s in (0, 3, 5):
        sc, anchors, taps, volt, _ = arr[s]
        want = O.epic_image(sc.grid_n, anchors, taps, volt.numpy())
        assert rel_err_planes(got[s], want).max() < REDUCED_TOL
    hai.hai_plan_destroy(plan)
    for a in arr:
        hai.hai_layout_destroy(a[4])


def test_plan_full_array_sampled_stations(hai, ctx):
    """All 512 stations of the uneven array in one plan (2 channels x 4
    samples); the oracle recomputes every 37th station."""
    C, T = 2, 4
    arr = make_array(hai, ctx, range(UNEVEN.n_station), C, T, random=True)
    plan = hai.hai_plan_create(ctx, [a[4] for a in arr], C, T)
    for a in arr:
        hai.hai_layout_destroy(a[4])            # the plan keeps its own copies
    vbuf = pack(plan, arr)
    img = torch.empty((plan.img_floats,), device="cuda")
    hai.hai_plan_autotune(plan, vbuf, img, 1)
    hai.hai_plan_run(plan, vbuf, img)
    hai.hai_sync(ctx)
    got = unpack(plan, img, arr, C)
    for s in range(0, UNEVEN.n_station, 37):
        sc, anchors, taps, volt, _ = arr[s]
        want = O.epic_image(sc.grid_n, anchors, taps, volt.numpy())
        assert rel_err_planes(got[s], want).max() < REDUCED_TOL, s
    hai.hai_plan_destroy(plan)


def test_plan_autotune_cache(hai, ctx, tmp_path):
    """The cached autotuner times a plan once and writes its shares; a second
    plan of the same shape takes them from the cache without timing, gets the
    same schedule, and images bit-identically."""
    C, T = 3, 9
    sizes = [30, 90, 250, 700]
    arr = make_array(hai, ctx, range(len(sizes)), C, T, sizes, random=True)
    cache = str(tmp_path / "plan_tune.txt")
    plans = [hai.hai_plan_create(ctx, [a[4] for a in arr], C, T) for _ in range(2)]
    try:
        vbuf = pack(plans[0], arr)
        imgs = [torch.empty((p.img_floats,), device="cuda") for p in plans]
        assert not hai.hai_plan_autotune_cached(plans[0], vbuf, imgs[0], cache, 1)
        assert " | units " in open(cache).read()
        assert hai.hai_plan_autotune_cached(plans[1], vbuf, imgs[1], cache, 1)
        s0, s1 = hai.hai_plan_schedule(plans[0]), hai.hai_plan_schedule(plans[1])
        assert [(g, c) for g, c, _ in s0] == [(g, c) for g, c, _ in s1]
        for p, im in zip(plans, imgs):
            hai.hai_plan_run(p, vbuf, im)
        hai.hai_sync(ctx)
        assert torch.equal(imgs[0].cpu(), imgs[1].cpu())
    finally:
        for p in plans:
            hai.hai_plan_destroy(p)
        for a in arr:
            hai.hai_layout_destroy(a[4])


def test_plan_rejects_unsupported_input(hai, ctx):
    sc = I.uneven_station(UNEVEN, 0, 50)
    pos, anchors, taps = station(sc)
    one_pol = hai.hai_layout_create(ctx, anchors, taps, sc.grid_n, 1)
    two_pol = hai.hai_layout_create(ctx, anchors, taps, sc.grid_n, 2)
    with pytest.raises(hai.HaiError) as e:
        hai.hai_plan_create(ctx, [two_pol, one_pol], 1, 4)
    assert e.value.status == 4
    with pytest.raises(hai.HaiError) as e:
        hai.hai_plan_create(ctx, [two_pol], 1, 4, hai.HAI_PREC_FP32)
    assert e.value.status == 4
    with pytest.raises(hai.HaiError) as e:
        hai.hai_plan_create(ctx, [two_pol], 0, 4)
    assert e.value.status == 1
    plan = hai.hai_plan_create(ctx, [two_pol], 1, 4)
    vbuf = torch.zeros(plan.volt_bytes + 16, dtype=torch.int8, device="cuda")
    img = torch.zeros(plan.img_floats + 4, device="cuda")
    # misaligned buffers are refused before anything launches
    rc = hai.load().hai_plan_run(plan.handle, vbuf.data_ptr() + 1, img.data_ptr(), None)
    assert rc == 1 and "aligned" in hai.hai_last_error()
    rc = hai.load().hai_plan_run(plan.handle, vbuf.data_ptr(), img.data_ptr() + 4, None)
    assert rc == 1
    hai.hai_plan_destroy(plan)
    hai.hai_layout_destroy(one_pol)
    hai.hai_layout_destroy(two_pol)
