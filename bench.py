"""Benchmark of the EPIC hot path on GB300 (one JSON line on rank 0).

A step is one cadence of the EPIC imager of the dense all-sky lattice
(16,384 elements, 512 x 512 grid, 16 channels, 2 polarisations, 10^4 samples):
gridding, the per-sample 2D DFT on tensor cores, squaring and accumulation,
through the C ABI (hai_epic_image).  value = imaged pixel x channel x pol x
sample per second.
`--impl reference` times the FP64 CPU oracle on a bounded sample instead.
Multi-GPU: every rank images its own cadence (channels are independent), no
collective on the data path; value is the sum over ranks / the max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "imaged pix·chan·pol·samples/s"
UNIT = "pix·chan·pol·samples/s"


PRECS = {"fp32": 0, "fp16": 1, "fp16_split": 2, "bf16": 3, "bf16_split": 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=list(PRECS), default="fp16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--no-components", action="store_true")
    ap.add_argument("--channels", type=int, default=0,
                    help="image only this many channels (small cases for profiling)")
    ap.add_argument("--samples", type=int, default=0,
                    help="samples per cadence of the headline workload (default 10^4)")
    ap.add_argument("--case", choices=["tc64", "fp32_64", "tc128", "corr", "xfft", "bf", "xbf", "sxfft", "fc", "big", "big16", "big2",
                                       "plan_hier", "plan_hier128"],
                    default=None,
                    help="run one small case of a kernel twice, untimed, and exit (for ncu captures)")
    return ap.parse_args()


_BACKEND = None


def dist_init(n, backend=None):
    """One process per GPU (RANK / LOCAL_RANK / WORLD_SIZE / MASTER_* from the
    launcher): NCCL on GPUs, gloo on hosts without one."""
    global _BACKEND
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        _BACKEND = backend or ("nccl" if torch.cuda.is_available() else "gloo")
        if _BACKEND == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    """The slowest rank's time (the job's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _BACKEND == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_channels(rank, C):
    """Channels are independent: rank r images its own band of C channels,
    [r C, (r + 1) C), with no collective on the data path (weak scaling)."""
    return rank * C, (rank + 1) * C


def job_value(ws, units_per_rank, max_ms):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return ws * units_per_rank / (max_ms * 1e-3)


HEADLINE_T = 10000


def workload(samples=0):
    """The dense all-sky lattice (128 x 128 elements at 0.5 lambda, 512^2 grid,
    1 x 1 unit taps, 16 channels, 2 pols) over the longest cadence of its
    range, 10^4 samples: the largest workload that fits one GPU (10.5 GB of
    voltages, 8.4e10 imaged units per cadence)."""
    import dataclasses
    from paper_2411_17804_gb300 import inputs as I
    cfg = dataclasses.replace(I.DENSE_ALLSKY_16384, n_time=samples or HEADLINE_T)
    cfg = dataclasses.replace(cfg, name=f"dense_allsky16384_grid512_T{cfg.n_time}")
    pos = I.station_layout(cfg)
    anchors, taps = I.station_kernel(cfg, pos)
    return cfg, pos, anchors, taps


def pruned_dft_flop(n, R, Cnz):
    """Algorithmic tensor-core FLOP of one field's two-stage DFT of the
    kernel's bounding box (R rows, Cnz columns): 8 (R N Cnz + N^2 R) real FLOP
    (8 per complex multiply-add)."""
    return 8.0 * (R * n * Cnz + n * n * R)


def stage2_flop(n, R):
    """The second stage's share: 8 N^2 R per field."""
    return 8.0 * n * n * R


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the samples go to a temporary file (or to $HAI_CLOCKS_CSV, kept), read back by stop()
        self.keep = "HAI_CLOCKS_CSV" in os.environ
        self.path = os.environ.get("HAI_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                     f"hai_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        if not self.keep:
            os.remove(self.path)
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return out


def epic_flops_per_unit(cfg):
    """Algorithmic FLOP per imaged unit (pixel x channel x pol x sample):
    radix-2 FFT 5 log2(N^2), gridding 8 N_e K^2 / N^2, squaring and
    accumulation 8 (XX, YY, XY: 8 FMA per pixel per sample for 2 pols)."""
    n = cfg.grid_n
    return 5 * math.log2(n * n) + 8.0 * cfg.n_elem * cfg.ksize ** 2 / (n * n) + 8.0


def corr_mma_flops(C, T, N, P):
    """Executed tensor-core FLOP of one correlator launch: tiles (row block of
    128 / P elements x two column blocks of 64 / P elements, a >= b somewhere
    in it) x 32-sample k blocks x 4 MMAs of 128 x 256 x 16."""
    em, E = 128 // P, 64 // P
    nbi, nbj = -(-N // em), -(-N // E)
    npairs = max((nbj + 1) // 2, nbi)
    tiles = sum(min(npairs, min(N - 1, (i + 1) * em - 1) // (2 * E) + 1) for i in range(nbi))
    stages = -(-T // 32)
    return C * tiles * stages * 4 * 2.0 * 128 * 256 * 16


def corr_useful_ops(C, T, N, P):
    """Integer operations the correlation itself needs: 8 per complex MAC
    (P^2 pol pairs, N(N+1)/2 baselines, T samples)."""
    return 8.0 * C * T * P * P * N * (N + 1) / 2


def time_call(fn, steps, warm, flush):
    import torch
    st = torch.cuda.current_stream()
    for _ in range(warm):
        fn(st)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.add_(1.0)
        ev[i][0].record(st)
        fn(st)
        ev[i][1].record(st)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def fp32_alu_peak_tflops(sm_count, sm_mhz):
    """CUDA-core FP32 peak: SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


def probe_peaks(hai, ctx):
    """The library's peak-rate probes, timed with CUDA events on the launching
    stream (best of 3 after a warm-up): scalar and packed FP32 FMA, and int8
    mma.sync (the legacy warp-level tensor path)."""
    import torch
    st = torch.cuda.current_stream()
    out = {}
    for name, kind, iters in (("fp32_ffma_tflops", 0, 20000), ("fp32_ffma2_tflops", 1, 20000),
                              ("imma_sync_s8_tops", 2, 4000)):
        hai.hai_probe_peak(ctx, kind, iters // 10, st)
        best = 0.0
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            ops = hai.hai_probe_peak(ctx, kind, iters, st)
            b.record(st)
            b.synchronize()
            best = max(best, ops / (a.elapsed_time(b) * 1e-3) / 1e12)
        out[name] = best
    out["fp32_tflops"] = max(out["fp32_ffma_tflops"], out["fp32_ffma2_tflops"])
    return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def image_error(got, want):
    """Per-(channel, plane) error of GPU images against the oracle's: the
    relative Frobenius error and the largest per-pixel error over the plane's
    peak (cross-pol planes measured against the auto planes' scale)."""
    n_chan = want.shape[0]
    got = got[:n_chan].astype(np.float64)
    w = want.reshape(n_chan, want.shape[1], -1)
    g = got.reshape(w.shape)
    d = np.linalg.norm(g - w, axis=-1)
    r = np.linalg.norm(w, axis=-1)
    r = np.maximum(r, 1e-3 * r[:, :2].max(axis=1, keepdims=True))
    pk = np.abs(w).max(axis=-1)
    pk = np.maximum(pk, 1e-3 * pk[:, :2].max(axis=1, keepdims=True))
    e = d / r
    px = np.abs(g - w).max(axis=-1) / pk
    return {"metric": "||I_gpu - I_oracle||_F / ||I_oracle||_F per (channel, plane); pixel: max|dI| / max|I_oracle|",
            "channels": n_chan, "max": float(e.max()), "median": float(np.median(e)),
            "pixel_max": float(px.max()), "per_plane_max": [float(x) for x in e.max(axis=0)]}


def cpu_baseline(cfg, anchors, taps, volt_host, gpu_imgs=None, min_s=10.0):
    """FP64 oracle on the host cores over a bounded sample of the cadence (the
    channels in volt_host, every sample), repeated until at least min_s seconds
    of CPU work have run.  Its images also give the per-image error of the GPU
    images of those channels (one entry per precision in gpu_imgs)."""
    from oracle import oracle as O
    n_chan, T = volt_host.shape[0], volt_host.shape[1]
    reps, want = 0, None
    t0 = time.perf_counter()
    while True:
        out_img = O.epic_image(cfg.grid_n, anchors, taps, volt_host)
        if want is None:
            want = out_img
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= min_s:
            break
    units = cfg.grid_n ** 2 * n_chan * cfg.n_pol * T * reps
    out = {"value": units / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
           "sample": f"{n_chan} of {cfg.n_chan} channels x all {T} samples of the cadence, x {reps} ({dt:.1f} s)"}
    # the same oracle on one core, over the first 128 samples of the first channel
    all_threads = O.num_threads()
    O.set_threads(1)
    try:
        t1 = time.perf_counter()
        O.epic_image(cfg.grid_n, anchors, taps, volt_host[:1, :128])
        d1 = time.perf_counter() - t1
    finally:
        O.set_threads(all_threads)
    out["one_core"] = {"value": cfg.grid_n ** 2 * cfg.n_pol * min(T, 128) / d1, "unit": UNIT, "cores": 1,
                       "sample": f"1 channel x {min(T, 128)} samples ({d1:.1f} s)"}
    errs = {k: image_error(v, want) for k, v in (gpu_imgs or {}).items()}
    return out, errs


def headline_config(cfg, prec_name, ws):
    return {"workload": cfg.name, "elements": cfg.n_elem, "channels": cfg.n_chan, "pols": cfg.n_pol,
            "samples": cfg.n_time, "grid": cfg.grid_n, "kernel_taps": cfg.ksize ** 2, "precision": prec_name,
            "l2": "inputs larger than L2 (10.5 GB of voltages per step), and a 256 MB write between steps",
            "parallelism": f"channel bands x{ws} (rank r images channels [r C, (r+1) C), no collective)"}


def run_reference(args, ws, rank):
    """The oracle itself (this workload's reference arm): every step images a
    bounded sample of the headline workload, 1 channel x 100 samples, on the
    host cores."""
    if rank != 0:
        return
    cfg, pos, anchors, taps = workload(args.samples)
    steps, warm = args.steps, args.warmup
    sample_chan, sample_t = 1, min(100, cfg.n_time)
    from oracle import oracle as O
    from paper_2411_17804_gb300 import inputs as I
    volt = I.station_voltages(cfg, pos, n_chan=sample_chan, n_time=sample_t).numpy()
    for _ in range(warm):
        O.epic_image(cfg.grid_n, anchors, taps, volt[:, :4])
    t0 = time.perf_counter()
    for _ in range(steps):
        O.epic_image(cfg.grid_n, anchors, taps, volt)
    dt = (time.perf_counter() - t0) / steps
    units = cfg.grid_n ** 2 * sample_chan * cfg.n_pol * sample_t
    v = units / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(cfg, args.prec, ws),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{sample_chan} of {cfg.n_chan} channels x {sample_t} of {cfg.n_time} "
                                       "samples per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def paper_cost(array, level, channels, samples, step_ms, measured="EPIC"):
    """The paper's own FLOP-cost estimate of one cadence (Table 2 formulas on
    the Table 1 row of `array`, per station or station beam), for every
    architecture of the stage, with the count of the `measured` architecture
    over the time measured for it here."""
    from paper_2411_17804_gb300 import cost as K
    n, ratio = K.level_args(K.ARRAYS[array], level)
    flop = {x: K.flop_per_cadence(x, n, ratio, channels, samples) for x in K.ARCHS}
    t_acc = samples * K.DELTA_T
    return {"source": f"Table 2 formulas, Table 1 {array} ({level}-station: n = {n}, ratio = {ratio:.4g}), "
                      f"n_p 2, delta t 25 us",
            "t_acc_s": t_acc, "channels_x_beams": channels, "flop_per_cadence": flop,
            "cheapest": min(flop, key=flop.get),
            "measured_arch": measured,
            "paper_flop_per_s_at_measured_time": flop[measured] / (step_ms * 1e-3),
            "voxels_per_channel": ratio * ratio}


def time_epic(hai, ctx, lay, volt, img, C, T, prec, steps, warm, flush, ws):
    import torch
    st = torch.cuda.current_stream()
    for _ in range(warm):
        hai.hai_epic_image(ctx, lay, volt, C, T, prec, img, 0, st)
    hai.hai_sync(ctx, st)
    hai.hai_profile_read(ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier(ws)
    torch.cuda.synchronize()
    for i in range(steps):
        flush.add_(1.0)                           # evict L2 between steps
        ev[i][0].record(st)
        hai.hai_epic_image(ctx, lay, volt, C, T, prec, img, 0, st)
        ev[i][1].record(st)
    torch.cuda.synchronize()
    barrier(ws)
    hai.hai_sync(ctx, st)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dom_ms, dom_n, launches = hai.hai_profile_read(ctx)
    # total step time, summed dominant-kernel time and library kernel launches
    # over the timed steps
    return float(np.sum(step_ms)), dom_ms, launches


def bf_component(hai, ctx, flush, peaks):
    """int8 station beamformer on the hierarchical workload's shape (256
    stations x 256 elements, 32 channels, 2 pols, 1000 samples, 16 beams),
    random int8 voltages and weights (the kernel's time does not depend on
    the values), int32 beams and requantised int8 beams.  HBM-bound: the
    algorithmic bytes are the voltages read plus the beams written."""
    import torch
    S, C, T, K, N, P = 256, 32, 1000, 16, 256, 2
    g = torch.Generator(device="cuda").manual_seed(11)
    volt = torch.randint(-128, 128, (S, C, T, P, N, 2), dtype=torch.int8, device="cuda", generator=g)
    w = torch.randint(-127, 128, (S, K, P, N, 2), dtype=torch.int8, device="cuda", generator=g)
    sat = torch.zeros(1, dtype=torch.int64, device="cuda")
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {"shape": {"stations": S, "channels": C, "samples": T, "beams": K, "elements": N, "pols": P}}
    for name, shift, dt, osz in (("int32", -1, torch.int32, 4), ("int8_requant", 10, torch.int8, 1)):
        beams = torch.empty((S, C, T, K, P, 2), dtype=dt, device="cuda")
        ms = time_call(lambda st: hai.hai_beamform(ctx, volt, w, S, C, T, K, N, P, shift, beams,
                                                   sat if shift >= 0 else None, st), 5, 3, flush)
        byts = volt.numel() + w.numel() + beams.numel() * osz
        gbs = byts / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "beam_samples_per_s": S * C * T * K * P / (ms * 1e-3),
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                  "frac": gbs / hbm, "traffic": None, "algorithmic_bytes": byts,
                                  "peak_source": "of measured hbm_gbs" if "hbm_gbs" in peaks
                                  else "of fallback 6.8 TB/s"}}
        del beams
    del volt, w
    return out


def plan_mma_flops(n, ne=None):
    """Executed tensor-core FLOP per (channel, sample) of a station of grid
    side n: N = 32: 3 products 128 x 64 x 32 per 4 samples; N = 64: 3 products
    128 x 128 x 64 per 2 samples; N = 128: per CTA of the 4-CTA cluster
    128 x 64 x 128 + 128 x 128 x 128 per sample."""
    if n == 32:
        return 2.0 * 3 * 128 * 64 * 32 / 4
    if n == 64:
        return 2.0 * 3 * 128 * 128 * 64 / 2
    return 2.0 * 4 * (128 * 64 * 128 + 128 * 128 * 128)


def plan_component(hai, ctx, flush, peaks, steps):
    """Batched uneven-station plan on the uneven array: 512 stations of
    log-uniform 16..1024 elements, grids 32..128, 128 channels x 2 pols x 64
    samples per cadence, one CUDA-graph launch per cadence after two
    autotuning rounds; uniform random int8 voltages (times do not depend on
    the values)."""
    import torch
    from paper_2411_17804_gb300 import inputs as I
    cfg = I.UnevenConfig()
    C, T = cfg.n_chan, cfg.n_time
    t0 = time.perf_counter()
    lays, grids = [], []
    for i in range(cfg.n_station):
        sc = I.uneven_station(cfg, i)
        pos = I.station_layout(sc)
        anchors, taps = I.station_kernel(sc, pos)
        lays.append(hai.hai_layout_create(ctx, anchors, taps, sc.grid_n, 2))
        grids.append(sc.grid_n)
    plan = hai.hai_plan_create(ctx, lays, C, T)
    for ly in lays:
        hai.hai_layout_destroy(ly)
    setup_s = time.perf_counter() - t0
    g = torch.Generator(device="cuda").manual_seed(12)
    volt = torch.randint(-128, 128, (plan.volt_bytes,), dtype=torch.int8, device="cuda", generator=g)
    img = torch.empty((plan.img_floats,), device="cuda")
    plan_cache = os.environ.get("HAI_PLAN_TUNE_CACHE") or os.path.join(tempfile.gettempdir(), "hai_plan_autotune.txt")
    from_cache = hai.hai_plan_autotune_cached(plan, volt, img, plan_cache, 2)
    sched = hai.hai_plan_schedule(plan)
    ms = time_call(lambda st: hai.hai_plan_run(plan, volt, img, st), steps, 3, flush)
    units = sum(n * n for n in grids) * C * 2 * T
    flops = sum(plan_mma_flops(n) for n in grids) * C * T
    pk = float(peaks.get("bf16_tflops", 1900.0))
    ach = flops / (ms * 1e-3) / 1e12
    # end to end: pinned host voltages in, images out, every cadence
    vh = torch.empty(volt.shape, dtype=torch.int8).pin_memory()
    ih = torch.empty(img.shape, dtype=torch.float32).pin_memory()
    st = torch.cuda.current_stream()
    for _ in range(2):
        volt.copy_(vh, non_blocking=True)
        hai.hai_plan_run(plan, volt, img, st)
        ih.copy_(img, non_blocking=True)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(3):
        volt.copy_(vh, non_blocking=True)
        hai.hai_plan_run(plan, volt, img, st)
        ih.copy_(img, non_blocking=True)
    torch.cuda.synchronize()
    e_ms = (time.perf_counter() - e0) * 1e3 / 3
    hier = plan_hierarchy(hai, ctx, plan, cfg, volt, img, flush, steps, ms,
                          sum(n * n for n in grids) * C * 2 * T)
    out = {"workload": cfg.name, "stations": cfg.n_station, "channels": C, "samples": T,
           "grid_classes": {str(n): grids.count(n) for n in sorted(set(grids))},
           "ms": ms, "units_per_s": units / (ms * 1e-3), "unit": UNIT,
           "graph_launches_per_cadence": 1, "kernels_per_cadence": len(sched),
           "schedule": [{"grid": n, "ctas": c, "alone_ms": m} for n, c, m in sched],
           "autotune": {"cache": plan_cache, "from_cache": from_cache},
           "setup_s": setup_s,
           "roofline": {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                        "peak_source": "of measured bf16_tflops (fp16 nominal ratio 1)"},
           "e2e": {"value": units / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(volt.numel()),
                   "d2h_bytes_per_step": int(img.numel() * 4)},
           "hierarchy": hier}
    hai.hai_plan_destroy(plan)
    del volt, img, vh, ih
    return out


def plan_hierarchy(hai, ctx, plan, cfg, volt, img, flush, steps, plan_ms, units):
    """The second level in the same graph launch: K beams per station
    (int8 weights towards a 2 x 2 lattice of directions), then the
    inter-station correlator + XFFT (256^2, 38 m cells) and the inter-station
    EPIC (128^2, 76 m cells, FP16) of every beam, for the 512 stations in a
    3 km core."""
    import torch
    from paper_2411_17804_gb300 import inputs as I
    K, S = cfg.n_beam, cfg.n_station
    pos = [I.station_layout(I.uneven_station(cfg, i)) for i in range(S)]
    dirs = I.beam_directions(K, cfg.lam_m, cfg.ref_diameter_m)
    wbuf, woff = I.uneven_beam_weights(cfg, pos, dirs)
    centres = I.uneven_centres(cfg)
    vl = hai.hai_vis_layout_create(ctx, centres, cfg.lam_m, cfg.xfft_cell_m, cfg.xfft_grid_n, dirs)
    el = [hai.hai_station_epic_layout_create(ctx, centres, cfg.lam_m, cfg.epic_cell_m, cfg.epic_grid_n, dirs, k)[0]
          for k in range(K)]
    w = torch.from_numpy(wbuf).cuda()
    hai.hai_plan_set_hierarchy(plan, K, w, woff, cfg.requant_shift, xfft=vl, epic=el, epic_prec=hai.HAI_PREC_FP16)
    nb, nv, nx, ne = hai.hai_plan_hier_sizes(plan)
    beams = torch.empty(nb, dtype=torch.int8, device="cuda")
    corr = torch.empty(nb, dtype=torch.int8, device="cuda")
    vis = torch.empty(nv, dtype=torch.int32, device="cuda")
    ximg = torch.empty(nx, device="cuda")
    eimg = torch.empty(ne, device="cuda")
    nsat = torch.zeros(1, dtype=torch.int64, device="cuda")
    run = lambda st: hai.hai_plan_run_hier(plan, volt, img, beams, corr, vis, ximg, eimg, nsat, st)
    ms = time_call(run, steps, 3, flush)
    # end to end: pinned voltages in; station images and both inter-station images out
    vh = torch.empty(volt.shape, dtype=torch.int8).pin_memory()
    outs = [(img, torch.empty(img.shape, dtype=torch.float32).pin_memory()),
            (ximg, torch.empty(ximg.shape, dtype=torch.float32).pin_memory()),
            (eimg, torch.empty(eimg.shape, dtype=torch.float32).pin_memory())]
    st = torch.cuda.current_stream()

    def cadence():
        volt.copy_(vh, non_blocking=True)
        run(st)
        for d, h in outs:
            h.copy_(d, non_blocking=True)
    for _ in range(2):
        cadence()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(3):
        cadence()
    torch.cuda.synchronize()
    e_ms = (time.perf_counter() - e0) * 1e3 / 3
    res = {"what": "station EPIC images + station beams -> inter-station correlator + XFFT and EPIC, one graph",
           "beams": K, "requant_shift": cfg.requant_shift, "ms": ms, "second_level_ms": ms - plan_ms,
           "xfft_grid": cfg.xfft_grid_n, "epic_grid": cfg.epic_grid_n, "epic_prec": "fp16",
           "saturated_beam_components": int(nsat.item()),
           "e2e": {"value": units / (e_ms * 1e-3), "unit": UNIT, "ms": e_ms,
                   "h2d_bytes_per_step": int(volt.numel()),
                   "d2h_bytes_per_step": int(sum(d.numel() * 4 for d, _ in outs))}}
    del beams, corr, vis, ximg, eimg, vh, outs
    hai.hai_vis_layout_destroy(vl)
    for ly in el:
        hai.hai_layout_destroy(ly)
    return res


def fft_correlator_component(hai, ctx, img, C, n, P, flush, peaks):
    """FFT correlator on the headline's accumulated images: the redundant-
    baseline visibility sums of the lattice at every lag (the inverse FFT,
    once per cadence).  HBM roofline: image read once, grid written once."""
    import torch
    grid = torch.empty((C, P, P, n, n, 2), device="cuda")
    fc_ms = time_call(lambda st: hai.hai_fft_correlate(ctx, img, C, n, P, grid, st), 10, 3, flush)
    fc_bytes = img.numel() * 4 + grid.numel() * 4
    fc_gbs = fc_bytes / (fc_ms * 1e-3) / 1e9
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    del grid
    return {"what": "inverse FFT of the accumulated images -> visibilities summed per lag, all 4 pol pairs",
            "ms": fc_ms, "lags_per_s": C * P * P * n * n / (fc_ms * 1e-3),
            "roofline": {"bound": "hbm", "achieved": fc_gbs, "peak": hbm, "unit": "GB/s", "frac": fc_gbs / hbm,
                         "algorithmic_bytes": fc_bytes}}


def ska_component(hai, ctx, flush, peaks, sms, steps, fp32_peak=None):
    """The SKA-low-shaped station (256 elements in a 38 m disk, 3 x 3 Gaussian
    taps, 64^2 grid, 64 channels x 2 pols x 2048 samples): EPIC on tensor
    cores (fp16, and the hi/lo split), on CUDA cores (FP32), end to end through
    host buffers, and the correlator + XFFT comparison path on the same
    cadence.  The tensor-core roofline counts the pruned DFT of the layout's
    own kernel box (8 (R N C + N^2 R) per field); the FP32 one the
    FFT-equivalent work per unit against the probed FP32 FMA peak."""
    import torch
    from paper_2411_17804_gb300 import inputs as I
    cfg = I.SKA_LOW_STATION_256
    pos = I.station_layout(cfg)
    anchors, taps = I.station_kernel(cfg, pos)
    C, T, P, n = cfg.n_chan, cfg.n_time, cfg.n_pol, cfg.grid_n
    volt = I.station_voltages(cfg, pos, device="cuda")
    lay = hai.hai_layout_create(ctx, anchors, taps, n, P)
    img = torch.empty((C, 4, n, n), device="cuda")
    units = cfg.units_per_cadence
    x0, y0, x1, y1 = hai.hai_layout_box(lay)
    R, Cnz = y1 - y0, x1 - x0
    pk = float(peaks.get("bf16_tflops", 1900.0))
    hai.hai_profile_read(ctx)
    out = {"workload": cfg.name, "elements": cfg.n_elem, "channels": C, "pols": P, "samples": T, "grid": n,
           "kernel_box": [Cnz, R]}
    for name, prec in (("fp16", hai.HAI_PREC_FP16), ("fp16_split", hai.HAI_PREC_FP16_SPLIT),
                       ("fp32", hai.HAI_PREC_FP32)):
        ns = steps if name == "fp16" else max(3, steps // 4)
        tot, dom, _ = time_epic(hai, ctx, lay, volt, img, C, T, prec, ns, 2, flush, 1)
        ms, dom = tot / ns, dom / ns
        e = {"ms": ms, "units_per_s": units / (ms * 1e-3), "kernel_ms": dom}
        if prec != hai.HAI_PREC_FP32:
            fl = pruned_dft_flop(n, R, Cnz) * C * T * P * (3 if name.endswith("split") else 1)
            ach = fl / (dom * 1e-3) / 1e12
            e["roofline"] = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                             "kernel": "epic_tc_kernel", "flop_per_field": pruned_dft_flop(n, R, Cnz),
                             "basis": f"pruned DFT of the {Cnz} x {R} kernel box, 8 (R N C + N^2 R) per field"}
        elif fp32_peak:
            fpu = epic_flops_per_unit(cfg)
            ach = fpu * units / (dom * 1e-3) / 1e12
            e["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                             "frac": ach / fp32_peak, "kernel": "epic64_kernel", "flop_per_unit": fpu,
                             "basis": "FFT-equivalent work 5 log2(N^2) + gridding + squaring per unit over the "
                                      "kernel's event time; peak measured by hai_probe_peak"}
        out[name] = e
    out["tc_over_fp32"] = out["fp32"]["ms"] / out["fp16"]["ms"]
    # end to end through the C ABI with host buffers (pinned)
    vh = volt.cpu().pin_memory()
    ih = torch.empty(img.shape, dtype=torch.float32).pin_memory()
    st = torch.cuda.current_stream()
    for _ in range(2):
        hai.hai_epic_image_host(ctx, lay, vh, C, T, hai.HAI_PREC_FP16, ih, 0, 0, st)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(5):
        hai.hai_epic_image_host(ctx, lay, vh, C, T, hai.HAI_PREC_FP16, ih, 0, 0, st)
    torch.cuda.synchronize()
    e_ms = (time.perf_counter() - e0) * 1e3 / 5
    out["e2e"] = {"value": units / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(volt.numel()),
                  "d2h_bytes_per_step": int(img.numel() * 4), "api": "hai_epic_image_host"}
    # the comparison path on the same cadence: correlator (exact int8) + XFFT
    N = cfg.n_elem
    vis = torch.empty((C, N * (N + 1) // 2, P, P, 2), dtype=torch.int32, device="cuda")
    cms = time_call(lambda st: hai.hai_correlate(ctx, volt, C, T, N, P, vis, 0, st), 10, 3, flush)
    xms = time_call(lambda st: hai.hai_xfft_image(ctx, lay, vis, C, img, 0, st), 10, 3, flush)
    mma = corr_mma_flops(C, T, N, P)
    out["correlator"] = {"ms": cms, "visibilities_per_s": C * N * (N + 1) / 2 * P * P / (cms * 1e-3),
                         "useful_tops": corr_useful_ops(C, T, N, P) / (cms * 1e-3) / 1e12,
                         "roofline": {"bound": "tensor", "achieved": mma / (cms * 1e-3) / 1e12, "peak": pk,
                                      "unit": "TFLOP/s", "frac": mma / (cms * 1e-3) / 1e12 / pk,
                                      "peak_source": "of measured bf16_tflops (fp16 nominal ratio 1)"}}
    out["xfft"] = {"ms": xms, "units_per_s": units / (xms * 1e-3),
                   "note": "per cadence after the correlator; XFFT cadence = correlator + xfft"}
    out["xfft_total_units_per_s"] = units / ((cms + xms) * 1e-3)
    out["paper_cost"] = paper_cost("SKA-low", "intra", C, T, out["fp16"]["ms"])
    hai.hai_layout_destroy(lay)
    del vis, volt, img, vh, ih
    return out


def hierarchy_component(hai, ctx, flush, peaks):
    """The hierarchical workload's cadence: 256 stations x 256 elements, 32
    channels, 2 pols, 1000 samples; int8 beamforming to 16 beams per station
    with requantisation, beams to correlator layout, the station correlator
    (32,896 pairs per beam and channel) and the FP64-steered XFFT on a 256^2
    station grid.  Uniform random int8 voltages (times do not depend on the
    values); units = station-image pixels x beams x channels x pols x samples."""
    import torch
    from paper_2411_17804_gb300 import inputs as I
    H = I.HierarchyConfig()
    S, C, T, K, P, ne, n = H.n_station, H.n_chan, H.n_time, H.n_beam, H.n_pol, H.station.n_elem, H.grid_n
    g = torch.Generator(device="cuda").manual_seed(13)
    volt = torch.randint(-128, 128, (S, C, T, P, ne, 2), dtype=torch.int8, device="cuda", generator=g)
    elem = I.station_layout(H.station)
    centres = I.station_centres(H)
    dirs = I.beam_directions(K, H.station.lam_m, H.station.diameter_m)
    w = torch.from_numpy(np.repeat(I.bf_weights(elem, H.station.lam_m, dirs, P)[None], S, axis=0)).cuda()
    lay = hai.hai_vis_layout_create(ctx, centres, H.station.lam_m, H.cell_m, n, dirs)
    beams = torch.empty((S, C, T, K, P, 2), dtype=torch.int8, device="cuda")
    cin = torch.empty((K, C, T, P, S, 2), dtype=torch.int8, device="cuda")
    vis = torch.empty((K * C, S * (S + 1) // 2, P, P, 2), dtype=torch.int32, device="cuda")
    img = torch.empty((K * C, 4, n, n), device="cuda")
    sat = torch.zeros(1, dtype=torch.int64, device="cuda")
    stages = {
        "beamform_requant": lambda st: hai.hai_beamform(ctx, volt, w, S, C, T, K, ne, P, H.requant_shift, beams, sat, st),
        "beams_to_corr": lambda st: hai.hai_beams_to_corr(ctx, beams, S, C, T, K, P, cin, st),
        "station_correlator": lambda st: hai.hai_correlate(ctx, cin.view(K * C, T, P, S, 2), K * C, T, S, P, vis, 0, st),
        "station_xfft": lambda st: hai.hai_xfft_station_image(ctx, lay, vis, C, img, st)}
    ms = {k: time_call(f, 5, 2, flush) for k, f in stages.items()}
    total = time_call(lambda st: [f(st) for f in stages.values()], 5, 2, flush)
    # the coherent inter-station alternative on the same beams: EPIC over the
    # stations (FP64-steered 1-cell weights, 128^2 array grid = padding 2 on
    # the 1 km core), tensor cores, one launch per beam direction
    ne_grid = 128
    elays = [hai.hai_station_epic_layout_create(ctx, centres, H.station.lam_m, H.cell_m, ne_grid, dirs, k, P)
             for k in range(K)]
    eimg = torch.empty((K, C, 4, ne_grid, ne_grid), device="cuda")

    def station_epic(st):
        for k in range(K):
            hai.hai_epic_image(ctx, elays[k][0], cin[k], C, T, hai.HAI_PREC_FP16, eimg[k], 0, st)

    ems = time_call(station_epic, 5, 2, flush)
    units = n * n * K * C * P * T
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    pk = float(peaks.get("bf16_tflops", 1900.0))
    bf_bytes = volt.numel() + w.numel() + beams.numel()
    tr_bytes = 2 * beams.numel()
    mma = corr_mma_flops(K * C, T, S, P)
    out = {"workload": H.name, "stations": S, "elements": ne, "channels": C, "samples": T, "beams": K,
           "station_grid": n, "pairs_off_grid": hai.hai_vis_layout_offgrid(lay),
           "stage_ms": ms, "ms": total, "units_per_s": units / (total * 1e-3), "unit": UNIT,
           "roofline": {
               "beamform_requant": {"bound": "hbm", "achieved": bf_bytes / (ms["beamform_requant"] * 1e-3) / 1e9,
                                    "peak": hbm, "unit": "GB/s"},
               "beams_to_corr": {"bound": "hbm", "achieved": tr_bytes / (ms["beams_to_corr"] * 1e-3) / 1e9,
                                 "peak": hbm, "unit": "GB/s"},
               "station_correlator": {"bound": "tensor", "achieved": mma / (ms["station_correlator"] * 1e-3) / 1e12,
                                      "peak": pk, "unit": "TFLOP/s"}}}
    for r in out["roofline"].values():
        r["frac"] = r["achieved"] / r["peak"]
    # XBF of the pairs the station grid drops (the 65 km tail), added onto the
    # XFFT image: one tensor-core GEMM against the layout's geometry phases
    xl = hai.hai_xbf_layout_create(ctx, centres, H.station.lam_m, H.cell_m, n, dirs, hai.HAI_XBF_OFFGRID_PAIRS, C,
                                   hai.HAI_PREC_FP16)
    xpairs, xbytes = hai.hai_xbf_layout_info(xl)
    xms = time_call(lambda st: hai.hai_xbf_station_image(ctx, xl, vis, C, img, 1, st), 5, 2, flush)
    rows = K * C * 4
    kd = -(-2 * xpairs // 64) * 64
    xflop = 2.0 * (-(-rows // 128) * 128) * kd * n * n
    out_xbf = {"what": "XBF of the pairs the station grid drops, accumulated onto the XFFT image",
               "pairs": xpairs, "phase_bytes": xbytes, "ms": xms,
               "roofline": {"bound": "tensor", "achieved": xflop / (xms * 1e-3) / 1e12, "peak": pk,
                            "unit": "TFLOP/s", "frac": xflop / (xms * 1e-3) / 1e12 / pk,
                            "flop": xflop}}
    hai.hai_xbf_layout_destroy(xl)
    # the same with hi/lo split operands (FP32-level accuracy, three times the work)
    xs = hai.hai_xbf_layout_create(ctx, centres, H.station.lam_m, H.cell_m, n, dirs, hai.HAI_XBF_OFFGRID_PAIRS, C,
                                   hai.HAI_PREC_FP16_SPLIT)
    xsms = time_call(lambda st: hai.hai_xbf_station_image(ctx, xs, vis, C, img, 1, st), 5, 2, flush)
    hai.hai_xbf_layout_destroy(xs)
    out_xbf["split"] = {"ms": xsms, "roofline": {"bound": "tensor", "achieved": 3 * xflop / (xsms * 1e-3) / 1e12,
                                                 "peak": pk, "unit": "TFLOP/s",
                                                 "frac": 3 * xflop / (xsms * 1e-3) / 1e12 / pk}}
    emma = plan_mma_flops(ne_grid) * K * C * T
    out["station_xbf_offgrid"] = out_xbf
    out["station_epic"] = {
        "what": "inter-station EPIC on the same requantised beams (alternative to correlator + XFFT)",
        "grid": ne_grid, "stations_dropped": elays[0][1], "ms": ems,
        "units_per_s": ne_grid * ne_grid * K * C * P * T / (ems * 1e-3),
        "roofline": {"bound": "tensor", "achieved": emma / (ems * 1e-3) / 1e12, "peak": pk, "unit": "TFLOP/s",
                     "frac": emma / (ems * 1e-3) / 1e12 / pk}}
    # inter-station stage of the paper's SKA-low-core (256 stations), per beam
    out["paper_cost_inter_station"] = paper_cost("SKA-low-core", "inter", C * K, T,
                                                 ms["station_correlator"] + ms["station_xfft"], "XFFT")
    out["paper_cost_inter_station"]["measured_epic_ms"] = ems
    out["paper_cost_inter_station"]["measured_xbf_offgrid_ms"] = xms
    for lay_k, _ in elays:
        hai.hai_layout_destroy(lay_k)
    del eimg
    hai.hai_vis_layout_destroy(lay)
    del volt, w, beams, cin, vis, img
    return out


def run_case(name):
    """Small cases sized for full ncu captures (inputs above L2, a few GB at most)."""
    import torch
    from paper_2411_17804_gb300 import hai, inputs as I
    ctx = hai.hai_create(0)
    if name in ("plan_hier", "plan_hier128"):   # the uneven array's plan with its second level (all stations,
        cfg = I.UnevenConfig()                   # or the first 128 for full captures: ~1 GB of voltages)
        if name == "plan_hier128":
            cfg.n_station = 128
        lays = []
        for i in range(cfg.n_station):
            sc = I.uneven_station(cfg, i)
            an, tp = I.station_kernel(sc, I.station_layout(sc))
            lays.append(hai.hai_layout_create(ctx, an, tp, sc.grid_n, 2))
        plan = hai.hai_plan_create(ctx, lays, cfg.n_chan, cfg.n_time)
        for ly in lays:
            hai.hai_layout_destroy(ly)
        g = torch.Generator(device="cuda").manual_seed(12)
        volt = torch.randint(-128, 128, (plan.volt_bytes,), dtype=torch.int8, device="cuda", generator=g)
        img = torch.empty((plan.img_floats,), device="cuda")
        flush = torch.empty(64 << 20, device="cuda")
        hai.hai_plan_autotune(plan, volt, img, 1)
        plan_hierarchy(hai, ctx, plan, cfg, volt, img, flush, 2, 0.0, 1)
        hai.hai_plan_destroy(plan)
    elif name == "bf":                    # 16 stations of the hierarchical shape: 525 MB of voltages
        S, C, T, K, N, P = 16, 32, 1000, 16, 256, 2
        g = torch.Generator(device="cuda").manual_seed(1)
        v = torch.randint(-128, 128, (S, C, T, P, N, 2), dtype=torch.int8, device="cuda", generator=g)
        w = torch.randint(-127, 128, (S, K, P, N, 2), dtype=torch.int8, device="cuda", generator=g)
        out = torch.empty((S, C, T, K, P, 2), dtype=torch.int8, device="cuda")
        for _ in range(2):
            hai.hai_beamform(ctx, v, w, S, C, T, K, N, P, 11, out)
    elif name in ("tc64", "fp32_64", "corr"):   # the SKA-low station: 16 channels (33.6 MB) for the EPIC
        cfg = I.SKA_LOW_STATION_256               # cases (tensor cores, FP32), 64 for corr
        pos = I.station_layout(cfg)
        an, tp = I.station_kernel(cfg, pos)
        C = cfg.n_chan if name == "corr" else 16
        v = I.station_voltages(cfg, pos, device="cuda", n_chan=C)
        if name != "corr":
            prec = hai.HAI_PREC_FP16 if name == "tc64" else hai.HAI_PREC_FP32
            lay = hai.hai_layout_create(ctx, an, tp, 64, 2)
            img = torch.empty((C, 4, 64, 64), device="cuda")
            for _ in range(2):
                hai.hai_epic_image(ctx, lay, v, C, cfg.n_time, prec, img, 0)
        else:
            N = cfg.n_elem
            vis = torch.empty((C, N * (N + 1) // 2, 2, 2, 2), dtype=torch.int32, device="cuda")
            for _ in range(2):
                hai.hai_correlate(ctx, v, C, cfg.n_time, N, 2, vis, 0)
    elif name == "xfft":                  # correlator + XFFT of the 64-channel SKA-low cadence
        cfg = I.SKA_LOW_STATION_256
        pos = I.station_layout(cfg)
        an, tp = I.station_kernel(cfg, pos)
        C, N = cfg.n_chan, cfg.n_elem
        v = I.station_voltages(cfg, pos, device="cuda", n_chan=C)
        lay = hai.hai_layout_create(ctx, an, tp, cfg.grid_n, 2)
        vis = torch.empty((C, N * (N + 1) // 2, 2, 2, 2), dtype=torch.int32, device="cuda")
        img = torch.empty((C, 4, cfg.grid_n, cfg.grid_n), device="cuda")
        for _ in range(2):
            hai.hai_correlate(ctx, v, C, cfg.n_time, N, 2, vis, 0)
            hai.hai_xfft_image(ctx, lay, vis, C, img, 0)
        torch.cuda.synchronize()
        hai.hai_layout_destroy(lay)
    elif name == "tc128":                 # a 700-element station of the uneven array, N = 128
        sc = I.uneven_station(I.UnevenConfig(), 0, 700)
        pos = I.station_layout(sc)
        an, tp = I.station_kernel(sc, pos)
        lay = hai.hai_layout_create(ctx, an, tp, 128, 2)
        C, T = 36, 256
        v = I.random_voltages((C, T, 2, len(pos), 2), seed=5, device="cuda")
        img = torch.empty((C, 4, 128, 128), device="cuda")
        for _ in range(2):
            hai.hai_epic_image(ctx, lay, v, C, T, hai.HAI_PREC_FP16, img, 0)
    elif name == "xbf":                   # the hierarchical array's dropped pairs, 4 beams x 8 channels
        H = I.HierarchyConfig()
        centres = I.station_centres(H)
        S, n, K, C = len(centres), H.grid_n, 4, 8
        dirs = I.beam_directions(H.n_beam, H.station.lam_m, H.station.diameter_m)[:K]
        g = torch.Generator(device="cuda").manual_seed(3)
        vis = torch.randint(-2**20, 2**20, (K * C, S * (S + 1) // 2, 2, 2, 2), dtype=torch.int32, device="cuda",
                            generator=g)
        xl = hai.hai_xbf_layout_create(ctx, centres, H.station.lam_m, H.cell_m, n, dirs, hai.HAI_XBF_OFFGRID_PAIRS, C,
                                   hai.HAI_PREC_FP16)
        img = torch.empty((K * C, 4, n, n), device="cuda")
        for _ in range(2):
            hai.hai_xbf_station_image(ctx, xl, vis, C, img, 0)
        torch.cuda.synchronize()
        hai.hai_xbf_layout_destroy(xl)
    elif name == "sxfft":                 # station XFFT of the hierarchical cadence: 16 beams x 32 channels
        H = I.HierarchyConfig()
        centres = I.station_centres(H)
        S, n, K, C = len(centres), H.grid_n, H.n_beam, 32
        dirs = I.beam_directions(H.n_beam, H.station.lam_m, H.station.diameter_m)
        g = torch.Generator(device="cuda").manual_seed(4)
        vis = torch.randint(-2**20, 2**20, (K * C, S * (S + 1) // 2, 2, 2, 2), dtype=torch.int32, device="cuda",
                            generator=g)
        vl = hai.hai_vis_layout_create(ctx, centres, H.station.lam_m, H.cell_m, n, dirs)
        img = torch.empty((K * C, 4, n, n), device="cuda")
        for _ in range(2):
            hai.hai_xfft_station_image(ctx, vl, vis, C, img)
        torch.cuda.synchronize()
        hai.hai_vis_layout_destroy(vl)
    elif name in ("big", "big16", "big2"):   # the dense lattice on tensor cores: 4 ch x 20 samples, 16 ch x
        cfg = I.DENSE_ALLSKY_16384           # 100, or one batch of the autotuned headline (2 ch x 409 samples:
        pos = I.station_layout(cfg)          # one launch of each kernel, as in the benchmark's steps)
        an, tp = I.station_kernel(cfg, pos)
        lay = hai.hai_layout_create(ctx, an, tp, 512, 2)
        C, T = {"big": (4, 20), "big16": (16, 100), "big2": (2, 409)}[name]
        v = I.random_voltages((C, T, 2, len(pos), 2), seed=5, device="cuda")
        img = torch.empty((C, 4, 512, 512), device="cuda")
        for _ in range(2):
            hai.hai_epic_image(ctx, lay, v, C, T, hai.HAI_PREC_FP16, img, 0)
    elif name == "fc":                    # FFT correlator on 16 channels of 512^2 images (67 MB in)
        img = torch.randn((16, 4, 512, 512), device="cuda")
        grid = torch.empty((16, 2, 2, 512, 512, 2), device="cuda")
        for _ in range(2):
            hai.hai_fft_correlate(ctx, img, 16, 512, 2, grid)
    torch.cuda.synchronize()
    hai.hai_destroy(ctx)
    print(json.dumps({"case": name, "ok": True}))


def main():
    args = parse()
    if args.case:
        run_case(args.case)
        return
    ws, rank, local = dist_init(args.gpus)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    from paper_2411_17804_gb300 import hai, inputs as I
    torch.cuda.set_device(local)
    cfg, pos, anchors, taps = workload(args.samples)
    if args.channels:
        import dataclasses
        cfg = dataclasses.replace(cfg, n_chan=args.channels)
    C, T, P, n = cfg.n_chan, cfg.n_time, cfg.n_pol, cfg.grid_n
    prec = PRECS[args.prec]
    chan0, _ = rank_channels(rank, C)
    volt = I.station_voltages(cfg, pos, device="cuda", chan0=chan0)
    ctx = hai.hai_create(local)
    lay = hai.hai_layout_create(ctx, anchors, taps, n, P)
    img = torch.empty((C, lay.n_planes, n, n), device="cuda")
    flush = torch.zeros(64 * 1024 * 1024, device="cuda")       # 256 MB > L2
    hai.hai_profile_enable(ctx, True, 1 << 16)
    units = cfg.units_per_cadence
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    probes = probe_peaks(hai, ctx)
    # the autotuner picks the channels per internal chunk of the large-grid
    # tensor path for this cadence (timed on a synthetic cadence, cached)
    tune_cache = os.environ.get("HAI_TUNE_CACHE") or os.path.join(tempfile.gettempdir(), "hai_autotune.txt")
    tuned = hai.hai_autotune(ctx, lay, C, T, prec, tune_cache) if prec != 0 else 0

    clocks = Clocks(local)
    clocks.start()
    total_ms, dom_ms, launches = time_epic(hai, ctx, lay, volt, img, C, T, prec, args.steps,
                                           args.warmup, flush, ws)
    clk = clocks.stop()
    total_ms = max_over_ranks(total_ms, ws)
    ms_step = total_ms / args.steps
    value = job_value(ws, units, ms_step)
    dom_per_step = dom_ms / args.steps                         # stage-2 (or FP32) kernel time per step

    # end to end through the C ABI with host buffers (pinned): hai_epic_image_host
    # copies every voltage in and every image out inside the call, chunks of
    # C/4 channels overlapping their copies with the imaging
    vh = volt.cpu().pin_memory()
    ih = torch.empty(img.shape, dtype=torch.float32).pin_memory()
    st = torch.cuda.current_stream()
    hai.hai_epic_image_host(ctx, lay, vh, C, T, prec, ih, 0, 0, st)
    torch.cuda.synchronize()
    barrier(ws)
    e0 = time.perf_counter()
    e_steps = 3
    for _ in range(e_steps):
        hai.hai_epic_image_host(ctx, lay, vh, C, T, prec, ih, 0, 0, st)
    torch.cuda.synchronize()
    e_ms = max_over_ranks((time.perf_counter() - e0) * 1e3 / e_steps, ws)
    hai.hai_profile_read(ctx)

    x0, y0, x1, y1 = hai.hai_layout_box(lay)
    R, Cnz = y1 - y0, x1 - x0
    fields = C * T * P
    pkt = float(peaks.get("bf16_tflops", 1900.0))
    split = 3 if args.prec.endswith("split") else 1
    if prec != hai.HAI_PREC_FP32:
        s2 = stage2_flop(n, R) * fields * split
        ach = s2 / (dom_per_step * 1e-3) / 1e12
        whole = pruned_dft_flop(n, R, Cnz) * fields * split / (ms_step * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": pkt, "unit": "TFLOP/s", "frac": ach / pkt,
                "traffic": None, "kernel": "big_s2_kernel",
                "peak_source": "of measured: MEASURED_PEAKS bf16_tflops (burst) x fp16/bf16 nominal ratio 1"
                               if "bf16_tflops" in peaks else "of fallback 1.9 PFLOP/s",
                "flop_per_field": stage2_flop(n, R) * split,
                "basis": f"stage 2 of the pruned DFT of the {Cnz} x {R} kernel box: 8 N^2 R per field "
                         f"(x{split} products), {fields} fields per step",
                "kernel_ms_per_step": dom_per_step,
                "whole_path": {"achieved": whole, "frac": whole / pkt,
                               "basis": "8 (R N C + N^2 R) per field over the step time (all kernels)"}}
    else:
        peak = probes["fp32_tflops"]
        achieved = epic_flops_per_unit(cfg) * units / (dom_per_step * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "epic_large (row and column FFT kernels)",
                "peak_source": "measured: hai_probe_peak FP32 FMA (best of scalar and packed)",
                "flop_per_unit": epic_flops_per_unit(cfg)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == hai.HAI_PREC_FP32 else args.prec[:4],
            "data": "synthetic", "config": dict(headline_config(cfg, args.prec, ws),
                                                autotuned={"channels_per_chunk": tuned, "cache": tune_cache}),
            "e2e": {"value": ws * units / (e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": int(volt.numel()), "d2h_bytes_per_step": int(img.numel() * 4),
                    "api": "hai_epic_image_host (host buffers, chunks of C/4 channels)"},
            "gpu_launches": int(launches), "clocks": clk, "roofline": roof, "probed_peaks": probes}
    # every operand form on the same cadence: the metric's comparison with
    # plain FP32 on CUDA cores, and the bf16 / split forms
    if not args.no_fp32_compare:
        forms = {}
        for name, pr in PRECS.items():
            if pr == prec:
                continue
            ns = 2 if pr == hai.HAI_PREC_FP32 else 3
            tf, df, _ = time_epic(hai, ctx, lay, volt, img, C, T, pr, ns, 1, flush, ws)
            forms[name] = {"value": ws * units / (tf / ns * 1e-3), "unit": UNIT, "ms_per_step": tf / ns}
        forms[args.prec] = {"value": value, "unit": UNIT, "ms_per_step": ms_step}
        line["by_precision"] = forms
        if "fp32" in forms and prec != hai.HAI_PREC_FP32:
            f32 = forms["fp32"]
            f32["roofline"] = {"bound": "alu", "unit": "TFLOP/s", "peak": probes["fp32_tflops"],
                               "achieved": epic_flops_per_unit(cfg) * units / (f32["ms_per_step"] * 1e-3) / 1e12,
                               "flop_per_unit": epic_flops_per_unit(cfg),
                               "basis": "FFT-equivalent work 5 log2(N^2) + gridding + squaring per unit, "
                                        "over the step time; peak measured by hai_probe_peak"}
            f32["roofline"]["frac"] = f32["roofline"]["achieved"] / f32["roofline"]["peak"]
            line["plain_fp32"] = f32
            line["tc_over_fp32"] = value / f32["value"]
    line["paper_cost"] = {"note": "the dense lattice is not a Table 1 array; see components.ska_station.paper_cost"}
    if not args.no_components:
        hai.hai_epic_image(ctx, lay, volt, C, T, prec, img, 0, st)
        line["components"] = {"fft_correlator": fft_correlator_component(hai, ctx, img, C, n, P, flush, peaks)}
        del volt, vh, ih
        torch.cuda.empty_cache()
        line["components"]["ska_station"] = ska_component(hai, ctx, flush, peaks, sms, 20,
                                                          probes.get("fp32_tflops"))
        line["components"]["beamformer"] = bf_component(hai, ctx, flush, peaks)
        line["components"]["batched_uneven"] = plan_component(hai, ctx, flush, peaks, 10)
        line["components"]["hierarchical"] = hierarchy_component(hai, ctx, flush, peaks)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # one channel of the cadence: every precision's GPU image of it against
        # the oracle's, which is also the timed CPU baseline
        v1 = I.station_voltages(cfg, pos, device="cuda", n_chan=1, chan0=chan0)
        i1 = torch.empty((1, 4, n, n), device="cuda")
        imgs = {}
        for name, pr in PRECS.items():
            hai.hai_epic_image(ctx, lay, v1, 1, T, pr, i1, 0, st)
            torch.cuda.synchronize()
            imgs[name] = i1.cpu().numpy()
        cb, errs = cpu_baseline(cfg, anchors, taps, v1.cpu().numpy(), gpu_imgs=imgs)
        line["cpu_baseline"] = cb
        line["image_error_vs_oracle"] = errs[args.prec]
        line["image_error_by_precision"] = {k: {"max": v["max"], "median": v["median"], "pixel_max": v["pixel_max"]}
                                            for k, v in errs.items()}
    hai.hai_layout_destroy(lay)
    hai.hai_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
