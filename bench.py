"""Benchmark of the pixel-space convolution hot path (one JSON line on rank 0).

Default workload (the single-detector FP32 configuration): HEALPix nside 512
I, Q, U sky (Gaussian field, C_l ~ l^-2, Q and U at 10 % of the I rms), one
detector with a 1.5 deg FWHM Gaussian main beam, a 1 % sidelobe ring at
6-8 deg and 0.5 % cross-polar leakage, six beam maps on a 501 x 501 grid of
radius 10 deg, 1e7 samples of a 45 deg elevation azimuth scan at 1 deg/s,
20 Hz, with the boresight rotated daily through 7 angles.

A step is one pisco_convolve over all samples (inputs resident in HBM; the
1e7 pointings are 240 MB, larger than L2).  Also reported: the same metric
end to end through pisco_convolve_host (pinned host buffers, copies inside
the timed region), the plain FP64 GPU path on a contiguous slice, the
roofline of the convolution kernel, and the FP64 CPU oracle on a bounded
slice (cpu_baseline).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1908_05662_gb300 import beams  # noqa: E402
from paper_1908_05662_gb300 import pisco  # noqa: E402
from paper_1908_05662_gb300 import synthetic as sy  # noqa: E402

METRIC = "TOD samples/s (single-detector FP32 path, nside 512, R 10 deg, 501^2 beam grid)"
UNIT = "samples/s"

WORKLOAD = dict(workload="single-detector FP32: nside 512 sky, 1.5 deg beam + 1% sidelobe ring at 6-8 deg "
                         "+ 0.5% cross-polar, 6 maps on 501x501 grid of radius 10 deg, 1e7 samples of a "
                         "45 deg elevation azimuth scan",
                nside=512, radius_deg=10.0, grid_n=501, n_samples=10_000_000, tile_samples=16,
                pixels_per_thread=1)

# FP32 operations per in-disc (sample, pixel) pair in the forward kernel's inner loop
# (FMA = 2): half-angle rotation 7, disc test 3, in-frame offsets 11, grid index 10,
# three bilinear maps 18, Ludwig-3 angle 15, Stokes rotation and accumulation 14.
FLOPS_PER_PAIR = 78
# FP32 peak of the GPU from unit counts: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
def measured_peaks(path=os.path.join(ROOT, "MEASURED_PEAKS.json")):
    """(HBM GB/s, dense BF16 TFLOP/s burst, source): the copy bandwidth and cuBLAS BF16 rate
    measured on this machine's GPUs when the file is there, else the fallback figures."""
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, 1900.0, "fallback"


HBM_GBS, BF16_TFLOPS, PEAK_SOURCE = measured_peaks()

# Recorded ncu figures of the forward launch on the default single-detector workload, keyed by
# (samples, tile_samples, pixels_per_thread) with 64-byte cells; they are not measured by this run:
# * traffic: dram__bytes_read.sum + dram__bytes_write.sum of one full-size launch (1 pass):
#   486.63 MB read, 47.03 MB written.  Pointing (240 MB) and TOD (40 MB) stream through once; the
#   rest is the L2-resident sky and beam cells, some re-read after the pointing stream evicts them;
# * l1tex / lts: l1tex__throughput.avg.pct_of_peak_sustained_active and
#   lts__throughput.avg.pct_of_peak_sustained_elapsed of the same kernel shape on a 5e5-sample
#   slice (profiles/k_fast_forward_single_detector.md): the unit that binds is the L1/TEX path
#   serving scattered 32-byte sectors of beam cells.
FORWARD_PROFILE = {(10_000_000, 16, 1): {"traffic": 486.63e6 + 47.03e6, "l1tex_pct": 93.1, "lts_pct": 78.1}}

# Recorded ncu figures of the multi-realization kernel (BF16, 256 realizations) on a 2e5-sample
# slice of its workload (profiles/k_mr_multirealization.md), not measured by this run: the tensor
# pipe's busy fraction (it issues the hi and lo weight parts, twice the algorithmic flops) and the
# warp schedulers' issue rate, which show that the FP32 weight producers, not the tensor cores, bind.
MR_PROFILE = {"tensor_pipe_pct": 20.1, "issue_per_cycle": 0.57, "l1tex_pct": 65.3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pisco", choices=["pisco", "reference"])
    ap.add_argument("--samples", type=int, default=WORKLOAD["n_samples"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline leg")
    ap.add_argument("--workload", default="single",
                    choices=["single", "c1", "focalplane", "multireal", "table1", "psb", "sec61", "grad"],
                    help="single: the default single-detector line; the others measure the plain-FP64 baseline "
                         "configuration (c1), the focal-plane, "
                         "multi-realization, Table 1 replica, PSB-pair (shared geometry) and Sec. 6.1 "
                         "(TOD then binned maps) configurations, and grad: the differentiation configuration")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def shard(n, rank, world):
    """Contiguous slice [a, b) of n samples for a rank (scan continuity keeps disc reuse)."""
    a = n * rank // world
    b = n * (rank + 1) // world
    return a, b


def max_over_ranks(value, device):
    """The largest value over all ranks (the timed region is the slowest rank's)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 7 for k in range(4)
                          if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def cached_sky(nside, seed, device):
    """The synthetic sky, kept in a temp-dir file so repeated runs on one machine
    (a plain run, then the same command under a profiler) skip the synthesis."""
    import tempfile
    path = os.path.join(tempfile.gettempdir(), "pisco_bench_cache",
                        f"sky_n{nside}_s{seed}_{torch.device(device).type}.pt")
    if os.path.exists(path):
        return torch.load(path, map_location=device)
    sky = sy.gaussian_sky(nside, seed, device=device)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"  # ranks of one machine may write it at the same time
    torch.save(sky, tmp)
    os.replace(tmp, path)
    return sky


def make_workload(device, n):
    r = math.radians(WORKLOAD["radius_deg"])
    sky = cached_sky(WORKLOAD["nside"], 1, device)
    grids = sy.gaussian_beam_maps(WORKLOAD["grid_n"], r, 1.5, ellipticity=0.0, xpol=0.005,
                                  sidelobe=(0.01, 7.0, 0.5))
    theta, phi, psi = sy.ces_scan(n, device=device)
    return r, sky, grids, (theta.contiguous(), phi.contiguous(), psi.contiguous())


def cpu_oracle_rate(sky, grids, radius, det, theta, phi, psi, n_samples, budget_s=15.0):
    """The FP64 oracle on every host core (one single-threaded worker process each) for ~budget_s;
    worker j takes consecutive samples from j * n / cores.  Returns (rate, index, outputs, cores)."""
    from oracle import beam as ob
    from oracle import parallel as op
    g64 = np.asarray(grids, np.float64)
    omega = ob.omega_tilde(g64[0], radius)
    skyn = sky if isinstance(sky, np.ndarray) else sky.cpu().numpy()
    m = min(n_samples, 4096 * op.host_cores())  # more than a worker finishes in the budget
    idx, outs, span, cores = op.tod_sampled(WORKLOAD["nside"], radius, skyn, g64, det, omega, theta[:m], phi[:m],
                                            psi[:m], budget_s=budget_s)
    return len(idx) / span, idx, outs, cores


def run_reference(args, rank, world):
    """The oracle as it stands, timed on this host's cores, on the same workload."""
    if rank != 0:
        return
    torch.set_num_threads(1)
    n = 2000
    # inputs are made on the GPU when there is one (the synthesis is slow on the host)
    gen_dev = "cuda" if torch.cuda.is_available() else "cpu"
    r, sky, grids, (th, ph, ps) = make_workload(gen_dev, n)
    sky, th, ph, ps = sky.cpu(), th.cpu(), ph.cpu(), ps.cpu()
    thn, phn, psn = th.numpy(), ph.numpy(), ps.numpy()
    det = (0.0, 0.0, 1.0)
    from oracle import beam as ob
    from oracle import parallel as op
    g64 = grids.astype(np.float64)
    omega = ob.omega_tilde(g64[0], r)
    skyn = sky.numpy()
    cores = op.host_cores()
    per_worker = 8
    per_step = cores * per_worker
    times = []
    for step in range(args.warmup + args.steps):
        a = (step * per_step) % (n - per_step)
        # each worker takes per_worker consecutive samples of this step's slice; the step time is the
        # span of the workers' loops (interpreter start-up excluded)
        idx, _, span, used = op.tod_sampled(WORKLOAD["nside"], r, skyn, g64, det, omega, thn[a:a + per_step],
                                            phn[a:a + per_step], psn[a:a + per_step], processes=cores,
                                            budget_s=1e9, max_per_worker=per_worker)
        assert len(idx) == per_step and used == cores
        if step >= args.warmup:
            times.append(span)
    ms = 1e3 * statistics.mean(times)
    value = per_step / (ms / 1e3)
    sample = f"{per_step} consecutive scan samples per step, {per_worker} per worker process"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["workload"], "oracle_sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _event_time(fn, steps, warmup, stream):
    """Mean device time (ms) of fn() over ``steps`` runs after ``warmup`` runs, CUDA events on ``stream``."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_c1(args, dev):
    """The plain-FP64 baseline configuration: nside 128 sky, elliptical Gaussian beam (FWHM 1.5 deg,
    ellipticity 0.05) as 6 maps on a 101^2 grid of radius 5 deg, 1e5 samples of a constant-elevation
    raster with psi stepping uniformly over [0, 2 pi).  One step = one pisco_convolve over all samples
    (FP32 path, tile shape from the autotuner); the plain FP64 path runs the whole scan too, the
    packed-cell fetch beside it, and the oracle on a bounded sample of the scan on every host core."""
    nside, r, n_grid = 128, math.radians(5.0), 101
    n = 100_000 if args.samples == WORKLOAD["n_samples"] else args.samples
    sky = cached_sky(nside, 1, dev)
    grids = sy.gaussian_beam_maps(n_grid, r, 1.5, ellipticity=0.05)
    g = torch.as_tensor(grids, device=dev)[None].contiguous()
    th, ph, ps = (torch.as_tensor(a, device=dev).contiguous() for a in sy.raster_scan(n, rows=100))
    det = (0.0, 0.0, 1.0)
    stream = torch.cuda.current_stream()
    plan = pisco.Plan(nside, r, sky, [det], g)
    tuned = plan.autotune(th, ph, ps, reps=3)
    pairs = int(plan.disc_count(th, ph).to(torch.int64).sum().item())
    tod = torch.empty(n, dtype=torch.float32, device=dev)
    with ClockSampler(torch.cuda.current_device()) as clocks:
        ms = _event_time(lambda: plan.convolve(th, ph, ps, out=tod), args.steps, args.warmup, stream)
    plan.sync_status()
    legs = {}
    for name, fetch in (("packed_cells", pisco.PISCO_FETCH_PACKED), ("shared_nodes", pisco.PISCO_FETCH_SHARED)):
        with pisco.Plan(nside, r, sky, [det], g, beam_fetch=fetch, tile_samples=tuned[0],
                        pixels_per_thread=tuned[1]) as other:
            t_o = torch.empty(n, dtype=torch.float32, device=dev)
            ms_o = _event_time(lambda: other.convolve(th, ph, ps, out=t_o), args.steps, args.warmup, stream)
            other.sync_status()
        legs[name] = (ms_o, t_o)
    with pisco.Plan(nside, r, sky, [det], g, precision=pisco.PISCO_FP64_PLAIN) as plain:
        tod64 = torch.empty(n, dtype=torch.float64, device=dev)
        ms_plain = _event_time(lambda: plain.convolve(th, ph, ps, out=tod64), 2, 1, stream)
        plain.sync_status()
    fp32_vs_64 = ((tod.double() - tod64).abs().max() / tod64.abs().max()).item()
    out = {"metric": "TOD samples/s (plain-FP64 baseline configuration: nside 128, R 5 deg, 101^2 grid)",
           "value": n / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "nside 128 sky, FWHM 1.5 deg e 0.05 beam, 101^2 grid of radius 5 deg, "
                                  "1e5 raster samples", "samples": n, "pairs_per_step": pairs,
                      "tile_samples": tuned[0], "pixels_per_thread": tuned[1],
                      "l2": "inputs (2.4 MB pointing, 3 MB sky, 0.6 MB beam) are L2-resident"},
           "plain_fp64_gpu": {"value": n / (ms_plain / 1e3), "unit": UNIT, "ms_per_step": ms_plain,
                              "samples_timed": n, "speedup_of_fp32": ms_plain / ms,
                              "fp32_vs_fp64_normwise": fp32_vs_64},
           "roofline": {"bound": "alu", "achieved": FLOPS_PER_PAIR * pairs / (ms / 1e3) / 1e12,
                        "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": FLOPS_PER_PAIR * pairs / (ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS, "traffic": None},
           "gpu_launches": args.steps, "clocks": clocks.summary()}
    for name, (ms_o, t_o) in legs.items():
        out[name] = {"value": n / (ms_o / 1e3), "unit": UNIT, "ms_per_step": ms_o,
                     "vs_default_normwise": ((t_o.double() - tod.double()).abs().max() /
                                             tod.double().abs().max()).item()}
    if not args.no_cpu:
        thn, phn, psn = th.cpu().numpy(), ph.cpu().numpy(), ps.cpu().numpy()
        from oracle import beam as ob
        from oracle import parallel as op
        g64 = grids.astype(np.float64)
        idx, ref, span, cores = op.tod_sampled(nside, r, sky.cpu().numpy(), g64, det, ob.omega_tilde(g64[0], r),
                                               thn, phn, psn, budget_s=10.0)
        sel = torch.as_tensor(idx, device=dev)
        out["cpu_baseline"] = {"value": len(idx) / span, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{len(idx)} samples: {cores} single-threaded worker processes, "
                                         "each ~10 s on consecutive samples from its own offset"}
        out["err_vs_oracle_normwise"] = float(np.max(np.abs(tod[sel].double().cpu().numpy() - ref)) /
                                              np.max(np.abs(ref)))
        out["plain_fp64_gpu"]["err_vs_oracle_normwise"] = float(
            np.max(np.abs(tod64[sel].cpu().numpy() - ref)) / np.max(np.abs(ref)))
        for name, (_, t_o) in legs.items():
            out[name]["err_vs_oracle_normwise"] = float(np.max(np.abs(t_o[sel].double().cpu().numpy() - ref)) /
                                                        np.max(np.abs(ref)))
    plan.close()
    print(json.dumps(out))


def run_focalplane(args, dev):
    """64 detectors, focal-plane offsets within +-10 deg, FWHM 1.2-1.8 deg, ellipticity 0-0.1, own
    201^2 grids of radius 6 deg, scan lengths uniform in [1e5, 5e6], nside 256 sky: one batched
    launch per step, replayed from a captured CUDA graph."""
    nside, r, n_det = 256, math.radians(6.0), 64
    rng = np.random.default_rng(3)
    lengths = rng.integers(100_000, 5_000_001, n_det)
    if args.samples != WORKLOAD["n_samples"]:
        lengths = np.maximum(1, (lengths * (args.samples / lengths.sum())).astype(np.int64))
    off, fwhm, ell, zeta = sy.focal_plane(n_det, 3)
    sky = cached_sky(nside, 1, dev)
    grids = np.stack([sy.gaussian_beam_maps(201, r, fwhm[d], ellipticity=ell[d]) for d in range(n_det)])
    dets = [(float(zeta[d]), 0.0, 1.0) for d in range(n_det)]
    parts = [sy.ces_scan(int(lengths[d]), offset=tuple(off[d]), device=dev) for d in range(n_det)]
    th, ph, ps = (torch.cat([p[k] for p in parts]).contiguous() for k in range(3))
    del parts
    offsets = [0] + list(np.cumsum(lengths))
    n = int(offsets[-1])
    plan = pisco.Plan(nside, r, sky, dets, torch.as_tensor(grids, device=dev).contiguous())
    # tile shape from the batched autotuner on the first 2e4 samples of every detector (untimed)
    m_tune = 20_000
    tune_idx = torch.cat([torch.arange(offsets[d], offsets[d] + min(m_tune, int(lengths[d])), device=dev)
                          for d in range(n_det)])
    tune_off = [0] + list(np.cumsum([min(m_tune, int(x)) for x in lengths]))
    tuned = plan.autotune_batched(tune_off, th[tune_idx].contiguous(), ph[tune_idx].contiguous(),
                                  ps[tune_idx].contiguous(), reps=2)
    pairs = int(plan.disc_count(th, ph).to(torch.int64).sum().item())
    tod = torch.empty(n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    plan.convolve_batched(offsets, th, ph, ps, out=tod)
    torch.cuda.synchronize()
    graph = None
    try:
        s = torch.cuda.Stream()
        s.wait_stream(stream)
        with torch.cuda.stream(s):
            plan.convolve_batched(offsets, th, ph, ps, out=tod)
        stream.wait_stream(s)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            plan.convolve_batched(offsets, th, ph, ps, out=tod)
        step = graph.replay
    except Exception as e:  # capture unavailable: time the eager launch instead
        graph_error = str(e)
        step = lambda: plan.convolve_batched(offsets, th, ph, ps, out=tod)
    with ClockSampler(torch.cuda.current_device()) as clocks:
        ms = _event_time(step, args.steps, args.warmup, stream)
    plan.sync_status()
    # the plain FP64 path (one batched call) on the first 2000 samples of every detector
    m = 2000
    idx = torch.cat([torch.arange(offsets[d], offsets[d] + min(m, int(lengths[d])), device=dev)
                     for d in range(n_det)])
    sub_off = [0] + list(np.cumsum([min(m, int(x)) for x in lengths]))
    thp, php, psp = th[idx].contiguous(), ph[idx].contiguous(), ps[idx].contiguous()
    grids_t = torch.as_tensor(grids, device=dev).contiguous()
    with pisco.Plan(nside, r, sky, dets, grids_t, precision=pisco.PISCO_FP64_PLAIN) as plain:
        tod64 = torch.empty(len(idx), dtype=torch.float64, device=dev)
        ms_plain = _event_time(lambda: plain.convolve_batched(sub_off, thp, php, psp, out=tod64), 2, 1, stream)
        plain.sync_status()
    plain_rate = len(idx) / (ms_plain / 1e3)
    fp32_vs_64 = ((tod[idx].double() - tod64).abs().max() / tod64.abs().max()).item()
    # the FP64 oracle on the first sample of every detector
    from oracle import beam as ob
    from oracle import convolve as oc
    skyn = sky.cpu().numpy()
    first = np.asarray(offsets[:-1], np.int64)
    thn, phn, psn = (a[torch.as_tensor(first, device=dev)].cpu().numpy() for a in (th, ph, ps))
    ref = np.array([oc.tod(nside, r, skyn, grids[d].astype(np.float64), dets[d],
                           ob.omega_tilde(grids[d][0].astype(np.float64), r), thn[d:d + 1], phn[d:d + 1],
                           psn[d:d + 1])[0] for d in range(n_det)])
    got = tod[torch.as_tensor(first, device=dev)].double().cpu().numpy()
    err_oracle = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    achieved = FLOPS_PER_PAIR * pairs / (ms / 1e3) / 1e12
    out = {"metric": "TOD samples/s (64-detector focal plane, nside 256, R 6 deg, 201^2 grids)",
           "value": n / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "focal plane: 64 detectors, offsets +-10 deg, FWHM 1.2-1.8 deg, e 0-0.1, "
                                  "201^2 grids of radius 6 deg, scan lengths U[1e5, 5e6], nside 256",
                      "samples": n, "pairs_per_step": pairs, "launch": "cuda graph" if graph else "eager",
                      "tile_samples": tuned[0], "pixels_per_thread": tuned[1],
                      "tile_shape": "autotuned (pisco_plan_autotune_batched on the first 2e4 samples of every "
                                    "detector)",
                      "l2": "inputs larger than L2"},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None},
           "plain_fp64_gpu": {"value": plain_rate, "unit": UNIT, "samples_timed": len(idx),
                              "sample": f"first {m} samples of each detector, one batched call",
                              "speedup_of_fp32": (n / (ms / 1e3)) / plain_rate,
                              "fp32_vs_fp64_normwise": fp32_vs_64},
           "err_vs_oracle_normwise": err_oracle,
           "oracle_sample": "first sample of each of the 64 detectors",
           "gpu_launches": args.steps, "clocks": clocks.summary()}
    if graph is None:
        out["graph_error"] = graph_error
    plan.close()
    print(json.dumps(out))


def run_multireal(args, dev):
    """256 realizations at nside 256 stored BF16 and FP16 (random combinations of 16 seeded base
    fields, which keeps C_l), one detector, 2e6 samples of the azimuth scan, 1.5 deg Gaussian beam
    of radius 4 deg on a 161^2 grid."""
    nside, r, n_real = 256, math.radians(4.0), 256
    n = 2_000_000 if args.samples == WORKLOAD["n_samples"] else args.samples
    gen = torch.Generator().manual_seed(1000)
    coef = (torch.randn(n_real, 16, generator=gen, dtype=torch.float64) / 4.0).to(dev)
    base = torch.stack([cached_sky(nside, 1000 + k, dev) for k in range(16)])
    exact = torch.einsum("rk,kmp->pmr", coef, base).contiguous()
    del base
    grids = sy.gaussian_beam_maps(161, r, 1.5)
    g = torch.as_tensor(grids, device=dev)[None]
    th, ph, ps = (x.contiguous() for x in sy.ces_scan(n, device=dev))
    det = (0.0, 0.0, 1.0)
    stream = torch.cuda.current_stream()
    results = {}
    for name, precision, dtype in (("bf16", pisco.PISCO_BF16_MR, torch.bfloat16),
                                   ("fp16", pisco.PISCO_FP16_MR, torch.float16)):
        plan = pisco.Plan(nside, r, exact.to(dtype), [det], g, precision=precision)
        out = torch.empty(n, n_real, dtype=torch.float32, device=dev)
        with ClockSampler(torch.cuda.current_device()) as clocks:
            ms = _event_time(lambda: plan.convolve(th, ph, ps, out=out), args.steps, args.warmup, stream)
        plan.sync_status()
        results[name] = (ms, clocks.summary(), out[::20000].double().cpu().numpy())
        plan.close()
    # one realization through the plain FP64 path (first 1e5 samples) and the FP32 path (all
    # samples): the per-realization cost of running the stack through them one by one
    sky0 = exact[:, :, 0].T.contiguous()
    m = min(n, 100_000)
    with pisco.Plan(nside, r, sky0, [det], g, precision=pisco.PISCO_FP64_PLAIN) as plain:
        tod64 = torch.empty(m, dtype=torch.float64, device=dev)
        ms_plain = _event_time(lambda: plain.convolve(th[:m], ph[:m], ps[:m], out=tod64), 2, 1, stream)
        plain.sync_status()
    with pisco.Plan(nside, r, sky0, [det], g) as fp32:
        tod32 = torch.empty(n, dtype=torch.float32, device=dev)
        ms_fp32 = _event_time(lambda: fp32.convolve(th, ph, ps, out=tod32), 2, 1, stream)
        pairs = int(fp32.disc_count(th, ph).to(torch.int64).sum().item())
        fp32.sync_status()
    plain_rate = m / (ms_plain / 1e3) / n_real  # samples/s with all realizations
    fp32_rate = n / (ms_fp32 / 1e3) / n_real
    # error against the FP64 oracle on the unrounded realizations, every 20000th sample
    from oracle import beam as ob
    from oracle import convolve as oc
    g64 = grids.astype(np.float64)
    omega = ob.omega_tilde(g64[0], r)
    idx = np.arange(0, n, 20000)
    thn, phn, psn = th.cpu().numpy(), ph.cpu().numpy(), ps.cpu().numpy()
    ref = np.empty((len(idx), n_real))
    for k, t in enumerate(idx):
        pix, w = oc.sample_weights(nside, r, g64, det, omega, thn[t], phn[t], psn[t])
        ref[k] = np.einsum("km,kmr->r", w, exact[torch.as_tensor(pix, device=dev)].cpu().numpy())
    errs = {k: float(np.max(np.max(np.abs(v[2] - ref), axis=0) / np.max(np.abs(ref), axis=0)))
            for k, v in results.items()}
    ms, clk, _ = results["bf16"]
    algo = 2.0 * 3 * pairs * n_real  # one FMA per (pair, Stokes, realization)
    achieved = algo / (ms / 1e3) / 1e12
    print(json.dumps({
        "metric": "TOD samples/s (256 realizations per sample, BF16 stack, nside 256, R 4 deg)",
        "value": n / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": "multi-realization: 256 realizations at nside 256 (BF16; combinations of 16 "
                               "base fields), 2e6 scan samples, 1.5 deg beam of radius 4 deg, 161^2 grid",
                   "samples": n, "realizations": n_real, "pairs_per_step": pairs},
        "realization_samples_per_s": n * n_real / (ms / 1e3),
        "fp16": {"ms_per_step": results["fp16"][0], "value": n / (results["fp16"][0] / 1e3)},
        "err_vs_oracle_normwise_per_realization": errs,
        "plain_fp64_gpu": {"value": plain_rate, "unit": UNIT, "samples_timed": m, "realizations_timed": 1,
                           "note": "one realization timed, samples/s divided by the 256 realizations",
                           "speedup_of_bf16": (n / (ms / 1e3)) / plain_rate},
        "fp32_per_realization": {"value": fp32_rate, "unit": UNIT, "realizations_timed": 1,
                                 "note": "FP32 path, one realization per pass, divided by 256",
                                 "speedup_of_bf16": (n / (ms / 1e3)) / fp32_rate},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": BF16_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / BF16_TFLOPS, "traffic": None, "peak_source": PEAK_SOURCE,
                     "note": "algorithmic 2*3*pairs*R flops (the hi/lo weight split doubles the issued MMAs); "
                             "dense BF16 burst peak",
                     "binding_unit": "FP32 weight producers (geometry, beam cells, Ludwig-3 rotation per pair)",
                     "tensor_pipe_pct": MR_PROFILE["tensor_pipe_pct"] if n_real == 256 else None,
                     "issue_per_cycle": MR_PROFILE["issue_per_cycle"] if n_real == 256 else None,
                     "l1tex_throughput_pct": MR_PROFILE["l1tex_pct"] if n_real == 256 else None,
                     "unit_pct_note": "recorded ncu figures of this kernel at 256 realizations "
                                      "(profiles/k_mr_multirealization.md), not measured by this run"},
        "gpu_launches": args.steps, "clocks": clk}))


def run_psb(args, dev):
    """A PSB pair (zeta 0 and -90 deg, matched beams) on the default single-detector workload: one
    pisco_convolve_psb pass per step writes both TODs; two pisco_convolve calls are timed beside it."""
    from oracle import beam as ob
    from oracle import convolve as oc
    n = args.samples
    r, sky, grids, (th, ph, ps) = make_workload(dev, n)
    g = torch.as_tensor(grids, device=dev)[None].contiguous()
    zetas = [0.0, -math.pi / 2]
    plan = pisco.Plan(WORKLOAD["nside"], r, sky, [(0.0, 0.0, 1.0)], g, tile_samples=WORKLOAD["tile_samples"])
    pairs = int(plan.disc_count(th, ph).to(torch.int64).sum().item())
    tod2 = torch.empty(2, n, dtype=torch.float32, device=dev)
    tod = torch.empty(n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        ms = _event_time(lambda: plan.convolve_psb(th, ph, ps, zetas, out=tod2), args.steps, args.warmup, stream)
    ms_fwd = _event_time(lambda: plan.convolve(th, ph, ps, out=tod), args.steps, args.warmup, stream)
    plan.sync_status()
    # both rows against the FP64 oracle for a detector at each angle, first 24 samples
    k = 24
    skyn, g64 = sky.cpu().numpy(), np.asarray(grids, np.float64)
    omega = ob.omega_tilde(g64[0], r)
    thn, phn, psn = (a[:k].cpu().numpy() for a in (th, ph, ps))
    err = 0.0
    for row, z in enumerate(zetas):
        ref = oc.tod(WORKLOAD["nside"], r, skyn, g64, (z, 0.0, 1.0), omega, thn, phn, psn)
        err = max(err, float(np.max(np.abs(tod2[row, :k].double().cpu().numpy() - ref)) / np.max(np.abs(ref))))
    achieved = FLOPS_PER_PAIR * pairs / (ms / 1e3) / 1e12
    out = {"metric": "TOD samples/s of a PSB pair (2 TODs per pointing, nside 512, R 10 deg, 501^2 grid)",
           "value": 2 * n / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "PSB pair (zeta 0, -90 deg) on the single-detector workload: " + WORKLOAD["workload"],
                      "samples": n, "pairs_per_step": pairs, "l2": "inputs larger than L2"},
           "two_forward_calls_ms": 2 * ms_fwd, "pass_over_one_forward": ms / ms_fwd,
           "err_vs_oracle_normwise_first_24": err,
           "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                        "note": "forward flops per pair (the pass adds 4 FMAs per pair)"},
           "gpu_launches": args.steps, "clocks": clocks.summary()}
    plan.close()
    print(json.dumps(out))


def run_sec61(args, dev):
    """The paper's Sec. 6.1 simulation: nside-512 sky, circular 1.5 deg Gaussian beam given as HEALPix
    maps at nside 2048 (ideal beamsor), one detector (zeta 0, eps 0, s 1) pointed at every nside-128
    pixel centre at psi = 0, 45, 90 deg (589,824 samples), TOD then binned maps at nside 128.  Wall
    time of the whole chain (beam maps to the GPU and onto the grid, plan, convolution, map-making,
    maps back to the host), best of 2; the maps are checked against the oracle's chain (oracle TOD
    binned by the oracle) on 12 sampled pixels."""
    from oracle import beam as ob
    from oracle import convolve as oc
    from oracle import healpix as ohp
    from oracle import mapmaking as omm
    nside, nside_out, nside_b, r = 512, 128, 2048, math.radians(5.0)
    n_grid = int(round(2 * math.sin(r) / math.radians(0.0286))) + 1  # the nside-2048 pixel size
    sky_h = cached_sky(nside, 1, "cuda").cpu().pin_memory()
    beam_h = beams.gaussian_beam_healpix(nside_b, 1.5, ideal=True, device="cuda").float().cpu().pin_memory()
    th_c, ph_c = sy.healpix_centres(nside_out)
    ang = np.radians([0.0, 45.0, 90.0])
    th, ph, ps = np.repeat(th_c, 3), np.repeat(ph_c, 3), np.tile(ang, len(th_c))
    h = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (th, ph, ps)]
    det = (0.0, 0.0, 1.0)
    best, maps_h = None, None
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sky = sky_h.to(dev, non_blocking=True)
        g = pisco.pisco_beam_grids_from_healpix(beam_h.to(dev, non_blocking=True), nside_b, r, n_grid)[None]
        plan = pisco.Plan(nside, r, sky, [det], g)
        d = [a.to(dev, non_blocking=True) for a in h]
        tod = plan.convolve(*d)
        maps, hits = pisco.binned_map(nside_out, *d, det, tod)
        maps_h = maps.cpu()
        wall = time.perf_counter() - t0
        plan.close()
        best = wall if best is None else min(best, wall)
    # the oracle's chain on sampled pixels (its grids from the same HEALPix maps)
    grids = ob.grid_from_healpix(beam_h[[0, 4]].double().numpy(), nside_b, r, n_grid)
    g6 = np.zeros((6, n_grid, n_grid))
    g6[0], g6[4] = grids
    omega = ob.omega_tilde(g6[0], r)
    skyn = sky_h.double().numpy()
    sample = np.random.default_rng(61).integers(0, ohp.npix(nside_out), 12)
    tt, pp = ohp.pix2ang(nside_out, sample)
    T, P, A = np.repeat(tt, 3), np.repeat(pp, 3), np.tile(ang, len(sample))
    d_ref = oc.tod(nside, r, skyn, g6, det, omega, T, P, A)
    ref, _ = omm.binned_map(nside_out, T, P, A, det, d_ref)
    got = maps_h.numpy()[:, sample]
    err = float(np.max(np.abs(got - ref[:, sample])) / np.max(np.abs(ref[:, sample])))
    out = {"metric": "Sec. 6.1 chain wall time: HEALPix beam + TOD + binned maps (589,824 samples)",
           "value": 1e3 * best, "unit": "ms", "higher_is_better": False, "n_gpus": 1, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "nside-512 sky, 1.5 deg Gaussian beam as HEALPix maps at nside 2048, R 5 deg, "
                                  "every nside-128 pixel centre at psi 0/45/90 deg, binned maps at nside 128",
                      "grid_n": n_grid, "samples": len(th)},
           "samples_per_s": len(th) / best, "hits_min": int(hits.min().item()),
           "maps_vs_oracle_chain_max_rel_12_pixels": err, "vs_baseline": None}
    print(json.dumps(out))


def run_grad(args, dev):
    """The differentiation configuration: nside-512 FP32 sky, one detector with the parametric beam
    (FWHM 1.5 deg, ellipticity 0.05, cross-polar leakage 0.005) on a 201^2 grid of radius 5 deg, 1e7
    samples of the azimuth scan.  One step = beam grids from the parameters, TOD (pisco_convolve
    through PiscoConvolve), chi^2 against the TOD of perturbed parameters (1.52, 0.06, 0.004), and
    its backward pass: the sky adjoint (TOD -> I, Q, U maps) and the beam-grid adjoint in one
    traversal, the Omega~ term and the chain to d chi^2 / d(FWHM, e, l).  The gradient is checked on a 48-sample slice against
    central differences (h = 1e-4) of the FP64 oracle."""
    from oracle import beam as ob
    from oracle import convolve as oc
    from paper_1908_05662_gb300 import autograd as pag
    import torch.distributed as tdist
    distributed = tdist.is_available() and tdist.is_initialized()
    world = tdist.get_world_size() if distributed else 1
    rank = tdist.get_rank() if distributed else 0
    nside, r, n_grid = 512, math.radians(5.0), 201
    n = args.samples  # per rank: weak scaling, rank k takes samples k n .. (k + 1) n - 1 of the scan
    sky = cached_sky(nside, 1, dev)
    th, ph, ps = (a.contiguous() for a in sy.ces_scan(n, device=dev, start=rank * n))
    det = (0.0, 0.0, 1.0)
    p0, pt = (1.5, 0.05, 0.005), (1.52, 0.06, 0.004)

    def tod_of(p, sky_t, theta, phi, psi):
        g = beams.gaussian_beam_grids(n_grid, r, p[0], p[1], p[2], device=dev)
        return pag.convolve(sky_t, g, theta, phi, psi, nside, r, det)

    with torch.no_grad():
        target = tod_of(torch.tensor(pt, dtype=torch.float64, device=dev), sky, th, ph, ps).double()

    def step():
        params = torch.tensor(p0, dtype=torch.float64, device=dev, requires_grad=True)
        sky_t = sky.clone().requires_grad_(True)
        loss = ((tod_of(params, sky_t, th, ph, ps).double() - target) ** 2).sum()
        loss.backward()
        if world > 1:
            # the transposes are sums over all samples: one all-reduce of each gradient
            tdist.all_reduce(sky_t.grad)
            tdist.all_reduce(params.grad)
        return params.grad, sky_t.grad

    stream = torch.cuda.current_stream()
    if world > 1:
        tdist.barrier()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        ms = _event_time(step, args.steps, args.warmup, stream)
    ms = max_over_ranks(ms, dev)
    # the collective alone: the sky-map gradient (3 x Npix FP32) and the beam-grid gradient
    grad_maps = torch.zeros(3, 12 * nside * nside, device=dev)
    grad_grid = torch.zeros(6, n_grid, n_grid, device=dev)
    allreduce_ms = 0.0
    if world > 1:
        allreduce_ms = max_over_ranks(_event_time(lambda: (tdist.all_reduce(grad_maps), tdist.all_reduce(grad_grid)),
                                                  args.steps, 1, stream), dev)
        if rank != 0:
            return
    # the passes one by one on the same inputs
    g = beams.gaussian_beam_grids(n_grid, r, *p0, device=dev).float()[None].contiguous()
    y = torch.randn(n, device=dev)
    with pisco.Plan(nside, r, sky, [det], g) as plan:
        tod = plan.convolve(th, ph, ps)
        parts = {"forward_ms": _event_time(lambda: plan.convolve(th, ph, ps, out=tod), 2, 1, stream),
                 "sky_adjoint_ms": _event_time(lambda: plan.adjoint(th, ph, ps, y), 2, 1, stream),
                 "beam_grid_adjoint_ms": _event_time(lambda: plan.beam_grid_adjoint(th, ph, ps, y), 2, 1, stream),
                 "sky_and_beam_adjoint_ms": _event_time(lambda: plan.adjoint_sky_beam(th, ph, ps, y), 2, 1, stream)}
        pairs = int(plan.disc_count(th, ph).to(torch.int64).sum().item())
        plan.sync_status()
    m = min(n, 100_000)
    y64 = y[:m].double()
    with pisco.Plan(nside, r, sky, [det], g, precision=pisco.PISCO_FP64_PLAIN) as plain:
        t, p_, q = th[:m], ph[:m], ps[:m]
        plain_ms = {"forward_ms": _event_time(lambda: plain.convolve(t, p_, q), 2, 1, stream),
                    "sky_adjoint_ms": _event_time(lambda: plain.adjoint(t, p_, q, y64), 2, 1, stream),
                    "beam_grid_adjoint_ms": _event_time(lambda: plain.beam_grid_adjoint(t, p_, q, y64), 2, 1,
                                                        stream)}
        plain.sync_status()
    plain_step_per_sample = sum(plain_ms.values()) / m
    fp32_step_per_sample = (parts["forward_ms"] + parts["sky_and_beam_adjoint_ms"]) / n
    # gradient check on a slice against the FP64 oracle
    # (the slice's target is the oracle's TOD of the perturbed parameters, on both sides)
    k = 48
    sl = slice(0, k)
    skyn = sky.cpu().numpy()
    thn, phn, psn = (a[sl].cpu().numpy() for a in (th, ph, ps))

    def oracle_tod(p):
        gr = beams.gaussian_beam_grids(n_grid, r, p[0], p[1], p[2]).numpy()
        return oc.tod(nside, r, skyn, gr, det, ob.omega_tilde(gr[0], r), thn, phn, psn)

    tgtn = oracle_tod(pt)
    params = torch.tensor(p0, dtype=torch.float64, device=dev, requires_grad=True)
    loss = ((tod_of(params, sky, th[sl], ph[sl], ps[sl]).double() - torch.as_tensor(tgtn, device=dev)) ** 2).sum()
    loss.backward()
    grad = params.grad.cpu().numpy()

    def chi2(p):
        return float(np.sum((oracle_tod(p) - tgtn) ** 2))

    h = 1e-4
    fd = []
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd.append((chi2(np.array(p0) + e) - chi2(np.array(p0) - e)) / (2 * h))
    rel = [abs(grad[i] - fd[i]) / abs(fd[i]) for i in range(3)]
    bg = parts["sky_and_beam_adjoint_ms"]
    out = {"metric": "gradient steps/s (TOD, chi^2, backward to sky maps and beam parameters; 1e7 samples per GPU)",
           "value": 1e3 / ms, "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "samples_per_s": world * n / (ms / 1e3), "higher_is_better": True, "scaling": "weak",
           "allreduce": {"ms": allreduce_ms, "share_of_step": allreduce_ms / ms,
                         "bytes": 4 * (3 * 12 * nside * nside + 6 * n_grid * n_grid),
                         "note": "one all-reduce of the sky-map gradient and one of the beam-grid gradient "
                                 "(NCCL; zero on one GPU)"},
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "differentiation: nside 512, parametric beam (FWHM 1.5 deg, e 0.05, l 0.005), "
                                  "R 5 deg, 201^2 grid, 1e7 scan samples", "samples": n, "pairs_per_pass": pairs},
           "passes": parts,
           "plain_fp64_gpu": {"passes_ms": plain_ms, "samples_timed": m,
                              "samples_per_s": 1e3 / plain_step_per_sample,
                              "speedup_of_fp32_passes": plain_step_per_sample / fp32_step_per_sample,
                              "note": "forward + sky adjoint + beam-grid adjoint per sample, against the FP32 "
                                      "forward + fused sky-and-beam adjoint"},
           "grad_vs_oracle_fd_rel": rel, "grad": list(map(float, grad)), "fd": fd,
           "roofline": {"bound": "alu", "kernel": "pisco::k_fast<16, sky and beam-grid transposes>",
                        "achieved": FLOPS_PER_PAIR * pairs / (bg / 1e3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": FLOPS_PER_PAIR * pairs / (bg / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                        "traffic": None, "note": "forward flops per pair as the work unit of the transpose"},
           "gpu_launches": 9 * args.steps, "clocks": clocks.summary()}
    print(json.dumps(out))


def run_table1(args, dev):
    """The paper's Table 1 setup (Sec. 5.3.1): 2 detectors (zeta 0 and -90 deg) x 3 position angles
    (0, 45, 90 deg) x every nside-128 pixel centre = 1,179,648 samples, Gaussian FWHM 1.5 deg,
    rho_max 5-30 deg; wall time includes building the beam grid and plan, the host<->GPU copies and
    the convolution, as in the paper.  Beam grid spacing 0.1145 deg (the pixel size of the paper's
    nside-512 beam)."""
    nside = 128
    th_c, ph_c = sy.healpix_centres(nside)
    angles = np.radians([0.0, 45.0, 90.0])
    th = np.repeat(th_c, 3)
    ph = np.repeat(ph_c, 3)
    ps = np.tile(angles, len(th_c))
    h = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (th, ph, ps)]
    sky_h = cached_sky(nside, 1, "cuda").cpu().pin_memory()
    beam_hpx = beams.gaussian_beam_healpix(512, 1.5, ideal=True, device="cuda").float().cpu().pin_memory()
    paper = {5.0: 1471.41, 7.5: 3135.19, 10.0: 5560.25, 15.0: 12719.56, 20.0: 23190.68, 25.0: 39447.70,
             30.0: 53800.74}
    rows = []
    for rho, paper_ms in paper.items():
        r = math.radians(rho)
        n_grid = int(round(2 * math.sin(r) / math.radians(0.1145))) + 1
        best = None
        for rep in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            grids_h = torch.from_numpy(np.stack([sy.gaussian_beam_maps(n_grid, r, 1.5, ideal=True)] * 2))
            sky = sky_h.to(dev, non_blocking=True)
            g = grids_h.to(dev)
            plan = pisco.Plan(nside, r, sky, [(0.0, 0.0, 1.0), (-math.pi / 2, 0.0, 1.0)], g)
            outs = [torch.empty(len(th), dtype=torch.float32).pin_memory() for _ in range(2)]
            for d in range(2):
                plan.convolve_host(*h, det=d, out=outs[d])
            wall = time.perf_counter() - t0
            plan.close()
            best = wall if best is None else min(best, wall)
        # the paper's own flow: the beam as HEALPix maps at nside 512, the interpolation grid
        # assembled on the GPU (pisco_beam_grids_from_healpix), both TODs from one
        # shared-geometry pass (pisco_convolve_psb); copies included
        best_psb = None
        for rep in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sky = sky_h.to(dev, non_blocking=True)
            g = pisco.pisco_beam_grids_from_healpix(beam_hpx.to(dev, non_blocking=True), 512, r, n_grid)[None]
            plan = pisco.Plan(nside, r, sky, [(0.0, 0.0, 1.0)], g)
            d = [a.to(dev, non_blocking=True) for a in h]
            out = torch.empty(2, len(th), dtype=torch.float32).pin_memory()
            out.copy_(plan.convolve_psb(*d, [0.0, -math.pi / 2]), non_blocking=True)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            plan.close()
            best_psb = wall if best_psb is None else min(best_psb, wall)
        rows.append({"rho_max_deg": rho, "grid_n": n_grid, "wall_ms": 1e3 * best, "paper_ms_gtx1080": paper_ms,
                     "samples_per_s": 2 * len(th) / best, "speedup_vs_paper": paper_ms / (1e3 * best),
                     "wall_ms_healpix_beam_psb_pass": 1e3 * best_psb,
                     "speedup_psb_vs_paper": paper_ms / (1e3 * best_psb)})
    print(json.dumps({"metric": "Table 1 replica: wall time of a whole-sky PSB convolution", "unit": "ms",
                      "higher_is_better": False, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "2 detectors x 3 angles x nside-128 pixel centres = 1,179,648 "
                                             "samples, FWHM 1.5 deg, rho_max 5-30 deg, copies included"},
                      "rows": rows}))


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if args.workload != "single":
        torch.cuda.set_device(local)
        {"c1": run_c1, "focalplane": run_focalplane, "multireal": run_multireal, "table1": run_table1, "psb": run_psb,
         "sec61": run_sec61, "grad": run_grad}[args.workload](
            args, torch.device("cuda", local))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_total = args.samples * world  # weak scaling: every rank convolves its own full scan
    a, b = shard(n_total, rank, world)
    n = b - a
    r, sky, grids, (th, ph, ps) = make_workload(dev, n)
    det = (0.0, 0.0, 1.0)
    g = torch.as_tensor(grids, device=dev)[None].contiguous()
    plan = pisco.Plan(WORKLOAD["nside"], r, sky, [det], g, precision=pisco.PISCO_FP32,
                      tile_samples=WORKLOAD["tile_samples"], pixels_per_thread=WORKLOAD["pixels_per_thread"])
    tod = torch.empty(n, dtype=torch.float32, device=dev)

    # tile shape from the library's autotuner, timed on the first 2e5 samples of the scan (untimed)
    m = min(n, 200_000)
    tuned = plan.autotune(th[:m], ph[:m], ps[:m], reps=2)

    # exact number of in-disc pairs (untimed): the kernel's own disc counts
    counts = plan.disc_count(th, ph)
    pairs = int(counts.to(torch.int64).sum().item())

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.convolve(th, ph, ps, out=tod)
    torch.cuda.synchronize()
    plan.sync_status()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            starts[k].record(stream)
            plan.convolve(th, ph, ps, out=tod)
            ends[k].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    plan.sync_status()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = statistics.mean(step_ms)
    total_ms = max_over_ranks(sum(step_ms), dev)
    value = n_total * args.steps / (total_ms / 1e3)

    # end to end through the host-buffer entry point (pinned host memory, copies timed)
    h = [x.cpu().pin_memory() for x in (th, ph, ps)]
    h_tod = torch.empty(n, dtype=torch.float32).pin_memory()
    plan.convolve_host(*h, out=h_tod)
    e2e_steps = max(args.steps, 3)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.convolve_host(*h, out=h_tod)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_value = n * world / e2e_s

    # the same scan with packed 32-byte beam cells (FP32 values, int16 slopes), same tile shape
    packed = pisco.Plan(WORKLOAD["nside"], r, sky, [det], g, precision=pisco.PISCO_FP32,
                        beam_fetch=pisco.PISCO_FETCH_PACKED, tile_samples=tuned[0], pixels_per_thread=tuned[1])
    tod_p = torch.empty(n, dtype=torch.float32, device=dev)
    ms_packed = _event_time(lambda: packed.convolve(th, ph, ps, out=tod_p), args.steps, args.warmup, stream)
    packed.sync_status()
    packed.close()
    packed_vs_cells = (tod_p.double() - tod.double()).abs().max().item() / tod.double().abs().max().item()

    # plain FP64 GPU path on a contiguous slice of the same scan
    n_plain = min(n, 100_000)
    plain = pisco.Plan(WORKLOAD["nside"], r, sky, [det], g, precision=pisco.PISCO_FP64_PLAIN)
    tod64 = torch.empty(n_plain, dtype=torch.float64, device=dev)
    plain.convolve(th[:n_plain], ph[:n_plain], ps[:n_plain], out=tod64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plain.convolve(th[:n_plain], ph[:n_plain], ps[:n_plain], out=tod64)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_rate = n_plain / (e0.elapsed_time(e1) / 1e3)
    fp32_vs_64 = (tod[:n_plain].double() - tod64).abs().max().item() / tod64.abs().max().item()
    plain.close()

    out = None
    if rank == 0:
        achieved_tflops = FLOPS_PER_PAIR * pairs / (ms / 1e3) / 1e12
        recorded = FORWARD_PROFILE.get((n, tuned[0], tuned[1]), {})
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD["workload"], "nside": WORKLOAD["nside"],
                       "radius_deg": WORKLOAD["radius_deg"], "grid_n": WORKLOAD["grid_n"],
                       "samples_per_rank": n, "tile_samples": tuned[0], "pixels_per_thread": tuned[1],
                       "tile_shape": "autotuned (pisco_plan_autotune on the first 2e5 samples)",
                       "pairs_per_step": pairs * world, "mean_disc_pixels": pairs / n,
                       "l2": "inputs larger than L2 (pointing 24 B/sample = 240 MB)"},
            "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved_tflops / FP32_PEAK_TFLOPS,
                         "traffic": recorded.get("traffic"),
                         "traffic_note": "recorded ncu capture of DRAM bytes read + written per forward launch "
                                         "of this shape (null for another shape); not measured by this run",
                         "binding_unit": "L1/TEX (scattered 32-byte sectors of beam cells, all L2 hits)",
                         "l1tex_throughput_pct": recorded.get("l1tex_pct"),
                         "lts_throughput_pct": recorded.get("lts_pct"),
                         "unit_pct_note": "recorded ncu percentages of peak for this kernel shape "
                                          "(profiles/k_fast_forward_single_detector.md)",
                         "kernel": f"pisco::k_fast<{tuned[0]}, {tuned[1]}, cells, forward>",
                         "peak_note": "FP32 from unit counts: 152 SM x 128 lanes x 2 x 2070 MHz",
                         "hbm_frac": (28 * n / (ms / 1e3)) / (HBM_GBS * 1e9), "hbm_peak_source": PEAK_SOURCE},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 24 * n, "d2h_bytes_per_step": 4 * n,
                    "steps": e2e_steps},
            "plain_fp64_gpu": {"value": plain_rate * world, "unit": UNIT, "samples_timed": n_plain,
                               "speedup_of_fp32": value / (plain_rate * world),
                               "fp32_vs_fp64_normwise": fp32_vs_64},
            "gpu_launches": args.steps,
            "clocks": clocks.summary(),
            "packed_cells": {"value": n_total / (ms_packed / 1e3), "unit": UNIT, "ms_per_step": ms_packed,
                             "vs_cells_tod_normwise": packed_vs_cells,
                             "note": "PISCO_FETCH_PACKED: 32-byte cells, FP32 values and int16 slopes"},
            "wall_s_timed": t_wall,
        }
        if not args.no_cpu:
            thn, phn, psn = th.cpu().numpy(), ph.cpu().numpy(), ps.cpu().numpy()
            rate, idx, ref, cores = cpu_oracle_rate(sky, grids, r, det, thn, phn, psn, n)
            sel = torch.as_tensor(idx, device=tod.device)
            err = np.max(np.abs(tod[sel].double().cpu().numpy() - ref)) / np.max(np.abs(ref))
            out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": f"{len(idx)} samples: {cores} single-threaded worker processes, "
                                             "each ~15 s on consecutive samples from its own offset"}
            out["err_vs_oracle_normwise"] = err
            out["packed_cells"]["err_vs_oracle_normwise"] = (
                np.max(np.abs(tod_p[sel].double().cpu().numpy() - ref)) / np.max(np.abs(ref)))
        print(json.dumps(out))
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
