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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pisco", choices=["pisco", "reference"])
    ap.add_argument("--samples", type=int, default=WORKLOAD["n_samples"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline leg")
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
    torch.save(sky, path + ".tmp")
    os.replace(path + ".tmp", path)
    return sky


def make_workload(device, n):
    r = math.radians(WORKLOAD["radius_deg"])
    sky = cached_sky(WORKLOAD["nside"], 1, device)
    grids = sy.gaussian_beam_maps(WORKLOAD["grid_n"], r, 1.5, ellipticity=0.0, xpol=0.005,
                                  sidelobe=(0.01, 7.0, 0.5))
    theta, phi, psi = sy.ces_scan(n, device=device)
    return r, sky, grids, (theta.contiguous(), phi.contiguous(), psi.contiguous())


def cpu_oracle_rate(sky, grids, radius, det, theta, phi, psi, n_samples, budget_s=15.0):
    """The FP64 oracle on consecutive samples until ~budget_s of CPU time; returns (rate, n, outputs)."""
    from oracle import beam as ob
    from oracle import convolve as oc
    g64 = np.asarray(grids, np.float64)
    omega = ob.omega_tilde(g64[0], radius)
    skyn = sky if isinstance(sky, np.ndarray) else sky.cpu().numpy()
    outs = []
    t0 = time.perf_counter()
    k = 0
    while k < n_samples and time.perf_counter() - t0 < budget_s:
        outs.append(oc.tod(WORKLOAD["nside"], radius, skyn, g64, det, omega, theta[k:k + 1], phi[k:k + 1],
                           psi[k:k + 1])[0])
        k += 1
    dt = time.perf_counter() - t0
    return k / dt, k, np.array(outs)


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
    per_step = 4
    times = []
    for step in range(args.warmup + args.steps):
        a = (step * per_step) % (n - per_step)
        t0 = time.perf_counter()
        from oracle import beam as ob
        from oracle import convolve as oc
        omega = ob.omega_tilde(np.asarray(grids[0], np.float64), r)
        oc.tod(WORKLOAD["nside"], r, sky.numpy(), grids.astype(np.float64), det, omega,
               thn[a:a + per_step], phn[a:a + per_step], psn[a:a + per_step])
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = per_step / (ms / 1e3)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["workload"], "oracle_sample": f"{per_step} consecutive scan samples per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} consecutive samples of the scan per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
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
    e2e_steps = 2
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.convolve_host(*h, out=h_tod)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_value = n * world / e2e_s

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
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD["workload"], "nside": WORKLOAD["nside"],
                       "radius_deg": WORKLOAD["radius_deg"], "grid_n": WORKLOAD["grid_n"],
                       "samples_per_rank": n, "tile_samples": WORKLOAD["tile_samples"],
                       "pairs_per_step": pairs * world, "mean_disc_pixels": pairs / n,
                       "l2": "inputs larger than L2 (pointing 24 B/sample = 240 MB)"},
            "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved_tflops / FP32_PEAK_TFLOPS, "traffic": None,
                         "kernel": "pisco::k_fast<16, forward>",
                         "peak_note": "FP32 from unit counts: 152 SM x 128 lanes x 2 x 2070 MHz",
                         "hbm_frac_of_measured": (28 * n / (ms / 1e3)) / 6758.2e9},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 24 * n, "d2h_bytes_per_step": 4 * n},
            "plain_fp64_gpu": {"value": plain_rate * world, "unit": UNIT, "samples_timed": n_plain,
                               "speedup_of_fp32": value / (plain_rate * world),
                               "fp32_vs_fp64_normwise": fp32_vs_64},
            "gpu_launches": args.steps,
            "clocks": clocks.summary(),
            "wall_s_timed": t_wall,
        }
        if not args.no_cpu:
            thn, phn, psn = th.cpu().numpy(), ph.cpu().numpy(), ps.cpu().numpy()
            rate, k, ref = cpu_oracle_rate(sky, grids, r, det, thn, phn, psn, n)
            err = np.max(np.abs(tod[:k].double().cpu().numpy() - ref)) / np.max(np.abs(ref))
            out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": f"first {k} consecutive samples of the scan (~15 s of CPU)"}
            out["err_vs_oracle_normwise"] = err
        print(json.dumps(out))
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
