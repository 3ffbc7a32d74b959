#!/usr/bin/env python3
"""Throughput benchmark of the fused iPiano step (Mpixel * accepted iterations / s).

Workload (paper-like sizes, plain FP32 solver): a batch of synthetic
textured images, 24 of 512x512 and 24 of 256x256, gamma speckle with
L cycling over {1, 4, 8}, the seeded 48 x 7 x 7 zero-mean unit-norm filter
bank with theta_i = 0.1, lambda = 5, beta = 0.8, L0 = 1, eta = 2, and 300
iPiano iterations with Lipschitz backtracking per image.  One step = restart
every image from its observation f (grad F(u^0), F, G on the device) and run
the 300 iterations of the whole batch through the C ABI (fe_reset + fe_step).

value  : sum of pixels x accepted iterations / device time of the K steps
         (CUDA events on the solver's stream), inputs resident in HBM.
e2e    : same metric through the C ABI with HOST (pinned) buffers: every
         step copies f in, solves, copies u out.
roofline: the fused trial kernel is bound by FP32 FMA issue: peak =
         152 SMs x 128 lanes x 2 flop x SM clock; algorithmic work is
         2 x 48 x 49 MACs = 9408 flop per pixel per trial.

``--impl reference`` times the FP64 CPU oracle (the only reference that
exists: the paper ships no code) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOP_PER_PIXEL_TRIAL = 2 * 48 * 49 * 2  # forward + adjoint bank, 2 flop per MAC
SMS, FP32_LANES = 152, 128
METRIC = "Mpixel*iter/s of fused iPiano step"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--n512", type=int, default=24)
    ap.add_argument("--n256", type=int, default=24)
    ap.add_argument("--prec", default="fp32")
    ap.add_argument("--loop-mode", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def workload(n512, n256):
    from paper_1404_5344_gb300 import synth
    shapes, Ls, fs = [], [], []
    looks = (1.0, 4.0, 8.0)
    j = 0
    for (n, s) in ((n512, 512), (n256, 256)):
        for i in range(n):
            u = synth.textured_image(s, s, seed=1000 + j)
            L = looks[j % 3]
            fs.append(synth.speckle(u, L=L, seed=5000 + j))
            shapes.append((s, s))
            Ls.append(L)
            j += 1
    k, th = synth.filter_bank(48, 7, seed=0, theta=0.1)
    return fs, k, th, shapes, Ls


SOLVER_KW = dict(lam=5.0, beta=0.8, L0=1.0, eta=2.0, c2=1e-6, max_backtrack=30)


def measured_bf16_sustained():
    """Dense BF16 tensor peak measured on this machine (seconds-long loop), else
    the profiling recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops_sustained"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 1700.0, "of fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index: int, path: str):
        self.path, self.proc = path, None
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for ln in open(self.path):
            p = [x.strip() for x in ln.split(",")]
            if len(p) >= 9:
                try:
                    rows.append((float(p[1]), float(p[2]), float(p[3]), p[5:9]))
                except ValueError:
                    pass
        if not rows:
            return None
        load = [r for r in rows if r[2] > 200.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(load)}


def cpu_baseline(fs, k, th, iters_total, seconds):
    """The FP64 oracle, as it stands, on a bounded sample: one 256x256 image
    of the workload, as many iterations as fit in about `seconds`."""
    import oracle as orc
    orc.build()
    f = next(x for x in fs if x.shape == (256, 256)) if any(x.shape == (256, 256) for x in fs) else fs[0]
    prm = dict(lam=SOLVER_KW["lam"], beta=SOLVER_KW["beta"], L0=SOLVER_KW["L0"], eta=SOLVER_KW["eta"],
               c2=SOLVER_KW["c2"], max_backtrack=SOLVER_KW["max_backtrack"])
    t0 = time.perf_counter()
    orc.ipiano(f, k, th, orc.params(max_iter=2, **prm))
    per_it = (time.perf_counter() - t0) / 2.0
    n = int(max(2, min(iters_total, seconds / max(per_it, 1e-6))))
    t0 = time.perf_counter()
    out = orc.ipiano(f, k, th, orc.params(max_iter=n, **prm))
    dt = time.perf_counter() - t0
    npx = f.size
    return {"value": round(npx * out["n"] / dt / 1e6, 4), "unit": "Mpixel*iter/s",
            "cores": orc.num_threads(), "kind": "oracle",
            "sample": "FP64 oracle, one %dx%d image of the workload, %d iPiano iterations "
                      "(%.1f s)" % (f.shape[0], f.shape[1], out["n"], dt)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    fs, k, th, shapes, Ls = workload(min(args.n512, 1), min(args.n256, 1))
    import oracle as orc
    orc.build()
    f = fs[-1]
    prm = orc.params(max_iter=4, lam=SOLVER_KW["lam"], beta=SOLVER_KW["beta"], L0=SOLVER_KW["L0"],
                     eta=SOLVER_KW["eta"], c2=SOLVER_KW["c2"], max_backtrack=SOLVER_KW["max_backtrack"])
    for _ in range(args.warmup):
        orc.ipiano(f, k, th, prm)
    times, its = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = orc.ipiano(f, k, th, prm)
        times.append(time.perf_counter() - t0)
        its += out["n"]
    T = sum(times)
    value = f.size * its / T / 1e6
    line = {"metric": METRIC, "value": round(value, 4), "unit": "Mpixel*iter/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * T / args.steps, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "FP64 CPU oracle on one 256x256 textured image of the batch, 4 iPiano "
                                   "iterations per step (bounded sample of the 24x512^2 + 24x256^2, "
                                   "300-iteration workload)", "iters_per_step": 4},
            "cpu_baseline": {"value": round(value, 4), "unit": "Mpixel*iter/s", "cores": orc.num_threads(),
                             "kind": "oracle", "sample": "one 256x256 image, 4 iterations per step"},
            "e2e": {"value": round(value, 4), "unit": "Mpixel*iter/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1404_5344_gb300 import build
    build.build()
    from paper_1404_5344_gb300 import fe

    fs, k, th, shapes, Ls = workload(args.n512, args.n256)
    npix = sum(h * w for h, w in shapes)
    stream = torch.cuda.Stream()
    f_dev = [torch.from_numpy(f).cuda() for f in fs]
    torch.cuda.synchronize()
    solver = fe.Solver(f_dev, k, th, prec=args.prec, stream=stream, loop_mode=args.loop_mode, **SOLVER_KW)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one_step():
        solver.reset(f_dev)
        ev_l0 = torch.cuda.Event(enable_timing=True)
        ev_l0.record(stream)
        st = solver.step(args.iters, sync=False)
        return st, ev_l0

    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(local, os.path.join(ROOT, "gpurun_out", "clocks_rank%d.csv" % rank)) \
        if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else ClockSampler(local, "/tmp/fe_clocks.csv")
    total_ms, loop_ms = 0.0, 0.0
    lc0 = solver.launch_count()
    pix_iters_done, trials, pix_trials = 0, 0, 0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, el = one_step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        loop_ms += el.elapsed_time(e1)
        # fe_reset restarts the counters: n = accepted iterations of this step
        infos = [solver.info(i) for i in range(len(fs))]
        pix_iters_done += sum(x["n"] * h * w for x, (h, w) in zip(infos, shapes))
        trials += sum(x["trials"] for x in infos)
        pix_trials += sum(x["trials"] * h * w for x, (h, w) in zip(infos, shapes))
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = solver.launch_count() - lc0
    statuses = sorted({x["status"] for x in infos})

    # max over ranks
    t_tensor = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t_tensor, op=dist.ReduceOp.MAX)
    T_ms = float(t_tensor.item())
    value = pix_iters_done * world / (T_ms / 1e3) / 1e6

    # Trial-kernel rate: algorithmic work of every image-trial that ran
    # (9408 flop per pixel, accepted and rejected trials alike) over the
    # device time of the iteration loop (trial launches + one loop-begin
    # kernel per step; the per-step restart is outside this window).  A
    # launch late in a step covers only the images still iterating, so work
    # is counted per image-trial, not per launch.
    trial_launches = max(1, launches - args.steps * (len(fs) + 2))
    per_launch_ms = loop_ms / trial_launches
    achieved_tflops = FLOP_PER_PIXEL_TRIAL * pix_trials / (loop_ms / 1e3) / 1e12
    sm_mhz_max = (clk or {}).get("sm_max_mhz") or 2070.0
    if args.prec == "fp32":
        bound, kernel = "alu", "fp32_tile_kernel<MODE_TRIAL>"
        peak_tflops = SMS * FP32_LANES * 2 * sm_mhz_max * 1e6 / 1e12
        basis = "FP32 FMA: 152 SMs x 128 lanes x 2 flop x %.0f MHz (max SM clock)" % sm_mhz_max
    else:
        # the trial kernel runs inside a seconds-long loop: sustained dense
        # BF16 peak (measured); TF32 at the nominal TF32/BF16 ratio 1.1/2.25
        bf16_sust, src = measured_bf16_sustained()
        ratio = 1.0 if args.prec == "bf16" else 1.1 / 2.25
        bound, kernel = "tensor", "tc_tile_kernel<MODE_TRIAL, %s>" % args.prec.upper()
        peak_tflops = bf16_sust * ratio
        basis = "dense %s tensor peak = %.1f TFLOP/s sustained BF16 (%s) x %.3f" % (
            args.prec.upper(), bf16_sust, src, ratio)

    # e2e through the C ABI with host buffers
    f_host = [torch.from_numpy(f).pin_memory() for f in fs]
    u_host = [torch.empty(f.shape, dtype=torch.float32).pin_memory() for f in fs]
    e2e_solver = fe.Solver([x.numpy() for x in f_host], k, th, prec=args.prec, stream=stream,
                           loop_mode=args.loop_mode, **SOLVER_KW)
    torch.cuda.synchronize()
    e2e_ms = 0.0
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        stream.synchronize()
        t0 = time.perf_counter()
        e2e_solver.reset([x.numpy() for x in f_host])
        e2e_solver.step(args.iters, sync=False)
        for i in range(len(fs)):
            e2e_solver.get_u(i, out=u_host[i].numpy())
        stream.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_value = npix * args.iters / (e2e_ms / e2e_steps / 1e3) / 1e6 * world
    e2e_solver.close()

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": "Mpixel*iter/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(T_ms / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "bf16": "bf16", "tf32": "tf32"}[args.prec], "data": "synthetic",
                "config": {"workload": "%dx512^2 + %dx256^2 textured images, L in {1,4,8} gamma speckle, "
                                       "48x7x7 seeded bank, lambda=5, %d iPiano iterations with "
                                       "Lipschitz backtracking, %s filter bank" % (
                                           args.n512, args.n256, args.iters, args.prec.upper()),
                           "images": len(fs), "pixels": npix, "iters": args.iters, "precision": args.prec,
                           "loop": "cuda-graph while node" if args.loop_mode == 1 else "host chunks",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": "256 MiB buffer written between timed steps; state 6 planes x "
                                 "%.0f MB" % (npix * 4 / 1e6)},
                "e2e": {"value": round(e2e_value, 2), "unit": "Mpixel*iter/s",
                        "h2d_bytes_per_step": int(npix * 4), "d2h_bytes_per_step": int(npix * 4)},
                "gpu_launches": int(launches), "trial_kernel_launches": int(trial_launches),
                "trials": int(trials), "statuses": statuses,
                "roofline": {"bound": bound, "achieved": round(achieved_tflops, 3),
                             "peak": round(peak_tflops, 3), "unit": "TFLOP/s",
                             "frac": round(achieved_tflops / peak_tflops, 4), "traffic": None,
                             "kernel": kernel, "peak_basis": basis,
                             "work": "9408 flop (2 x 48 x 49 MAC) per pixel per trial, every image-trial",
                             "per_launch_ms": round(per_launch_ms, 4)},
                "clocks": clk}
        if clk and clk.get("sm_mhz") and args.prec == "fp32":
            line["roofline"]["frac_at_observed_clock"] = round(
                achieved_tflops / (SMS * FP32_LANES * 2 * clk["sm_mhz"] * 1e6 / 1e12), 4)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(fs, k, th, args.iters, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
