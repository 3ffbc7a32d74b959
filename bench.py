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
roofline: the fused trial kernel is bound by FP32 FMA issue: peak = the
         FP32 FMA rate measured by the library's own microbenchmark
         (fe_peak), beside the rate derived from the device's SM count x 128
         lanes x 2 flop x SM clock; algorithmic work is 2 x 48 x 49 MACs =
         9408 flop per pixel per trial.  The tensor-core forms take the
         measured dense BF16 peak (TF32: x 1.1 / 2.25), beside this library's
         own tcgen05 stream rate.
peaks  : measured rates of FP32 FMA (scalar and packed), FP64 FMA, the
         special-function unit (rcp, lg2) and the tensor cores (BF16, TF32).
forms  : the TF32 and BF16 forms and the combined model on the same
         workload, and the batching form's time to tolerance (64 uneven
         images, FP32 and BF16, against 64 sequential FP32 solves).

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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOP_PER_PIXEL_TRIAL = 2 * 48 * 49 * 2  # forward + adjoint bank, 2 flop per MAC
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one trial
# launch with every image active, per pixel, from one ncu capture of the
# current kernels on 24 x 512^2 (profiles/*_trial_24x512.md); None where no
# capture of the current kernel exists
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per pixel-trial
# of the persistent trial kernel: one ncu capture of one persistent launch
# (one step: 300 iterations of 24 x 512^2 + 24 x 256^2), divided by the
# step's pixel-trials (profiles/persistent_trial_kernels_24x512.md)
TRAFFIC_PER_PIXEL_TRIAL = {("fp32", "variant"): 5.741133e+10 / 2431909888,
                           ("bf16", "variant"): 6.098123e+10 / 2450784256,
                           ("bf16r", "variant"): 6.099123e+10 / 2450325504,
                           ("tf32", "variant"): 5.992256e+10 / 2428305408,
                           ("fp32", "combined"): 5.818879e+10 / 2471952384}
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
    ap.add_argument("--model", default="variant", choices=["variant", "combined"],
                    help="variant: Eq. variant in u (lambda = 5); combined: Eq. newmodel in w = log u "
                         "(lambda1 = 160, lambda2 = 0.004, FP32 form)")
    ap.add_argument("--loop-mode", type=int, default=2,
                    help="0 host chunks of per-trial launches, 1 graph while node of per-trial launches, "
                         "2 one persistent launch per step (default), 3 the same without a graph")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the other forms (TF32, BF16, combined model, batch of 64) in the default line")
    ap.add_argument("--no-peaks", action="store_true", help="skip the peak-rate microbenchmarks")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="paper",
                    choices=["paper", "batch64", "warmstart", "precision", "quality", "cnn"],
                    help="paper: the Mpixel*iter/s workload above; batch64: time to the energy "
                         "tolerance of 64 uneven images in one context vs 64 sequential FP32 solves; "
                         "warmstart: solver-generated pairs, CNN training, then time to tolerance "
                         "from the CNN start vs from f on 512x512 images; precision: one 4096x4096 L=1 "
                         "image in FP32, TF32 and BF16, errors against FP32 and the FP64 oracle; quality: "
                         "PSNR / SSIM of despeckled images over a sweep of the data weights; cnn: inference "
                         "and training-step time of the warm-start network")
    ap.add_argument("--prec-size", type=int, default=4096, help="precision: image side")
    ap.add_argument("--prec-iters", type=int, default=200, help="precision: iterations per form")
    ap.add_argument("--ws-pairs", type=int, default=20000, help="warmstart: 256x256 training pairs")
    ap.add_argument("--ws-steps", type=int, default=4000, help="warmstart: Adam steps")
    ap.add_argument("--ws-batch", type=int, default=32, help="warmstart: crops per Adam step")
    ap.add_argument("--ws-crop", type=int, default=128, help="warmstart: crop side")
    ap.add_argument("--ws-eval", type=int, default=8, help="warmstart: held-out 512x512 images")
    ap.add_argument("--ws-procs", type=int, default=0, help="warmstart: image-generation processes (0: all cores)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--lam", type=float, default=0.02,
                    help="data weight of the batch64 workload (at lambda = 5 the tolerance is met in 1-2 steps)")
    ap.add_argument("--max-iter", type=int, default=3000)
    ap.add_argument("--clocks-csv", default=None,
                    help="where the nvidia-smi clock samples of the timed region are written "
                         "(default: a file in the system's temporary directory)")
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
# combined model (Eq. newmodel): the paper's lambda1, lambda2 for L = 1 (Sec. III-B)
COMBINED_KW = dict(SOLVER_KW, lam=0.004, lam1=160.0, model="combined")


def model_kw(args):
    """Solver keywords of the throughput workload's model."""
    return COMBINED_KW if getattr(args, "model", "variant") == "combined" else SOLVER_KW


def oracle_prm(orc, kw, max_iter):
    """The oracle's parameters for the same model and solver settings."""
    return orc.params(max_iter=max_iter, lam=kw["lam"], beta=kw["beta"], L0=kw["L0"], eta=kw["eta"],
                      c2=kw["c2"], max_backtrack=kw["max_backtrack"],
                      model=orc.MODEL_COMBINED if kw.get("model") == "combined" else orc.MODEL_VARIANT,
                      lam1=kw.get("lam1", 0.0))


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


def cpu_baseline(fs, k, th, iters_total, seconds, kw=SOLVER_KW):
    """The FP64 oracle, as it stands, on a bounded sample: one 256x256 image
    of the workload, as many iterations as fit in about `seconds`."""
    import oracle as orc
    orc.build()
    f = next(x for x in fs if x.shape == (256, 256)) if any(x.shape == (256, 256) for x in fs) else fs[0]
    t0 = time.perf_counter()
    orc.ipiano(f, k, th, oracle_prm(orc, kw, 2))
    per_it = (time.perf_counter() - t0) / 2.0
    n = int(max(2, min(iters_total, seconds / max(per_it, 1e-6))))
    t0 = time.perf_counter()
    out = orc.ipiano(f, k, th, oracle_prm(orc, kw, n))
    dt = time.perf_counter() - t0
    npx = f.size
    cores = orc.num_threads()
    # the same oracle on one core (a few iterations of the same image)
    orc.set_threads(1)
    try:
        t1 = time.perf_counter()
        out1 = orc.ipiano(f, k, th, oracle_prm(orc, kw, 3))
        dt1 = time.perf_counter() - t1
    finally:
        orc.set_threads(cores)
    return {"value": round(npx * out["n"] / dt / 1e6, 4), "unit": "Mpixel*iter/s",
            "cores": cores, "kind": "oracle",
            "sample": "FP64 oracle, one %dx%d image of the workload, %d iPiano iterations "
                      "(%.1f s)" % (f.shape[0], f.shape[1], out["n"], dt),
            "single_core": {"value": round(npx * out1["n"] / dt1 / 1e6, 4), "cores": 1,
                            "sample": "the same image, %d iterations (%.1f s)" % (out1["n"], dt1)}}


def combine_ranks(local_ms, local_units, dist=None, device="cpu"):
    """Replicas: every rank solves its own batch with no exchange on the data
    path.  The job's time is the slowest rank's (MAX) and its work the sum of
    every rank's units (SUM); one rank returns its own numbers."""
    if dist is None:
        return float(local_ms), float(local_units)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def workload_config(args, npix, nimg):
    """The throughput workload's config, shared by both arms."""
    return {"workload": "%dx512^2 + %dx256^2 textured images, L in {1,4,8} gamma speckle, "
                        "48x7x7 seeded bank, %s, %d iPiano iterations with "
                        "Lipschitz backtracking, %s filter bank" % (
                            args.n512, args.n256,
                            "combined model (Eq. newmodel) in w = log u, lambda1=160, "
                            "lambda2=0.004" if args.model == "combined" else "lambda=5",
                            args.iters, args.prec.upper()),
            "images": nimg, "pixels": npix, "iters": args.iters, "precision": args.prec,
            "model": args.model}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    fs, k, th, shapes, Ls = workload(min(args.n512, 1), min(args.n256, 1))
    import oracle as orc
    orc.build()
    f = fs[-1]
    prm = oracle_prm(orc, model_kw(args), 4)
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
            "config": workload_config(args, args.n512 * 512 * 512 + args.n256 * 256 * 256, args.n512 + args.n256),
            "cpu_baseline": {"value": round(value, 4), "unit": "Mpixel*iter/s", "cores": orc.num_threads(),
                             "kind": "oracle",
                             "sample": "FP64 oracle (the reference arm: the paper ships no code), each step a "
                                       "bounded sample of the workload: one 256x256 image of the batch, "
                                       "4 iPiano iterations"},
            "e2e": {"value": round(value, 4), "unit": "Mpixel*iter/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def batch64_inputs():
    """The batching form's workload: 64 textured images, sides log-uniform in
    [128, 1536] (seed 7), L alternating 1 / 4, the seeded bank."""
    from paper_1404_5344_gb300 import synth
    sizes = synth.uneven_sizes(64, 128, 1536, seed=7)
    fs = []
    for j, s in enumerate(sizes):
        u = synth.textured_image(s, s, seed=2000 + j)
        fs.append(synth.speckle(u, L=1.0 if j % 2 == 0 else 4.0, seed=6000 + j))
    k, th = synth.filter_bank(48, 7, seed=0, theta=0.1)
    return sizes, fs, k, th


def _event_timer(torch, stream):
    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out
    return timed


def batch64_batched(fe, torch, f_dev, k, th, prec, kw, steps, warmup, tol, max_iter, stream):
    """Time to tolerance of the whole batch in ONE context (one CUDA-graph
    launch drives every image's device-side loop); includes the restart from
    f, excludes context creation.  Returns (best ms, per-image infos, tile)."""
    timed = _event_timer(torch, stream)
    batch = fe.Solver(f_dev, k, th, prec=prec, stream=stream, **kw)
    tile = batch.tile
    for _ in range(max(1, warmup)):
        batch.reset(f_dev)
        batch.solve(max_iter, tol)
    t = []
    st = None
    for _ in range(max(1, steps)):
        batch.reset(f_dev)
        ms, st = timed(lambda: batch.solve(max_iter, tol))
        t.append(ms)
    infos = [batch.info(i) for i in range(len(f_dev))]
    batch.close()
    return min(t), infos, tile, st


def batch64_sequential(fe, torch, f_dev, k, th, kw, tol, max_iter, stream):
    """64 sequential single-image FP32 solves at the same tolerance (each
    context autotunes its own tile); the sum of their event times."""
    timed = _event_timer(torch, stream)
    singles = [fe.Solver([f], k, th, prec="fp32", stream=stream, **kw) for f in f_dev]
    for j in range(min(4, len(singles))):
        singles[j].reset([f_dev[j]])
        singles[j].solve(max_iter, tol)
    t_seq, its, per = 0.0, [], []
    for j, s in enumerate(singles):
        s.reset([f_dev[j]])
        ms, _ = timed(lambda: s.solve(max_iter, tol))
        t_seq += ms
        its.append(s.info(0)["n"])
        per.append({"side": int(f_dev[j].shape[0]), "iterations": its[-1], "ms": round(ms, 3),
                    "tile": "%dx%d%s" % (s.tile + ("/cluster4" if s.cluster == 4 else "",))})
        s.close()
    batch64_sequential.per_image = per
    return t_seq, its


def run_batch64(args):
    """Batching form: 64 textured images, sides log-uniform in [128, 1536]
    (seeded), L alternating 1 / 4, solved to |H^{n+1} - H^n| / |H^{n+1} - G(f)| < tol
    in ONE context (one CUDA-graph launch drives every image's device-side
    loop, per-image alpha_n and L_n) in the requested form, against 64
    sequential single-image FP32 solves at the same tolerance.  Both timings
    include the restart from f (initial gradient) and exclude context
    creation; CUDA events on the solvers' stream."""
    import torch
    from paper_1404_5344_gb300 import build
    build.build()
    from paper_1404_5344_gb300 import fe
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    sizes, fs, k, th = batch64_inputs()
    npix = sum(s * s for s in sizes)
    stream = torch.cuda.Stream()
    f_dev = [torch.from_numpy(f).cuda() for f in fs]
    torch.cuda.synchronize()
    kw = dict(SOLVER_KW, lam=args.lam)
    tb, infos, tile, st = batch64_batched(fe, torch, f_dev, k, th, args.prec, kw, args.steps, args.warmup,
                                          args.tol, args.max_iter, stream)
    its = [x["n"] for x in infos]
    trials = [x["trials"] for x in infos]
    t_seq, its_seq = batch64_sequential(fe, torch, f_dev, k, th, kw, args.tol, args.max_iter, stream)
    line = {"metric": "time to |dH|/|H - G(f)| < %g (s)" % args.tol, "value": round(tb / 1e3, 4), "unit": "s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "bf16r": "bf16", "tf32": "tf32"}[args.prec],
            "data": "synthetic",
            "config": {"workload": "64 textured images, sides log-uniform in [128, 1536] (seed 7), L in {1, 4}, "
                                   "48x7x7 seeded bank, lambda=%g, tol=%g on |dH|/|H - G(f)|, max_iter=%d" % (
                                       args.lam, args.tol, args.max_iter),
                       "pixels": npix, "precision": args.prec, "loop": "one CUDA-graph launch per solve",
                       "tile": "%s (autotuned for the batch; each sequential solve autotunes its own)" % (tile,)},
            "sequential_fp32_s": round(t_seq / 1e3, 4),
            "speedup_vs_sequential_fp32": round(t_seq / tb, 3),
            "iterations": {"batched_min": min(its), "batched_max": max(its), "batched_mean": round(sum(its) / len(its), 2),
                           "sequential_mean": round(sum(its_seq) / len(its_seq), 2)},
            "trials_max": max(trials), "status": st,
            "per_image_sequential": getattr(batch64_sequential, "per_image", None),
            "mpixel_iter_per_s": round(sum(n * s * s for n, s in zip(its, sizes)) / (tb / 1e3) / 1e6, 2)}
    print(json.dumps(line), flush=True)
    return 0


def run_warmstart(args):
    """Warm-start form: ``--ws-pairs`` seeded 256x256 observations (L
    alternating 1 / 4) converged by the batched FP32 solver to the energy
    tolerance, the 5-layer CNN trained on random crops of those pairs by the
    library's own forward / backward / Adam kernels, then ``--ws-eval``
    held-out 512x512 observations solved to the same tolerance from f and
    from u0 = CNN(f) (falling back to f where H(u0) >= H(f)).  value = the
    warm-started time (CNN inference + solve) summed over the held-out
    images; CUDA events on the solvers' stream."""
    from paper_1404_5344_gb300 import synth, warmstart
    procs = args.ws_procs or os.cpu_count() or 1
    t0 = time.perf_counter()
    F, _ = warmstart.make_observations(args.ws_pairs, 256, seed=200_000, procs=procs)
    Ft, _ = warmstart.make_observations(args.ws_eval, 512, seed=900_000, procs=min(procs, args.ws_eval))
    t_gen = time.perf_counter() - t0
    import torch
    from paper_1404_5344_gb300 import build
    build.build()
    from paper_1404_5344_gb300 import fe
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    k, th = synth.filter_bank(48, 7, seed=0, theta=0.1)
    kw = dict(SOLVER_KW, lam=args.lam)
    stream = torch.cuda.Stream()
    Fd = torch.from_numpy(F).cuda()
    del F
    torch.cuda.synchronize()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3, out

    t_sol, (Ud, its) = timed(lambda: warmstart.solve_targets(Fd, k, th, tol=args.tol, max_iter=args.max_iter,
                                                             batch=256, stream=stream, solver_kw=kw))
    net = fe.CNN(seed=1, stream=stream)
    with torch.cuda.stream(stream):
        t_train, losses = timed(lambda: warmstart.train(net, Fd, Ud, args.ws_steps, batch=args.ws_batch,
                                                         crop=args.ws_crop, lr=2e-3, seed=0, decay_from=0.5))
    del Fd, Ud
    fts = [torch.from_numpy(x).cuda() for x in Ft]
    # one untimed pass warms the contexts' code paths, then the timed pass
    warmstart.evaluate(net, fts[:1], k, th, tol=args.tol, max_iter=args.max_iter, stream=stream, solver_kw=kw)
    res = warmstart.evaluate(net, fts, k, th, tol=args.tol, max_iter=args.max_iter, stream=stream, solver_kw=kw)
    t_plain = sum(r["ms_plain_eq"] for r in res) / 1e3
    t_warm = sum(r["ms_cnn"] + r["ms_warm_eq"] for r in res) / 1e3
    dec = [(r["H_f"] - r["H_plain"]) for r in res]
    line = {"metric": "time to the energy H* = H_plain + 1e-3 (H(f) - H_plain) from the CNN start (s); H_plain = "
                      "energy where plain iPiano meets |dH|/|H - G(f)| < %g" % args.tol,
            "value": round(t_warm, 4), "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "warm start: %d seeded 256x256 textured observations (L in {1, 4}) "
                                   "converged by the batched FP32 solver, CNN 5x conv3x3 32 ch BF16 weights "
                                   "trained %d Adam steps on %d crops of %dx%d, evaluated on %d held-out "
                                   "512x512 observations; lambda=%g, tol=%g, max_iter=%d" % (
                                       args.ws_pairs, args.ws_steps, args.ws_batch, args.ws_crop, args.ws_crop,
                                       args.ws_eval, args.lam, args.tol, args.max_iter)},
            "plain_fp32_s": round(t_plain, 4), "speedup_vs_plain": round(t_plain / t_warm, 3),
            "iterations": {"plain": sum(r["iters_plain_eq"] for r in res),
                           "warm": sum(r["iters_warm_eq"] for r in res),
                           "per_image_plain": [r["iters_plain_eq"] for r in res],
                           "per_image_warm": [r["iters_warm_eq"] for r in res]},
            "all_reached_target": all(r["reached_plain_eq"] and r["reached_warm_eq"] for r in res),
            "cnn_used": sum(r["used_cnn"] for r in res), "cnn_ms_per_image": round(
                sum(r["ms_cnn"] for r in res) / len(res), 4),
            "relative_change_rule_alone": {
                "plain_s": round(sum(r["ms_plain"] for r in res) / 1e3, 4),
                "warm_s": round(sum(r["ms_cnn"] + r["ms_warm"] for r in res) / 1e3, 4),
                "iterations_plain": [r["iters_plain"] for r in res],
                "iterations_warm": [r["iters_warm"] for r in res],
                "energy_gap_rel_to_decrease": [round((r["H_warm"] - r["H_plain"]) / d, 6)
                                               for r, d in zip(res, dec)]},
            "all_converged": all(r["converged_plain"] and r["converged_warm"] for r in res),
            "pipeline_s": {"generate_cpu": round(t_gen, 2), "solve_targets": round(t_sol, 2),
                           "train": round(t_train, 2)},
            "targets_iterations": {"min": min(its), "mean": round(float(np.mean(its)), 1), "max": max(its)},
            "train_loss": {"first100": round(float(np.mean(losses[:100])), 5),
                           "last100": round(float(np.mean(losses[-100:])), 5)}}
    print(json.dumps(line), flush=True)
    return 0


def _round_bank(k, prec):
    """The precision form's model: the bank rounded once to the operand type
    (BF16 round-to-nearest-even, TF32 round-to-nearest, ties away)."""
    if prec == "fp32":
        return np.asarray(k, np.float32)
    b = np.ascontiguousarray(k, np.float32).view(np.uint32).astype(np.uint64)
    if prec in ("bf16", "bf16r"):
        b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    else:
        b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32).reshape(np.shape(k))


def run_precision(args):
    """Precision forms on one large image (L = 1, lambda = 0.02, the same
    iteration count for every form): final u against the FP32 run, PSNR
    against the clean image, and the error of single steps against the FP64
    oracle with the form's rounded bank on 512 x 512 crops.  A crop step is
    exact by construction: grad F has a radius of 6 pixels, so the oracle
    steps a window with a 6-pixel margin from the GPU's own (u^n, u^{n-1})
    at the GPU's L_n and only the inner crop is compared."""
    import torch
    from paper_1404_5344_gb300 import build, synth
    build.build()
    from paper_1404_5344_gb300 import fe
    import oracle as orc
    orc.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    S, n_it = args.prec_size, args.prec_iters
    clean = synth.textured_image(S, S, seed=31)
    f = synth.speckle(clean, L=1.0, seed=32)
    k, th = synth.filter_bank(48, 7, seed=0, theta=0.1)
    kw = dict(SOLVER_KW, lam=args.lam)
    stream = torch.cuda.Stream()
    fd = torch.from_numpy(f).cuda()
    crops = [(0, 0), (S // 2 - 256, S // 2 - 256), (S - 512, S - 512)]
    checkpoints = [0, n_it // 2, n_it - 1]
    res, u_fp32 = {}, None
    for prec in ("fp32", "tf32", "bf16", "bf16r"):
        kq = _round_bank(k, prec).astype(np.float64)
        prm = orc.params(lam=kw["lam"], beta=kw["beta"], L0=kw["L0"], eta=kw["eta"], c2=kw["c2"], max_iter=1)
        step_err = 0.0
        with fe.Solver([fd], k, th, prec=prec, stream=stream, **kw) as s:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            done, t_ms = 0, 0.0
            for c in checkpoints:
                if c > done:
                    e0.record(stream)
                    s.step(c - done, sync=False)
                    e1.record(stream)
                    e1.synchronize()
                    t_ms += e0.elapsed_time(e1)
                    done = c
                u, up, _, info = s.get_state(0)
                assert s.step(1) == fe.FE_OK
                done += 1
                u1 = s.get_u(0)
                L = s.info(0)["L"]
                for (y, x) in crops:
                    y0, x0 = max(0, y - 6), max(0, x - 6)
                    y1, x1 = min(S, y + 512 + 6), min(S, x + 512 + 6)
                    r = orc.ipiano_fixed(f[y0:y1, x0:x1], kq, th, prm, [L], u[y0:y1, x0:x1], up[y0:y1, x0:x1])
                    # the crop lies >= 6 pixels inside the window except at image borders
                    ref = r["u"][y - y0:y - y0 + 512, x - x0:x - x0 + 512]
                    got = u1[y:y + 512, x:x + 512]
                    step_err = max(step_err, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
            if done < n_it:
                e0.record(stream)
                s.step(n_it - done, sync=False)
                e1.record(stream)
                e1.synchronize()
                t_ms += e0.elapsed_time(e1)
            uf = s.get_u(0)
            info = s.info(0)
        if prec == "fp32":
            u_fp32 = uf
        res[prec] = {"step_err_vs_oracle": step_err,
                     "final_u_err_vs_fp32": float(np.max(np.abs(uf.astype(np.float64) - u_fp32))
                                                  / np.max(np.abs(u_fp32))),
                     "final_u_mean_abs_err_vs_fp32": float(np.mean(np.abs(uf.astype(np.float64) - u_fp32))
                                                           / np.mean(np.abs(u_fp32))),
                     "psnr_db": round(synth.psnr(uf, clean), 6), "iterations": int(info["n"]),
                     "H": info["H"], "ms_per_iter": round(t_ms / max(1, n_it - len(checkpoints)), 4)}
    for prec in res:
        res[prec]["psnr_delta_vs_fp32_db"] = round(res[prec]["psnr_db"] - res["fp32"]["psnr_db"], 6)
    traj = precision_trajectory(fe, orc, stream, args)
    line = {"metric": "precision forms: error against FP32 and the FP64 oracle", "value":
            res["bf16"]["psnr_delta_vs_fp32_db"], "unit": "dB (BF16 PSNR - FP32 PSNR)", "n_gpus": 1,
            "higher_is_better": True, "vs_baseline": None, "dtype": "f32/tf32/bf16", "data": "synthetic",
            "config": {"workload": "%dx%d textured image (seed 31), L=1 speckle (seed 32), 48x7x7 seeded bank, "
                                   "lambda=%g, %d iPiano iterations per form; oracle steps on three 512x512 crops "
                                   "(corner, centre, corner) at iterations %s" % (S, S, args.lam, n_it, checkpoints)},
            "psnr_noisy_db": round(synth.psnr(f, clean), 4), "forms": res, "trajectory_vs_fp64_oracle": traj}
    print(json.dumps(line), flush=True)
    return 0


def precision_trajectory(fe, orc, stream, args, S=512, n_it=200):
    """Final-u error of every form after n_it iterations on one S x S image
    (L = 1, lambda = args.lam) against the FP64 oracle iterating with the
    GPU's accepted L_n replayed (fixed-L update rule), with the form's rounded
    bank and with the unrounded FP32 bank; PSNR against the clean image."""
    from paper_1404_5344_gb300 import synth
    clean = synth.textured_image(S, S, seed=43)
    f = synth.speckle(clean, L=1.0, seed=44)
    k, th = synth.filter_bank(48, 7, seed=0, theta=0.1)
    kw = dict(SOLVER_KW, lam=args.lam)
    prm = orc.params(lam=kw["lam"], beta=kw["beta"], L0=kw["L0"], eta=kw["eta"], c2=kw["c2"], max_iter=1)
    out = {"workload": "%dx%d textured image (seed 43), L=1 speckle (seed 44), lambda=%g, %d iterations; oracle "
                       "with the GPU's L_n replayed" % (S, S, args.lam, n_it)}
    cache = {}
    for prec in ("fp32", "tf32", "bf16", "bf16r"):
        Ls = []
        with fe.Solver([f], k, th, prec=prec, stream=stream, **kw) as s:
            for _ in range(n_it):
                s.step(1)
                Ls.append(s.info(0)["L"])
            ug = s.get_u(0).astype(np.float64)
        r = {"psnr_db": round(synth.psnr(ug, clean), 6)}
        for name, kb in (("rounded_bank", _round_bank(k, prec)), ("fp32_bank", np.asarray(k, np.float32))):
            key = (name if prec != "fp32" else "fp32_bank", prec if name == "rounded_bank" else "fp32", tuple(Ls))
            if key not in cache:
                cache[key] = orc.ipiano_fixed(f, kb.astype(np.float64), th, prm, Ls, f)["u"]
            u_ref = cache[key]
            r[name] = {"max_rel": float(np.max(np.abs(ug - u_ref)) / np.max(np.abs(u_ref))),
                       "mean_rel": float(np.mean(np.abs(ug - u_ref)) / np.mean(np.abs(u_ref))),
                       "psnr_delta_db": round(synth.psnr(ug, clean) - synth.psnr(u_ref, clean), 6)}
        out[prec] = r
    return out


def run_cnn(args):
    """The warm-start network alone (fe_cnn_*): inference u0 = f exp(CNN(log f))
    on one 512x512 observation and one Adam training step on 32 crops of
    128x128, each the mean of args.steps calls after args.warmup, CUDA events
    on the network's stream.  Seeded observations in [15, 240]; the targets of
    the training step are 1.01 f (the step's cost does not depend on them)."""
    import torch
    from paper_1404_5344_gb300 import build
    build.build()
    from paper_1404_5344_gb300 import fe
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream()
    net = fe.CNN(seed=1, stream=stream)
    rng = np.random.default_rng(0)
    f = torch.from_numpy(rng.uniform(15, 240, (512, 512)).astype(np.float32)).cuda()
    fb = torch.from_numpy(rng.uniform(15, 240, (32, 128, 128)).astype(np.float32)).cuda()
    ub = fb * 1.01
    u0 = torch.empty_like(f)
    torch.cuda.synchronize()

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / args.steps

    with torch.cuda.stream(stream):
        t_inf = timed(lambda: net.forward(f, u0=u0))
        t_train = timed(lambda: net.train_step(fb, ub, 1e-4))
    line = {"metric": "warm-start CNN inference time per 512x512 observation", "value": round(t_inf, 4), "unit": "ms",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "vs_baseline": None, "dtype": "bf16 weights, f32 activations", "data": "synthetic",
            "config": {"workload": "5-layer 3x3 CNN 1-32-32-32-32-1; inference on one 512x512 observation, one "
                                   "Adam step on 32 crops of 128x128"},
            "train_step_ms": round(t_train, 4)}
    print(json.dumps(line), flush=True)
    return 0


# the paper's (lambda1, lambda2) of the combined model per number of looks (Sec. III-B)
PAPER_LAMBDAS = {1: (160.0, 0.004), 3: (310.0, 0.008), 8: (550.0, 0.02)}


def run_quality(args):
    """PSNR and SSIM (fe_psnr, fe_ssim) of despeckled synthetic images against
    their clean versions, over a sweep of the data weights: for each number
    of looks L in {1, 3, 8} (three 256 x 256 textured images each), the
    combined model at 1/4, 1 and 4 times the paper's (lambda1, lambda2) for
    that L, the log-domain model (lambda2 = 0) and the variant model at the
    same factors of lambda1 and lambda2; each with the seeded bank as built
    and scaled by 0.05 (the bank is not the paper's learned one, and its
    scale sets where rho' acts).  Solves to tol on the relative energy
    change, max_iter iterations at most."""
    import torch
    from paper_1404_5344_gb300 import build, synth
    build.build()
    from paper_1404_5344_gb300 import fe
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    k, th = synth.filter_bank(48, 7, seed=0, theta=0.1)
    stream = torch.cuda.Stream()
    tol, max_it = max(args.tol, 1e-5), min(args.max_iter, 1000)
    results, t0 = [], time.perf_counter()
    for L, (l1, l2) in PAPER_LAMBDAS.items():
        clean = [synth.textured_image(256, 256, seed=700 + 10 * L + j) for j in range(3)]
        noisy = [synth.speckle(c, L=float(L), seed=800 + 10 * L + j) for j, c in enumerate(clean)]
        cd = [torch.from_numpy(c).cuda() for c in clean]
        nd = [torch.from_numpy(n).cuda() for n in noisy]
        base = {"L": L, "psnr": float(np.mean([fe.psnr(n, c) for n, c in zip(nd, cd)])),
                "ssim": float(np.mean([fe.ssim(n, c) for n, c in zip(nd, cd)]))}
        results.append(dict(base, config="noisy"))
        for scale in (1.0, 0.05):
            for m in (0.25, 1.0, 4.0):
                for name, kw in (("combined", dict(model="combined", lam=m * l2, lam1=m * l1)),
                                 ("log-domain", dict(model="combined", lam=0.0, lam1=m * l1)),
                                 ("variant", dict(lam=m * l2))):
                    kw = dict(SOLVER_KW, **kw)
                    with fe.Solver(nd, k * scale, th, stream=stream, **kw) as s:
                        st = s.solve(max_it, tol)
                        us = [s.get_u(j, out=torch.empty_like(nd[j])) for j in range(3)]
                        its = [s.info(j)["n"] for j in range(3)]
                    results.append({"L": L, "config": name, "factor": m, "bank_scale": scale,
                                    "lambda1": kw.get("lam1", 0.0), "lambda2": kw["lam"],
                                    "psnr": float(np.mean([fe.psnr(u, c) for u, c in zip(us, cd)])),
                                    "ssim": float(np.mean([fe.ssim(u, c) for u, c in zip(us, cd)])),
                                    "iterations": its, "status": int(st)})
    best = {}
    for r in results:
        if r["config"] != "noisy" and (r["L"] not in best or r["ssim"] > best[r["L"]]["ssim"]):
            best[r["L"]] = r
    line = {"metric": "despeckling quality sweep (mean SSIM of the best setting at L=1)",
            "value": round(best[1]["ssim"], 4), "unit": "SSIM", "n_gpus": 1, "higher_is_better": True,
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "3 textured 256x256 images per L in {1, 3, 8}; combined, log-domain and "
                                   "variant models at 1/4, 1, 4 x the paper's lambdas per L; bank scale 1 and "
                                   "0.05; tol %g, max_iter %d" % (tol, max_it)},
            "seconds": round(time.perf_counter() - t0, 2),
            "best": {str(L): {k2: v for k2, v in r.items() if k2 != "iterations"} for L, r in best.items()},
            "results": [{k2: (round(v, 4) if isinstance(v, float) else v) for k2, v in r.items()} for r in results]}
    print(json.dumps(line), flush=True)
    return 0


PEAK_KINDS = ("ffma", "ffma2", "dfma", "mufu_rcp", "mufu_lg2", "tc_bf16", "tc_tf32")


def measure_peaks(fe, local):
    """Measured rates of the units the kernels are bound by (fe_peak: CUDA
    events, each kind timed in isolation, best of 5 launches of ~20 ms), with
    the SM clocks sampled meanwhile.  FMA and tensor kinds in TFLOP/s, MUFU
    kinds in Tinstr/s."""
    clocks = ClockSampler(local, os.path.join(tempfile.gettempdir(), "fe_peak_clocks_%d.csv" % os.getpid()))
    out = {}
    try:
        for kind in PEAK_KINDS:
            r = fe.peak(kind, target_ms=20.0, reps=5)
            out[kind] = round(r["rate"] / 1e12, 3)
    finally:
        clk = clocks.stop()
    out["unit"] = "TFLOP/s (fma, tensor kinds); Tinstr/s (mufu kinds)"
    out["sms"] = fe.device_sms()
    out["clocks"] = clk
    out["method"] = ("fe_peak: CUDA-core kinds on every SM at full occupancy, 8 independent chains per "
                     "thread; tensor kinds one CTA per SM issuing M128xN256 tcgen05.mma (K 16 BF16, 8 TF32) "
                     "into one TMEM accumulator; best of 5 launches of ~20 ms after a warm-up")
    return out


LOOP_NAMES = {0: "host chunks of per-trial launches",
              1: "cuda-graph while node of per-trial launches",
              2: "one persistent launch per step (cuda graph)",
              3: "one persistent launch per step (no graph)"}


def measure_throughput(fe, torch, args, f_dev, k, th, shapes, prec, model, steps, warmup, stream, flush,
                       clock_path=None, dist=None, local=0):
    """One throughput measurement of the workload: `warmup` untimed steps,
    then `steps` timed steps (each: restart every image from f + args.iters
    iPiano iterations of the whole batch through the C ABI), a 256 MiB buffer
    written before each step (L2 flush), CUDA events on the solver's stream."""
    kw = COMBINED_KW if model == "combined" else SOLVER_KW
    solver = fe.Solver(f_dev, k, th, prec=prec, stream=stream, loop_mode=args.loop_mode, **kw)
    tile, cluster = solver.tile, solver.cluster

    def one_step():
        solver.reset(f_dev)
        ev_l0 = torch.cuda.Event(enable_timing=True)
        ev_l0.record(stream)
        solver.step(args.iters, sync=False)
        return ev_l0

    for _ in range(warmup):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local, clock_path) if clock_path else None
    total_ms, loop_ms = 0.0, 0.0
    lc0 = solver.launch_count()
    pix_iters, trials, pix_trials = 0, 0, 0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        el = one_step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        loop_ms += el.elapsed_time(e1)
        # fe_reset restarts the counters: n = accepted iterations of this step
        infos = [solver.info(i) for i in range(len(f_dev))]
        pix_iters += sum(x["n"] * h * w for x, (h, w) in zip(infos, shapes))
        trials += sum(x["trials"] for x in infos)
        pix_trials += sum(x["trials"] * h * w for x, (h, w) in zip(infos, shapes))
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    launches = solver.launch_count() - lc0
    statuses = sorted({x["status"] for x in infos})
    solver.close()
    return {"total_ms": total_ms, "loop_ms": loop_ms, "pix_iters": pix_iters, "trials": trials,
            "pix_trials": pix_trials, "launches": launches, "statuses": statuses, "tile": tile,
            "cluster": cluster, "clocks": clk, "steps": steps}


def roofline_of(prec, model, r, npix, peaks, sm_mhz_max, loop_mode=2):
    """Roofline object of the trial kernel: algorithmic work (9408 flop per
    pixel per trial, every image-trial that ran) over the device time of the
    iteration loop, against the measured peak of the unit that bounds it."""
    achieved = FLOP_PER_PIXEL_TRIAL * r["pix_trials"] / (r["loop_ms"] / 1e3) / 1e12
    sms = peaks.get("sms") or 0
    # time of one trial launch over the whole batch, from the work-weighted
    # average: loop time / (pixel-trials / pixels); late launches of a step
    # cover only the images still iterating, so a plain average per launch
    # would not be a full-batch time
    full_ms = r["loop_ms"] / (r["pix_trials"] / npix)
    # loop modes 2 and 3 run one persistent launch per step (one-CTA tiles)
    persistent = loop_mode in (2, 3) and r["cluster"] == 1
    mode_name = "MODE_PTRIAL" if persistent else "MODE_TRIAL"
    bpt = TRAFFIC_PER_PIXEL_TRIAL.get((prec, model)) if persistent else None
    if prec == "fp32":
        derived = sms * 128 * 2 * sm_mhz_max * 1e6 / 1e12
        peak = peaks.get("ffma") or derived
        rl = {"bound": "alu", "kernel": "fp32_tile_kernel<%s>" % mode_name,
              "peak_basis": ("measured FP32 FMA rate (fe_peak ffma, %d SMs at full occupancy)" % sms
                             if peaks.get("ffma") else "FP32 FMA from unit counts"),
              "peak_derived": round(derived, 3),
              "peak_derived_basis": "%d SMs (from the device) x 128 FP32 lanes x 2 flop x %.0f MHz (max SM "
                                    "clock)" % (sms, sm_mhz_max)}
    else:
        bf16_sust, src = measured_bf16_sustained()
        ratio = 1.0 if prec in ("bf16", "bf16r") else 1.1 / 2.25
        peak = bf16_sust * ratio
        rl = {"bound": "tensor", "kernel": "tc_tile_kernel<%s, %s>" % (mode_name, prec.upper()),
              "peak_basis": "dense %s tensor peak = %.1f TFLOP/s sustained BF16 (%s) x %.3f" % (
                  prec.upper(), bf16_sust, src, ratio),
              "peak_measured_tcgen05": peaks.get("tc_" + prec[:4]),
              "peak_measured_tcgen05_basis": "fe_peak tc_%s: this library's own M128xN256 tcgen05.mma stream, "
                                             "burst" % prec}
    rl.update({"achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
               "frac": round(achieved / peak, 4),
               "traffic": round(bpt * r["pix_trials"] / r["steps"]) if bpt else None,
               "traffic_per_full_batch_trial": round(bpt * npix) if bpt else None,
               "traffic_basis": ("ncu DRAM bytes of one persistent launch (one step of 24x512^2 + 24x256^2, 300 "
                                 "iterations) = %.2f bytes per pixel-trial, times this run's pixel-trials per launch "
                                 "(one launch per step); per full-batch trial: times the batch's pixels" % bpt
                                 if bpt else None),
               "work": "9408 flop (2 x 48 x 49 MAC) per pixel per trial, every image-trial",
               "ms_per_full_batch_trial": round(full_ms, 4)})
    if prec == "fp32":
        rl["frac_of_derived"] = round(achieved / rl["peak_derived"], 4)
    return rl


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch64(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "quality":
        return run_quality(args)
    if args.workload == "cnn":
        return run_cnn(args)

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
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    r = measure_throughput(fe, torch, args, f_dev, k, th, shapes, args.prec, args.model, args.steps,
                           args.warmup, stream, flush, clock_path=args.clocks_csv or os.path.join(
                               tempfile.gettempdir(), "fe_clocks_%d_rank%d.csv" % (os.getpid(), rank)),
                           dist=dist, local=local)
    clk = r["clocks"]
    T_ms, units = combine_ranks(r["total_ms"], r["pix_iters"], dist, device="cuda")
    value = units / (T_ms / 1e3) / 1e6
    launches = r["launches"]
    # fe_reset launches two kernels per image (prep, data-term floor) and the
    # initial-gradient kernel; fe_step one begin kernel; the rest are trial
    # launches (one per step when the loop is persistent)
    trial_launches = max(1, launches - args.steps * (2 * len(fs) + 2))

    # e2e through the C ABI with host buffers
    kw = model_kw(args)
    f_host = [torch.from_numpy(f).pin_memory() for f in fs]
    u_host = [torch.empty(f.shape, dtype=torch.float32).pin_memory() for f in fs]
    e2e_solver = fe.Solver([x.numpy() for x in f_host], k, th, prec=args.prec, stream=stream,
                           loop_mode=args.loop_mode, **kw)
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
    e2e_T, e2e_units = combine_ranks(e2e_ms / e2e_steps, npix * args.iters, dist, device="cuda")
    e2e_value = e2e_units / (e2e_T / 1e3) / 1e6
    e2e_solver.close()

    # measured peaks (outside the timed region) and the roofline against them
    peaks = measure_peaks(fe, local) if not args.no_peaks else {"sms": fe.device_sms()}
    sm_mhz_max = (clk or {}).get("sm_max_mhz") or 2070.0
    rl = roofline_of(args.prec, args.model, r, npix, peaks, sm_mhz_max, args.loop_mode)

    # the other forms on the same workload (and the batching form), so that
    # one run carries every form's number under the same clock record
    forms = None
    if not args.no_forms and world == 1:
        forms = measure_forms(fe, torch, args, f_dev, k, th, shapes, npix, stream, flush, peaks, sm_mhz_max,
                              local)

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": "Mpixel*iter/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(T_ms / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "bf16": "bf16", "bf16r": "bf16", "tf32": "tf32"}[args.prec], "data": "synthetic",
                "config": dict(workload_config(args, npix, len(fs)), **{
                           "loop": LOOP_NAMES.get(args.loop_mode, str(args.loop_mode)),
                           "tile": "%dx%d%s (%s)" % (r["tile"] + (" on a 4-CTA cluster" if r["cluster"] == 4 else "",
                                                                  "autotuned" if args.prec == "fp32" else "fixed")),
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": "256 MiB buffer written between timed steps; state 6 planes x "
                                 "%.0f MB" % (npix * 4 / 1e6)}),
                "e2e": {"value": round(e2e_value, 2), "unit": "Mpixel*iter/s",
                        "h2d_bytes_per_step": int(npix * 4), "d2h_bytes_per_step": int(npix * 4)},
                "gpu_launches": int(launches), "trial_kernel_launches": int(trial_launches),
                "trials": int(r["trials"]), "pixel_trials": int(r["pix_trials"]), "statuses": r["statuses"],
                "roofline": rl, "clocks": clk, "peaks": peaks}
        if clk and clk.get("sm_mhz") and args.prec == "fp32" and peaks.get("sms"):
            line["roofline"]["frac_of_derived_at_observed_clock"] = round(
                rl["achieved"] / (peaks["sms"] * 128 * 2 * clk["sm_mhz"] * 1e6 / 1e12), 4)
        if forms is not None:
            line["forms"] = forms
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(fs, k, th, args.iters, args.cpu_seconds, kw)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def measure_forms(fe, torch, args, f_dev, k, th, shapes, npix, stream, flush, peaks, sm_mhz_max, local):
    """The precision forms (TF32, BF16) and the combined model on the same
    throughput workload, and the batching form's time to tolerance (FP32 and
    BF16 in one context against 64 sequential FP32 solves), each under its
    own clock record.  Fewer steps than the headline: these are reported
    beside it, not in its place."""
    out = {}
    steps, warmup = max(1, min(args.steps, 5)), max(3, min(args.warmup, 3))
    for name, prec, model in (("bf16", "bf16", args.model), ("bf16r", "bf16r", args.model), ("tf32", "tf32", args.model),
                              ("combined_fp32", "fp32", "combined"), ("combined_bf16", "bf16", "combined")):
        if prec == args.prec and model == args.model:
            continue
        r = measure_throughput(fe, torch, args, f_dev, k, th, shapes, prec, model, steps, warmup, stream, flush,
                               clock_path=os.path.join(tempfile.gettempdir(), "fe_clocks_%d_%s.csv" % (
                                   os.getpid(), name)), local=local)
        out[name] = {"value": round(r["pix_iters"] / (r["total_ms"] / 1e3) / 1e6, 2), "unit": "Mpixel*iter/s",
                     "precision": prec, "model": model, "steps": steps, "warmup": warmup,
                     "ms_per_step": round(r["total_ms"] / steps, 3), "statuses": r["statuses"],
                     "tile": "%dx%d" % r["tile"], "roofline": roofline_of(prec, model, r, npix, peaks, sm_mhz_max, args.loop_mode),
                     "clocks": r["clocks"]}
    # batching form: time to tolerance of 64 uneven images
    sizes, bfs, bk, bth = batch64_inputs()
    bf_dev = [torch.from_numpy(f).cuda() for f in bfs]
    torch.cuda.synchronize()
    kw = dict(SOLVER_KW, lam=args.lam)
    clocks = ClockSampler(local, os.path.join(tempfile.gettempdir(), "fe_clocks_%d_batch64.csv" % os.getpid()))
    res = {}
    for prec in ("fp32", "bf16"):
        tb, infos, tile, st = batch64_batched(fe, torch, bf_dev, bk, bth, prec, kw, 2, 1, args.tol, args.max_iter,
                                              stream)
        its = [x["n"] for x in infos]
        res[prec] = {"s": round(tb / 1e3, 4), "status": st, "tile": str(tile), "iterations_max": max(its),
                     "iterations_mean": round(sum(its) / len(its), 1)}
    t_seq, its_seq = batch64_sequential(fe, torch, bf_dev, bk, bth, kw, args.tol, args.max_iter, stream)
    clk = clocks.stop()
    for prec in res:
        res[prec]["speedup_vs_sequential_fp32"] = round(t_seq / 1e3 / res[prec]["s"], 3)
    out["batch64"] = {"metric": "time to |dH|/|H - G(f)| < %g (s), lower is better" % args.tol,
                      "workload": "64 textured images, sides log-uniform in [128, 1536] (seed 7, %d pixels), "
                                  "L in {1, 4}, lambda=%g, max_iter=%d" % (sum(s * s for s in sizes), args.lam,
                                                                           args.max_iter),
                      "batched": res, "sequential_fp32_s": round(t_seq / 1e3, 4),
                      "sequential_iterations_mean": round(sum(its_seq) / len(its_seq), 1), "clocks": clk}
    return out


if __name__ == "__main__":
    sys.exit(main())
