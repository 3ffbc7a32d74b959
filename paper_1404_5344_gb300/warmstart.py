"""Learned warm start for iPiano: training data made by the solver, training
and inference by the library's CNN kernels (``fe_cnn_*``), and the comparison
against plain iPiano from the observation.

Pipeline (all compute on the GPU through the C ABI; torch only holds device
buffers and cuts crops):

1. ``make_observations``: seeded textured images and gamma speckle (synth).
2. ``solve_targets``: u* = iPiano solution from f (batched contexts, the
   device-side loop, to the relative energy tolerance or a fixed iteration
   count).
3. ``train``: Adam on random crops, loss mean (d - (log u* - log f))^2.
4. ``evaluate``: for held-out images, iterations and device time of plain
   iPiano from f versus iPiano from u0 = CNN(f) to the SAME ENERGY: plain
   iPiano first runs to the relative energy tolerance (its energy H_plain
   there defines the target), then both runs start over and stop at the
   first accepted iterate with H <= H* = H_plain + eps (H(f) - H_plain)
   (fe_solve_to_energy).  The energy H(u0) is checked first: if it is not
   below H(f), the solve starts from f (plain iPiano stays the fallback and
   the measure of the CNN's error).  Runs that stop on the relative-change rule alone are also
   reported (their energies can differ).
"""
from __future__ import annotations

import numpy as np

from . import synth
from .fe import CNN, FE_OK, Solver  # noqa: F401  (re-exported for users)

# lambda = 0.02: the I-divergence weight (lambda_2) of the combined model for
# L = 8 in Sec. III-B; at lambda = 5 the data term pins u to f and the solver
# meets the tolerance after 1-2 steps, which leaves nothing to warm-start
SOLVER_KW = dict(lam=0.02, beta=0.8, L0=1.0, eta=2.0, c2=1e-6, max_backtrack=30)


def _observation(j, size, looks, seed):
    u = synth.textured_image(size, size, seed=seed + j)
    return synth.speckle(u, L=looks[j % len(looks)], seed=seed + 1_000_003 + j), u


def _observation_range(task):
    j0, j1, size, looks, seed = task
    F = np.empty((j1 - j0, size, size), np.float32)
    for j in range(j0, j1):
        F[j - j0] = _observation(j, size, looks, seed)[0]
    return F


def make_observations(n, size, looks=(1.0, 4.0), seed=0, procs=1, chunk=256):
    """n speckled textured images (float32 [n, size, size]) and their clean
    versions.  Image j uses seed + j and L = looks[j % len(looks)], so the
    result does not depend on ``procs``.  With procs > 1 the images are made
    by a spawn-started process pool and the clean images are not returned
    (None): call it before the first CUDA call or not, spawn is safe."""
    if procs <= 1:
        F = np.empty((n, size, size), np.float32)
        U = np.empty((n, size, size), np.float32)
        for j in range(n):
            F[j], U[j] = _observation(j, size, looks, seed)
        return F, U
    import multiprocessing as mp
    tasks = [(a, min(a + chunk, n), size, tuple(looks), seed) for a in range(0, n, chunk)]
    F = np.empty((n, size, size), np.float32)
    with mp.get_context("spawn").Pool(procs) as pool:
        for (a, b, *_), part in zip(tasks, pool.imap(_observation_range, tasks)):
            F[a:b] = part
    return F, None


def solve_targets(F, filters, theta, tol=1e-6, max_iter=1000, prec="fp32", batch=64, stream=None,
                  solver_kw=None):
    """u* for every f in F (a torch CUDA tensor [n, H, W]); returns a torch
    CUDA tensor of the same shape and the accepted iteration counts.  One
    context serves every full batch (fe_reset loads the next f)."""
    import torch
    kw = dict(SOLVER_KW if solver_kw is None else solver_kw)
    Ut = torch.empty_like(F)
    iters = []
    solver = None
    try:
        for a in range(0, F.shape[0], batch):
            fs = [F[i] for i in range(a, min(a + batch, F.shape[0]))]
            if solver is None or solver.nimg != len(fs):
                if solver is not None:
                    solver.close()
                solver = Solver(fs, filters, theta, prec=prec, stream=stream, **kw)
            else:
                solver.reset(fs)
            solver.solve(max_iter, tol)
            for j in range(len(fs)):
                solver.get_u(j, out=Ut[a + j])
                iters.append(solver.info(j)["n"])
    finally:
        if solver is not None:
            solver.close()
    return Ut, iters


def train(cnn, F, Ut, steps, batch=32, crop=64, lr=1e-3, seed=0, log_every=0, decay_from=1.0):
    """Adam on random crops of (F, Ut) (torch CUDA tensors [n, H, W]); the
    learning rate falls linearly to lr/10 over the steps after
    ``decay_from`` x steps.  Returns the per-step losses."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    n, H, W = F.shape
    ar = torch.arange(crop, device=F.device)
    losses = []
    d0 = int(decay_from * steps)
    for it in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g).to(F.device)
        ys = torch.randint(0, H - crop + 1, (batch,), generator=g).to(F.device)
        xs = torch.randint(0, W - crop + 1, (batch,), generator=g).to(F.device)
        yy = (ys[:, None] + ar[None, :])[:, :, None]
        xx = (xs[:, None] + ar[None, :])[:, None, :]
        ii = idx[:, None, None]
        fb = F[ii, yy, xx].contiguous()
        ub = Ut[ii, yy, xx].contiguous()
        lr_t = lr if it < d0 else lr * (1.0 - 0.9 * (it - d0) / max(1, steps - d0))
        losses.append(cnn.train_step(fb, ub, lr_t))
        if log_every and (it + 1) % log_every == 0:
            print("step %d loss %.5f" % (it + 1, float(np.mean(losses[-log_every:]))), flush=True)
    return losses


def evaluate(cnn, fs, filters, theta, tol=1e-6, max_iter=3000, prec="fp32", stream=None, solver_kw=None,
             eps=1e-3):
    """Plain iPiano from f vs iPiano from the CNN prediction, per image (fs:
    list of torch CUDA tensors [H, W]), at equal energy: the target is H* =
    H_plain + eps (H(f) - H_plain), H_plain the energy where plain iPiano
    meets the relative tolerance tol; both runs stop at the first accepted
    iterate with H <= H* (max_iter at most).  Times are CUDA-event device
    times of the solves (the CNN inference is timed separately).  Also
    returned: both runs stopped by the relative-change rule alone."""
    import torch
    kw = dict(SOLVER_KW if solver_kw is None else solver_kw)
    st = stream if stream is not None else torch.cuda.current_stream()
    out = []

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        r = fn()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1), r

    for f in fs:
        with Solver([f], filters, theta, prec=prec, stream=stream, **kw) as plain:
            t_plain, _ = timed(lambda: plain.solve(max_iter, tol))
            ip = plain.info(0)
            H_f = plain.energy(0, f)[0]
            H_star = ip["H"] + eps * (H_f - ip["H"])
            plain.reset([f])
            t_plain_eq, _ = timed(lambda: plain.solve_to_energy(max_iter, H_star))
            ipe = plain.info(0)
        u0 = torch.empty_like(f)
        t_cnn, _ = timed(lambda: cnn.forward(f, u0=u0))
        with Solver([f], filters, theta, prec=prec, stream=stream, u0=u0, **kw) as warm:
            H_u0 = warm.energy(0, u0)[0]
            used = H_u0 < H_f
            start = [u0] if used else None

            def restart():
                warm.reset([f], u0=start)

            restart()
            t_warm_eq, _ = timed(lambda: warm.solve_to_energy(max_iter, H_star))
            iwe = warm.info(0)
            restart()
            t_warm, _ = timed(lambda: warm.solve(max_iter, tol))
            iw = warm.info(0)
        out.append(dict(iters_plain=int(ip["n"]), iters_warm=int(iw["n"]), ms_plain=t_plain,
                        ms_warm=t_warm, ms_cnn=t_cnn, H_plain=ip["H"], H_warm=iw["H"],
                        H_f=H_f, H_u0=H_u0, used_cnn=bool(used),
                        converged_plain=bool(ip["converged"]), converged_warm=bool(iw["converged"]),
                        H_target=H_star, iters_plain_eq=int(ipe["n"]), iters_warm_eq=int(iwe["n"]),
                        ms_plain_eq=t_plain_eq, ms_warm_eq=t_warm_eq,
                        H_plain_eq=ipe["H"], H_warm_eq=iwe["H"],
                        reached_plain_eq=bool(ipe["H"] <= H_star), reached_warm_eq=bool(iwe["H"] <= H_star)))
    return out
