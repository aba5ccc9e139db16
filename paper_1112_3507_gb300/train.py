"""Train the learned warm start / preconditioner on solves the plain solver
generates.

    python -m paper_1112_3507_gb300.train --samples 20000 --epochs 6 --out weights.bin

Data: problems `inputs.config_training_2d(seed)` (n x n, density contrast
U[5,30], Ma log-uniform in [1e-3, 1e-1], 1% density noise, smoothed-noise
right-hand side) for seeds first_seed .. first_seed + samples - 1, generated
on CPU worker processes; each is solved to rtol 1e-10 by this library's
batched mixed-precision solver (lm_batch_solve).  Network input: the
feature builder on the rhs (lm_net_features); target: x* / s (s = the
feature builder's scale).  Loss: mean squared error.  Optimiser: Adam on the
FP32 master weights, learning rate decayed by cosine.  Every arithmetic step
runs in the library's kernels; torch only holds device memory.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "unet_16_32_48_64.bin")


def _gen(seed_n):
    seed, n = seed_n
    from paper_1112_3507_gb300 import inputs as I
    p = I.config_training_2d(seed, n=n)
    return (p.rho_old.astype(np.float64).ravel(), p.rho_new.astype(np.float64).ravel(),
            p.cs2.astype(np.float64).ravel(), p.dt, p.f.ravel())


def make_dataset(seeds, n, torch, lm, workers, batch=64, log=print):
    """Features [S, n, n, 3] and normalised targets [S, n, n] on the GPU."""
    S = len(seeds)
    N = n * n
    feats = torch.empty((S, N * 3), dtype=torch.float32, device="cuda")
    targs = torch.empty((S, N), dtype=torch.float32, device="cuda")
    scales = np.zeros(S)
    from paper_1112_3507_gb300 import inputs as I
    proto = I.config_training_2d(int(seeds[0]), n=n)
    grids = [lm.Grid.for_problem(proto) for _ in range(min(batch, S))]
    xbuf = torch.empty(N, dtype=torch.float64, device="cuda")
    fdev = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in grids]
    ctx = mp.get_context("spawn")
    t0 = time.time()
    iters = []
    with ctx.Pool(processes=workers) as pool:
        for b0 in range(0, S, len(grids)):
            chunk = list(range(b0, min(S, b0 + len(grids))))
            data = pool.map(_gen, [(int(seeds[i]), n) for i in chunk])
            for g, fd, d in zip(grids, fdev, data):
                ro, rn, c2, dt, f = d
                g.set_coefficients(ro, rn, c2, dt)
                fd.copy_(torch.from_numpy(f))
                g.set_rhs(fd)
            use = grids[:len(chunk)]
            res = lm.batch_solve(use, rtol=1e-10, max_outer=20, inner_max_iter=12)
            iters += [r["iters"] for r in res]
            for k, (i, g, fd) in enumerate(zip(chunk, use, fdev)):
                s = g.features(fd, feats[i])
                g.solution(xbuf)
                targs[i].copy_((xbuf / s).to(torch.float32))
                scales[i] = s
            if b0 // len(grids) % 20 == 0:
                log(f"  data {b0 + len(chunk)}/{S}  {time.time() - t0:.1f}s  inner iters mean {np.mean(iters):.1f}")
    for g in grids:
        g.close()
    return feats, targs, scales


def train(args, log=print):
    import torch

    from paper_1112_3507_gb300 import lowmach as lm

    torch.cuda.set_device(0)
    n = args.n
    seeds = np.arange(args.first_seed, args.first_seed + args.samples)
    t0 = time.time()
    feats, targs, _ = make_dataset(seeds, n, torch, lm, args.workers, log=log)
    t_data = time.time() - t0
    trms = targs.pow(2).mean(dim=1).sqrt().cpu().numpy()
    log(f"dataset: {args.samples} solves of {n}x{n} in {t_data:.1f}s; target rms "
        f"min {trms.min():.3e} median {np.median(trms):.3e} max {trms.max():.3e}")
    rng = np.random.default_rng(args.seed)
    # He-normal initial weights in the library's parameter order
    net = lm.Net(tuple(args.channels))
    shapes = _param_shapes(3, tuple(args.channels))
    p0 = []
    for name, shp in shapes:
        if len(shp) == 1:
            p0.append(np.zeros(shp))
        else:
            p0.append(rng.standard_normal(shp) * math.sqrt(2.0 / int(np.prod(shp[:-1]))))
    net.set_params(np.concatenate([a.ravel() for a in p0]))
    B = args.batch
    steps_per_epoch = args.samples // B
    total = steps_per_epoch * args.epochs
    y = torch.empty(B * n * n, device="cuda")
    gy = torch.empty_like(y)
    history = []
    t1 = time.time()
    step = 0
    for ep in range(args.epochs):
        perm = torch.as_tensor(rng.permutation(args.samples), device="cuda")
        acc = 0.0
        for k in range(steps_per_epoch):
            idx = perm[k * B:(k + 1) * B]
            x = feats.index_select(0, idx).reshape(-1)
            t = targs.index_select(0, idx).reshape(-1)
            lr = args.lr * 0.5 * (1.0 + math.cos(math.pi * step / max(total, 1)))
            net.forward(x, y, B, n, n)
            want = (k % 50 == 0) or (k == steps_per_epoch - 1)
            loss = net.mse(y, t, gy, want_loss=want)
            net.backward(gy)
            net.adam(max(lr, 1e-6))
            step += 1
            if want:
                acc = loss
                history.append((step, loss))
        log(f"  epoch {ep + 1}/{args.epochs}: loss {acc:.4e}  {time.time() - t1:.1f}s")
    torch.cuda.synchronize()
    t_train = time.time() - t1
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    net.save(args.out)
    summary = {"samples": args.samples, "n": n, "epochs": args.epochs, "batch": B, "lr": args.lr,
               "channels": list(args.channels), "data_seconds": t_data, "train_seconds": t_train,
               "steps": total, "loss_first": history[0][1] if history else None,
               "loss_last": history[-1][1] if history else None, "weights": os.path.abspath(args.out)}
    log(json.dumps(summary))
    return summary


def _param_shapes(cin, ch):
    shapes = []
    prev = cin
    for l, c in enumerate(ch):
        shapes += [(f"A{l}", (3, 3, prev, c)), (f"a{l}", (c,)), (f"B{l}", (3, 3, c, c)), (f"b{l}", (c,))]
        prev = c
    for l in (2, 1, 0):
        cc = ch[l + 1] + ch[l]
        shapes += [(f"C{l}", (3, 3, cc, ch[l])), (f"c{l}", (ch[l],)), (f"D{l}", (3, 3, ch[l], ch[l])),
                   (f"d{l}", (ch[l],))]
    shapes += [("O", (ch[0], 1)), ("o", (1,))]
    return shapes


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--samples", type=int, default=20000)
    ap.add_argument("--first-seed", type=int, default=10000)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--channels", type=int, nargs=4, default=[16, 32, 48, 64])
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    args = ap.parse_args()
    train(args)


if __name__ == "__main__":
    if os.path.dirname(HERE) not in sys.path:
        sys.path.insert(0, os.path.dirname(HERE))
    main()
