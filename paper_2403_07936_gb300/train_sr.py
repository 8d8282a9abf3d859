"""Train the SR prolongation's generator on error pairs produced by the solver.

    python -m paper_2403_07936_gb300.train_sr --out weights.mgsrw [--steps 6000]

Pairs (Sec. 2.3 / Sec. 3.2 train the generator on coarse / fine fields; here
the fields are the multigrid's own errors).  For a seeded source f on an n x n
periodic grid, with x* its exact solution (a solve to 1e-12) and x_k the
iterate after k mixed-precision V-cycles from zero:

* pre-smooth the top level: x_s = S^nu1(x_k), and restrict its residual,
  b_c = 4 FW(b - A x_s) (one k_down launch);
* the fine-grid error the coarse correction should supply is e_f = x* - x_s
  (mean removed), the coarse error is e_c = A_c^+ b_c (a coarse solve);
* with s = max|e_c|, the generator's input is q = e_c / s and its target
  t = (e_f - P_cubic e_c) / s, so that the SR prolongation
  P_cubic e_c + s G(e_c / s) reproduces e_f.

Every step of the pair generation runs in the library (mg_solve, mg_vcycle,
mg_op_down, mg_op_up), and the training in its trainer kernels; torch only
holds device memory and does casts and the symmetry augmentation (the eight
rotations / reflections of the square and even shifts, which map red points
to red points and coarse node I to fine node 2I, so they are symmetries of the
whole V-cycle).  Seeds start at 10^6, disjoint from the test and benchmark
seeds.  The result is a weight blob for mg_load_prolong_weights.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def make_pairs(mg, n, seeds, cycles, nu=2, dev="cuda:0"):
    """Solver-produced (q, t) pairs: q (P, n/2, n/2), t (P, n, n), float32 on dev."""
    import numpy as np
    import torch

    from synthetic.sources import default_kmax, turbulent_source
    levels = int(np.log2(n // 8)) + 1
    ctx = mg.Context(levels, n)
    ctxc = mg.Context(levels - 1, n // 2)
    h = 2 * np.pi / n
    hc = 2 * h
    qs, ts = [], []
    zeros = torch.zeros((n, n), device=dev)
    for sd in seeds:
        f = torch.tensor(turbulent_source(n, default_kmax(n), sd), device=dev)
        xs = torch.zeros_like(f)
        ctx.solve(f, xs, tol=1e-12)
        b32 = (h * h * (f - f.mean())).float()
        x = torch.zeros_like(f)
        for _ in range(cycles):
            x32 = x.float()
            xsm = torch.empty_like(x32)
            bc = torch.empty((n // 2, n // 2), device=dev)
            mg.op_down(x32, xsm, b32, bc, nu=nu)
            ef = xs - xsm.double()
            ef -= ef.mean()
            fc = (bc.double() / (hc * hc)).contiguous()
            ec = torch.zeros_like(fc)
            ctxc.solve(fc, ec, tol=1e-12)
            ec32 = ec.float().contiguous()
            pe = torch.empty((n, n), device=dev)
            mg.op_up(zeros, pe, zeros, ec32, nu=0)
            s = float(ec32.abs().max()) or 1.0
            qs.append(ec32 / s)
            ts.append(((ef - pe.double()) / s).float())
            ctx.vcycle(f, x)
    return torch.stack(qs), torch.stack(ts)


def d4_index(n, k, flip, dev=None):
    """Gather indices (iy, ix) of the symmetry (rotate k quarter turns, then
    optionally reflect x) of a periodic n x n grid about node (0, 0):
    out = a[..., iy, ix].  A quarter turn maps point (y, x) to (x, -y); the
    reflection maps (y, x) to (y, -x); indices are mod n."""
    import torch
    y = torch.arange(n, device=dev)[:, None].expand(n, n)
    x = torch.arange(n, device=dev)[None, :].expand(n, n)
    if flip:  # out[q] = rot[phi(q)]
        x = (-x) % n
    for _ in range(k):  # rot^k(in)[q] = in[rho^-k(q)], rho^-1(y, x) = (-x, y)
        y, x = (-x) % n, y
    return y, x


def augment(q, t, gen):
    """The same random square symmetry and even shift applied to the coarse q and
    the fine t (batched, last two axes)."""
    import torch
    k = int(torch.randint(0, 4, (1,), generator=gen))
    flip = bool(torch.randint(0, 2, (1,), generator=gen))
    nc, n = q.shape[-1], t.shape[-1]
    sy, sx = (int(v) for v in torch.randint(0, nc, (2,), generator=gen))
    cy, cx = d4_index(nc, k, flip, q.device)
    fy, fx = d4_index(n, k, flip, t.device)
    q = q[..., cy, cx].roll((sy, sx), (-2, -1))
    t = t[..., fy, fx].roll((2 * sy, 2 * sx), (-2, -1))
    return q.contiguous(), t.contiguous()


def train(args):
    import numpy as np
    import torch

    from paper_2403_07936_gb300 import build, mg, sr
    from synthetic.weights import random_weights
    build.build()
    dev = "cuda:0"
    n, nc = args.n, args.n // 2
    t0 = time.time()
    tr_seeds = [10 ** 6 + i for i in range(args.sources)]
    va_seeds = [2 * 10 ** 6 + i for i in range(args.val_sources)]
    q_tr, t_tr = make_pairs(mg, n, tr_seeds, args.cycles)
    q_va, t_va = make_pairs(mg, n, va_seeds, args.cycles)
    t_pairs = time.time() - t0
    w0 = random_weights(args.seed, gain=args.gain)
    w0["out.w"] = w0["out.w"] * 0.01
    w0["out.b"] = w0["out.b"] * 0.0
    tr = mg.Trainer(nc, nc, args.batch, sr.pack_weights(w0), lr=args.lr)
    gen = torch.Generator()
    gen.manual_seed(args.seed)
    yv = torch.empty((args.batch, n, n), device=dev)

    def val_ratio():
        """||t - G(q)|| / ||t|| over the held-out pairs: the fraction of the cubic's
        error left after the SR correction (1 = no gain)."""
        num = den = 0.0
        for i in range(0, q_va.shape[0] - args.batch + 1, args.batch):
            tr.forward(q_va[i:i + args.batch].contiguous(), yv)
            tv = t_va[i:i + args.batch]
            num += float(((yv - tv) ** 2).sum())
            den += float((tv ** 2).sum())
        return (num / den) ** 0.5

    log = [{"step": 0, "val_ratio": val_ratio()}]
    P = q_tr.shape[0]
    t1 = time.time()
    for step in range(1, args.steps + 1):
        idx = torch.randint(0, P, (args.batch,), generator=gen)
        q, t = augment(q_tr[idx.to(dev)], t_tr[idx.to(dev)], gen)
        if step == int(0.7 * args.steps):
            tr.set_lr(args.lr * 0.1)
        loss = tr.step(q, t)
        if step % args.log_every == 0 or step == args.steps:
            log.append({"step": step, "loss": loss, "val_ratio": val_ratio(),
                        "elapsed_s": time.time() - t1})
            print(json.dumps(log[-1]), flush=True)
    blob = tr.weights()
    with open(args.out, "wb") as fp:
        fp.write(blob)
    summary = {"n": n, "pairs_train": int(P), "pairs_val": int(q_va.shape[0]), "cycles_per_source": args.cycles,
               "steps": args.steps, "batch": args.batch, "lr": args.lr, "pair_generation_s": t_pairs,
               "train_s": time.time() - t1, "val_ratio_initial": log[0]["val_ratio"],
               "val_ratio_final": log[-1]["val_ratio"], "log": log}
    with open(args.out + ".json", "w") as fp:
        json.dump(summary, fp, indent=1)
    return summary


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--n", type=int, default=256, help="fine grid of the training fields")
    ap.add_argument("--sources", type=int, default=840)
    ap.add_argument("--val-sources", type=int, default=32)
    ap.add_argument("--cycles", type=int, default=3)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--gain", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--log-every", type=int, default=500)
    args = ap.parse_args()
    s = train(args)
    print(json.dumps({k: v for k, v in s.items() if k != "log"}))


if __name__ == "__main__":
    main()
