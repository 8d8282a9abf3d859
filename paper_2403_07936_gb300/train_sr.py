"""Train the SR prolongation's generator on error pairs produced by the solver.

    python -m paper_2403_07936_gb300.train_sr --out weights.mgsrw

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

Fields of several sizes feed one training set of 128^2 coarse (256^2 fine)
pairs: 256^2 fields as they are (periodic, every pixel in the loss), and
crops of 512^2 to 2048^2 fields (s from the whole field, as in a solve).  A
crop is not periodic, but the trainer's convolutions wrap around its edges,
so the loss mask keeps only the fine pixels whose receptive field (the
generator's reach, 2 n_blocks + 3 coarse cells) stays inside the crop.

Every step of the pair generation runs in the library (mg_solve, mg_vcycle,
mg_op_down, mg_op_up), and the training in its trainer kernels (the
convolutions on the tcgen05 tensor cores with bf16 operands, the trainer's
default for 128-pixel crops); torch only
holds device memory and does casts, crops and the symmetry augmentation (the
eight rotations / reflections of the square and even shifts, which map red
points to red points and coarse node I to fine node 2I, so they are
symmetries of the whole V-cycle; the loss mask is transformed with the
pair).  Seeds start at 10^6 (training) and 2 x 10^6 (validation), disjoint
from the test and benchmark seeds.  The result is a weight blob for
mg_load_prolong_weights and a log of the training.
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


def augment(q, t, gen, m=None):
    """The same random square symmetry and even shift applied to the coarse q,
    the fine t and (if given) the fine loss mask m (batched, last two axes)."""
    import torch
    k = int(torch.randint(0, 4, (1,), generator=gen))
    flip = bool(torch.randint(0, 2, (1,), generator=gen))
    nc, n = q.shape[-1], t.shape[-1]
    sy, sx = (int(v) for v in torch.randint(0, nc, (2,), generator=gen))
    cy, cx = d4_index(nc, k, flip, q.device)
    fy, fx = d4_index(n, k, flip, t.device)
    q = q[..., cy, cx].roll((sy, sx), (-2, -1))
    t = t[..., fy, fx].roll((2 * sy, 2 * sx), (-2, -1))
    if m is None:
        return q.contiguous(), t.contiguous()
    m = m[..., fy, fx].roll((2 * sy, 2 * sx), (-2, -1))
    return q.contiguous(), t.contiguous(), m.contiguous()


def crop_pairs(q, t, crop):
    """Cut whole-field pairs (P, n/2, n/2) / (P, n, n) into non-overlapping
    crop x crop coarse (2 crop fine) pairs."""
    P, nc = q.shape[0], q.shape[-1]
    k = nc // crop
    qc = q.reshape(P, k, crop, k, crop).permute(0, 1, 3, 2, 4).reshape(P * k * k, crop, crop)
    tc = t.reshape(P, k, 2 * crop, k, 2 * crop).permute(0, 1, 3, 2, 4).reshape(P * k * k, 2 * crop, 2 * crop)
    return qc.contiguous(), tc.contiguous()


def interior_mask(crop, reach, dev):
    """Fine-pixel loss weights of a crop: 1 where the pixel's coarse cell is at
    least `reach` cells from every edge of the crop, else 0."""
    import torch
    c = torch.arange(2 * crop, device=dev) // 2
    ok = (c >= reach) & (c < crop - reach)
    return (ok[:, None] & ok[None, :]).float()


def pair_set(mg, sizes, seed0, cycles, crop, reach, dev="cuda:0"):
    """Pairs of every (fine size, sources) in sizes, as crop^2 coarse pairs:
    q (P, crop, crop), t (P, 2 crop, 2 crop), kind (P,) = 0 whole periodic
    field, 1 crop; seeds seed0 + 10^5 * (size index) + i."""
    import torch
    qs, ts, kinds, counts = [], [], [], {}
    for j, (n, m) in enumerate(sizes):
        seeds = [seed0 + 10 ** 5 * j + i for i in range(m)]
        q, t = make_pairs(mg, n, seeds, cycles, dev=dev)
        if n // 2 > crop:
            q, t = crop_pairs(q, t, crop)
            kinds.append(torch.ones(q.shape[0], dtype=torch.int64, device=dev))
        else:
            kinds.append(torch.zeros(q.shape[0], dtype=torch.int64, device=dev))
        qs.append(q)
        ts.append(t)
        counts[n] = int(q.shape[0])
    return torch.cat(qs), torch.cat(ts), torch.cat(kinds), counts


def train(args):
    import numpy as np
    import torch

    from paper_2403_07936_gb300 import build, mg, sr
    from synthetic.weights import random_weights
    build.build()
    dev = "cuda:0"
    crop = args.crop
    reach = 2 * 8 + 3  # generator_reach of the 8-block generator, in coarse cells
    sizes = [tuple(int(v) for v in item.split(":")) for item in args.sizes.split(",")]
    val_sizes = [(n, args.val_sources) for n, _ in sizes]
    t0 = time.time()
    q_tr, t_tr, k_tr, n_tr = pair_set(mg, sizes, 10 ** 6, args.cycles, crop, reach, dev)
    q_va, t_va, k_va, n_va = pair_set(mg, val_sizes, 2 * 10 ** 6, args.cycles, crop, reach, dev)
    t_pairs = time.time() - t0
    masks = torch.stack([torch.ones((2 * crop, 2 * crop), device=dev), interior_mask(crop, reach, dev)])
    w0 = random_weights(args.seed, gain=args.gain)
    w0["out.w"] = w0["out.w"] * 0.01
    w0["out.b"] = w0["out.b"] * 0.0
    tr = mg.Trainer(crop, crop, args.batch, sr.pack_weights(w0), lr=args.lr)
    gen = torch.Generator()
    gen.manual_seed(args.seed)
    yv = torch.empty((args.batch, 2 * crop, 2 * crop), device=dev)

    def val_ratio():
        """||m (t - G(q))|| / ||m t|| over the held-out pairs, per source size
        and in all: the fraction of the cubic's error left after the SR
        correction (1 = no gain)."""
        num, den = {}, {}
        size_of = np.repeat([n for n, _ in val_sizes], [n_va[n] for n, _ in val_sizes])
        for i in range(0, q_va.shape[0] - args.batch + 1, args.batch):
            tr.forward(q_va[i:i + args.batch].contiguous(), yv)
            m = masks[k_va[i:i + args.batch]]
            tv = t_va[i:i + args.batch]
            e = ((m * (yv - tv)) ** 2).sum(dim=(1, 2))
            d = ((m * tv) ** 2).sum(dim=(1, 2))
            for j in range(args.batch):
                n = int(size_of[i + j])
                num[n] = num.get(n, 0.0) + float(e[j])
                den[n] = den.get(n, 0.0) + float(d[j])
        out = {str(n): (num[n] / den[n]) ** 0.5 for n in num}
        out["all"] = (sum(num.values()) / sum(den.values())) ** 0.5
        return out

    log = [{"step": 0, "val_ratio": val_ratio()}]
    P = q_tr.shape[0]
    t1 = time.time()
    for step in range(1, args.steps + 1):
        idx = torch.randint(0, P, (args.batch,), generator=gen).to(dev)
        q, t, m = augment(q_tr[idx], t_tr[idx], gen, masks[k_tr[idx]])
        if step == int(0.7 * args.steps):
            tr.set_lr(args.lr * 0.1)
        loss = tr.step(q, t, m)
        if step % args.log_every == 0 or step == args.steps:
            log.append({"step": step, "loss": loss, "val_ratio": val_ratio(),
                        "elapsed_s": time.time() - t1})
            print(json.dumps(log[-1]), flush=True)
    train_s = time.time() - t1
    blob = tr.weights()
    with open(args.out, "wb") as fp:
        fp.write(blob)
    flop_step = 2 * args.batch * (2 * crop) ** 2 / 4 * 64 * 576 * (16 + 4) * 3  # fwd + 2 bwd GEMMs
    summary = {"sizes": {str(n): c for n, c in sizes}, "crop_coarse": crop, "loss_mask_reach": reach,
               "pairs_train": int(P), "pairs_train_by_size": {str(k): v for k, v in n_tr.items()},
               "pairs_val": int(q_va.shape[0]), "pairs_val_by_size": {str(k): v for k, v in n_va.items()},
               "cycles_per_source": args.cycles, "steps": args.steps, "batch": args.batch, "lr": args.lr,
               "pair_generation_s": t_pairs, "train_s": train_s,
               "train_tflops": flop_step * args.steps / train_s / 1e12, "tensor_cores": tr.tensor_cores,
               "gemm_arithmetic": ("tcgen05 tensor cores, bf16 operands, fp32 accumulation" if tr.tensor_cores
                                   else "fp32 on the CUDA cores"),
               "val_ratio_initial": log[0]["val_ratio"], "val_ratio_final": log[-1]["val_ratio"], "log": log}
    with open(args.out + ".json", "w") as fp:
        json.dump(summary, fp, indent=1)
    return summary


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--sizes", default="256:1334,1024:167,2048:42",
                    help="fine size:sources of the training fields (3 pairs per source; larger fields cropped)")
    ap.add_argument("--crop", type=int, default=128, help="coarse size of a training pair")
    ap.add_argument("--val-sources", type=int, default=8, help="held-out sources per size")
    ap.add_argument("--cycles", type=int, default=3)
    ap.add_argument("--steps", type=int, default=15000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--gain", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--log-every", type=int, default=1000)
    args = ap.parse_args()
    s = train(args)
    print(json.dumps({k: v for k, v in s.items() if k != "log"}))


if __name__ == "__main__":
    main()
