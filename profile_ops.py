"""Profiling driver: repeated launches of one library operator on random data.

    python profile_ops.py --op up --n 2048 --reps 5

Runs `--reps` launches of the chosen operator through the C ABI on cuda:0
(after building the library) and prints the mean CUDA-event time per launch.
It exists so that an `ncu` capture of a single kernel (`-k`, `-c 1..3`) has a
small, self-contained command line; the inputs are random, since only the
memory traffic and the instruction mix are of interest.

ops:
  down   finest-level k_down (nu sweeps, residual, full weighting), FP32 or
         FP64 (--dtype)
  up     finest-level k_up (cubic prolongation, correction, nu sweeps), FP32
         or FP64 (--dtype)
  outer  outer residual of FP64 data (exact stencil sum) with norms, float output
  conv   one tensor-core SR convolution layer (mode 0: conv + PReLU) on an
         n/2 x n/2 coarse grid of 64 channels
  generator  the whole SR generator (seeded weights) on an n/2 x n/2 coarse
         error: s = max|e|, conv 1->64, the tensor-core layers, conv 64->1
  solve  a whole solve of a seeded turbulent source (host-loop execution, so
         every kernel is a separate launch), mixed or FP64 (--precision);
         time per solve; --cold-start declares x = 0 to the library
         (mg_set_zero_guess), as the bench does
  train  one Adam step of the SR generator trainer on a batch of 4 periodic
         crops of 128^2 coarse pixels (the training configuration; the
         tensor-core GEMMs, or the FP32 CUDA-core GEMMs with --fp32-gemm); time
         per step
  link   the host link: copies of n x n FP64 arrays between pinned host memory
         and the device with cudaMemcpyAsync - host to device (f and x, as a
         solve from host buffers stages them), device to host (x), and both
         directions at once on two streams; GB/s of each (no library kernel)
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["down", "up", "outer", "conv", "generator", "solve", "link", "train"],
                    required=True)
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--nu", type=int, default=2)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32", help="down / up: element type")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed", help="solve: precision")
    ap.add_argument("--fp32-gemm", action="store_true", help="train: FP32 CUDA-core GEMMs instead of tensor cores")
    ap.add_argument("--cold-start", action="store_true", help="solve: declare x = 0 (mg_set_zero_guess)")
    args = ap.parse_args()

    import torch

    from paper_2403_07936_gb300 import build, mg
    build.build()
    dev = torch.device("cuda:0")
    n = args.n
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    if args.op == "link":
        link_bandwidth(n, max(args.reps, 10))
        return
    if args.op in ("down", "up"):
        dt = torch.float64 if args.dtype == "f64" else torch.float32
        x = torch.randn((n, n), device=dev, generator=g, dtype=dt)
        xo = torch.empty_like(x)
        b = torch.randn((n, n), device=dev, generator=g, dtype=dt)
        bc = torch.empty((n // 2, n // 2), device=dev, dtype=dt)
        ec = torch.randn((n // 2, n // 2), device=dev, generator=g, dtype=dt)
        if args.op == "down":
            def run():
                mg.op_down(x, xo, b, bc, nu=args.nu)
        else:
            def run():
                mg.op_up(x, xo, b, ec, nu=args.nu)
    elif args.op == "outer":
        f = torch.randn((n, n), device=dev, dtype=torch.float64, generator=g)
        x = torch.randn((n, n), device=dev, dtype=torch.float64, generator=g)
        s32 = torch.empty((n, n), device=dev, dtype=torch.float32)
        out = torch.empty(4, device=dev, dtype=torch.float64)

        def run():
            mg.op_outer_residual(f, x, 0.0, s32, out)
    elif args.op == "solve":
        import math

        from synthetic.sources import default_kmax, turbulent_source
        ctx = mg.Context(int(math.log2(n // 8)) + 1, n, precision=args.precision)
        ctx.set_graph_execution(False)
        if args.cold_start:
            ctx.set_zero_guess(True)
        f = torch.tensor(turbulent_source(n, default_kmax(n), 1), device=dev)
        x = torch.zeros_like(f)

        def run():
            x.zero_()
            ctx.solve(f, x)
    elif args.op == "train":
        from paper_2403_07936_gb300 import sr
        from synthetic.weights import random_weights
        crop, batch = 128, 4
        tr = mg.Trainer(crop, crop, batch, sr.pack_weights(random_weights(5, gain=0.5)), lr=1e-5)
        tr.tensor_cores = not args.fp32_gemm
        q = torch.randn((batch, crop, crop), device=dev, generator=g)
        tgt = torch.randn((batch, 2 * crop, 2 * crop), device=dev, generator=g) * 0.1

        def run():
            tr.step(q, tgt)
    elif args.op == "generator":
        import math

        from paper_2403_07936_gb300 import sr
        from synthetic.weights import random_weights
        ctx = mg.Context(int(math.log2(n // 8)) + 1, n)
        ctx.load_weights(sr.pack_weights(random_weights(3, gain=0.5)))
        ec = torch.randn((n // 2, n // 2), device=dev, generator=g) * 1e-3
        out = torch.empty((n, n), device=dev)

        def run():
            mg.op_sr_generator(ctx, ec, out)
    else:
        H = W = n // 2
        xin = torch.randn((H + 2, W + 2, 64), device=dev, generator=g).to(torch.bfloat16)
        w = (torch.randn((9, 64, 64), device=dev, generator=g) * 0.05).to(torch.bfloat16)
        bias = torch.zeros(64, device=dev)
        pre = torch.full((64,), 0.2, device=dev)
        out = torch.empty((H + 2, W + 2, 64), device=dev, dtype=torch.bfloat16)

        def run():
            mg.op_sr_conv(0, H, W, xin, None, w, bias, pre, out)
    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    print(f"{args.op} n={n} reps={args.reps} us_per_launch={e0.elapsed_time(e1) / args.reps * 1e3:.2f}")


def link_bandwidth(n: int, reps: int):
    import torch
    dev = torch.device("cuda:0")
    hf = torch.ones((n, n), dtype=torch.float64).pin_memory()
    hx = torch.ones((n, n), dtype=torch.float64).pin_memory()
    df = torch.empty((n, n), dtype=torch.float64, device=dev)
    dx = torch.empty((n, n), dtype=torch.float64, device=dev)
    nbytes = hf.numel() * 8
    side = torch.cuda.Stream()

    def h2d():
        df.copy_(hf, non_blocking=True)
        dx.copy_(hx, non_blocking=True)

    def d2h():
        hx.copy_(dx, non_blocking=True)

    def duplex():
        cur = torch.cuda.current_stream()
        side.wait_stream(cur)
        df.copy_(hf, non_blocking=True)
        with torch.cuda.stream(side):
            hx.copy_(dx, non_blocking=True)
        cur.wait_stream(side)

    for name, fn, moved in (("h2d f+x", h2d, 2 * nbytes), ("d2h x", d2h, nbytes), ("h2d f || d2h x", duplex, 2 * nbytes)):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        print(f"link {name}: {moved / 1e6:.1f} MB in {ms * 1e3:.1f} us = {moved / (ms * 1e-3) / 1e9:.1f} GB/s")


if __name__ == "__main__":
    main()
