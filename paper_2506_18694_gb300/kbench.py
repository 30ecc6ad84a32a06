"""Microbenchmark of one solver kernel through the C ABI (CUDA-event timing).

    python -m paper_2506_18694_gb300.kbench --kernel jacobi --dim 2 --n 4096 --prec c64

Prints one JSON line: average device time per launch and the effective bandwidth from
the kernel's algorithmic bytes (each input vector read once, each output written once).
Inputs of 2D n >= 4096 or 3D n >= 256 exceed the 129 MB L2, so the figure is an HBM one.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import hh

# algorithmic bytes per fine node, per complex entry size e (8 for c64, 16 for c128)
BYTES = {
    "apply": lambda e, d: 2 * e,                      # read x, write y
    "jacobi": lambda e, d: 3 * e,                     # read x, b; write x'
    "resid_restrict": lambda e, d: 2 * e + e / 2 ** d,  # read x, b; write coarse r
    "vcycle": None,                                   # reported as time only
}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", default="jacobi", choices=sorted(BYTES))
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--prec", default="c64", choices=["c64", "c128"])
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--rows", type=int, default=0, help="tile rows/planes (0 = automatic)")
    ap.add_argument("--form", type=int, default=0, help="tile form (options.tile_form)")
    ap.add_argument("--batch", type=int, default=1, help="problems in the batch (vectors nb x nodes)")
    ap.add_argument("--autotune", action="store_true", help="tune tile shapes first")
    args = ap.parse_args(argv)
    prec = hh.HH_C64 if args.prec == "c64" else hh.HH_C128
    dt = torch.complex64 if prec == hh.HH_C64 else torch.complex128
    e = 8 if prec == hh.HH_C64 else 16
    k = 80.0
    bc = [hh.SOMMERFELD] * (2 * args.dim)
    levels = 4 if args.kernel == "vcycle" else 2
    kk = k if args.batch == 1 else [k] * args.batch
    p = hh.Problem(args.dim, args.n, kk, 0.0, k, bc,
                   hh.default_options(precision=prec, levels=levels, restart=1, tile_rows=args.rows,
                                                    tile_form=args.form))
    if args.autotune:
        p.autotune()
    N = p.size()
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(N, dtype=dt, device="cuda", generator=g)
    b = torch.randn(N, dtype=dt, device="cuda", generator=g)
    y = torch.empty_like(x)
    rc = torch.empty(p.size(1), dtype=dt, device="cuda")
    fn = {
        "apply": lambda: p.apply(0, "AL", x, y),
        "jacobi": lambda: p.jacobi(0, b, x, y),
        "resid_restrict": lambda: p.residual_restrict(0, b, x, rc),
        "vcycle": lambda: p.vcycle(b, y),
    }[args.kernel]
    s = torch.cuda.current_stream()
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(s)
    for _ in range(args.reps):
        fn()
    end.record(s)
    end.synchronize()
    t = start.elapsed_time(end) / args.reps / 1e3
    out = {"kernel": args.kernel, "dim": args.dim, "n": args.n, "batch": args.batch, "nodes": N, "prec": args.prec,
           "rows": args.rows, "form": args.form, "autotune": args.autotune, "us": t * 1e6}
    if BYTES[args.kernel] is not None:
        byt = BYTES[args.kernel](e, args.dim) * N
        out.update({"bytes": byt, "gbs": byt / t / 1e9})
    else:
        out["dof_per_s"] = N / t
    p.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
