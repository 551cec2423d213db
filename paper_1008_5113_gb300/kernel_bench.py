"""Microbenchmark of one hot-path kernel of the engine (for timing and for profilers).

    python -m paper_1008_5113_gb300.kernel_bench --K 10 --walkers 16 --which tri --sweeps 20

builds a context of `walkers` walkers of the K^3 simple-cubic system, optionally takes
them through `sweeps` sweeps of the dense Sherman-Morrison engine first (the state of an
equilibrated chain; the sparse factors are then built from it), and times `reps`
back-to-back applications of one kernel per walker through `vmc_kernel_bench`: the L and
U triangular solves (`tri`), the SpMV in the working precision (`spmv`) or the whole
preconditioner apply (`precond`).  Prints one JSON line: time per apply, algorithmic
bytes per apply and GB/s.  Synthetic inputs from seeds; nothing is read from disk.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--K", type=int, default=10)
    ap.add_argument("--walkers", type=int, default=16)
    ap.add_argument("--kappa", type=float, default=2.0)
    ap.add_argument("--rc", type=float, default=1.5)
    ap.add_argument("--precision", type=int, default=1, help="0 FP64, 1 mixed (FP32 kernels)")
    ap.add_argument("--which", default="tri", choices=["tri", "spmv", "precond"])
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--sweeps", type=int, default=0, help="dense-engine sweeps before the factorisation")
    ap.add_argument("--lfil", type=int, default=-1)
    ap.add_argument("--group", type=int, default=8, help="trisolve_group (1: level by level)")
    ap.add_argument("--row-cap", type=int, default=0, help="trisolve_row_cap (0: the default)")
    args = ap.parse_args(argv)

    import numpy as np
    import torch

    from paper_1008_5113_gb300 import vmc
    from paper_1008_5113_gb300.build import build_library

    build_library()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    systems = [(args.K, 0, 1.0, args.kappa, args.rc)] * args.walkers
    seeds = list(range(1, args.walkers + 1))
    state = None
    if args.sweeps > 0:
        sd = torch.tensor(seeds, dtype=torch.int64, device="cuda")
        ctxd = vmc.vmc_create(systems, vmc.params(precision=0, engine=vmc.ENGINE_DENSE_SM), stream=stream)
        vmc.vmc_init_positions(ctxd, seeds, 0.1)
        vmc.vmc_sweep_async(ctxd, args.sweeps, 0.2, sd)
        vmc.vmc_synchronize(ctxd)
        state = np.concatenate([vmc.vmc_get_positions(ctxd, w).reshape(-1) for w in range(args.walkers)])
        vmc.vmc_destroy(ctxd)
    ctx = vmc.vmc_create(systems, vmc.params(precision=args.precision, lfil_extra=args.lfil,
                                             trisolve_group=args.group, trisolve_row_cap=args.row_cap),
                         stream=stream)
    try:
        if state is None:
            vmc.vmc_init_positions(ctx, seeds, 0.1)
        else:
            vmc.vmc_set_positions_all(ctx, state)
        which = {"tri": 0, "spmv": 1, "precond": 2}[args.which]
        vmc.vmc_kernel_bench(ctx, which, 2)  # warm-up launch
        vmc.vmc_synchronize(ctx)
        vmc.vmc_reset_stats(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        vmc.vmc_kernel_bench(ctx, which, args.reps)
        e1.record(stream)
        torch.cuda.synchronize()
        vmc.vmc_synchronize(ctx)
        ms = e0.elapsed_time(e1)
        st = [vmc.vmc_get_stats(ctx, w) for w in range(args.walkers)]
        by = sum(s["alg_bytes"] for s in st)
        out = {"kernel": args.which, "n": args.K ** 3, "walkers": args.walkers, "precision": args.precision,
               "state_sweeps": args.sweeps, "lfil": args.lfil, "group": args.group, "row_cap": args.row_cap,
               "levels": (st[0]["levels_L"], st[0]["levels_U"]), "groups": (st[0]["groups_L"], st[0]["groups_U"]),
               "stream_bytes": st[0]["stream_bytes"],
               "us_per_apply": 1000.0 * ms / args.reps, "bytes_per_apply": by / args.reps,
               "gbs": by / (ms / 1000.0) / 1e9, "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
        print(json.dumps(out), flush=True)
    finally:
        vmc.vmc_destroy(ctx)


if __name__ == "__main__":
    main()
