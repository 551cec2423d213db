"""Benchmark of the sparse determinant-ratio engine (one JSON line on rank 0).

Workload: n = 1000 electrons/orbitals on a 10x10x10 simple-cubic lattice (a = 1),
Gaussian orbitals exp(-2 |r - Z|^2) cut at r_c = 1.5, 64 independent walkers
(seeds 1..64), electrons started at the sites + N(0, 0.1^2), Metropolis steps
N(0, 0.2^2), FP64 arithmetic ("plain FP64 batched").  One bench step = one sweep
of every walker: 64 x 1000 determinant ratios through the whole hot path
(proposal, Slater row, ILUTP-preconditioned GMRES solve with refinement,
stability monitor/reorder/refactor, Metropolis test, row commit and
preconditioner update).  Synthetic data, nothing read from disk.

Reported beside the headline: the same workload in mixed precision, the plain
FP64 one-walker-per-launch path (the metric's denominator), the roofline of the
dominant kernel from its algorithmic-byte counter, and the FP64 CPU oracle timed
on the host cores.

Multi-GPU (torchrun): every rank runs its own 64 walkers (weak scaling, replicas:
walkers are independent Markov chains, nothing is exchanged on the data path);
value = all ratios / max-over-ranks time.

--impl reference: the reference arm is the FP64 CPU oracle (Sherman-Morrison
chain of the standard algorithm, OpenMP over walkers) timed on the host cores on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "det-ratio evals/sec over walker batch vs plain FP64 path; % of HBM roofline"
UNIT = "det-ratio evals/s"
K_LAT, KAPPA, RC, A, JITTER, SIGMA, WALKERS = 10, 2.0, 1.5, 1.0, 0.1, 0.2, 64
N = K_LAT ** 3
WORKLOAD = "sc10_n1000_kappa2_rc1.5_w64_fp64"


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def strip_c_comments(text: str) -> str:
    """C/C++/CUDA source without its comments, trailing blanks and empty lines (string and
    character literals are kept as written)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = ("".join(out)).split("\n")
    return "\n".join(ln.rstrip() for ln in lines if ln.strip())


def sources_digest() -> str:
    """SHA-256 over the CUDA sources and the C header with their comments removed: it
    identifies the code the kernels are built from, and comment edits leave it alone."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1008_5113_gb300", "csrc")
    for f in sorted(os.listdir(csrc)) + ["../../include/vmc.h"]:
        path = os.path.normpath(os.path.join(csrc, f))
        if os.path.isfile(path):
            h.update(f.encode())
            h.update(strip_c_comments(open(path, encoding="utf-8").read()).encode())
    return h.hexdigest()


def profiled_traffic(summary: str):
    """DRAM bytes per launch of the dominant kernel from a committed ncu summary, or None
    when the summary is absent or was taken from other kernel sources."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "sources_sha256")):
            k, v = line.strip().strip("`").split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("sources_sha256") != sources_digest() or "traffic_bytes_per_launch" not in fields:
        return None
    return float(fields["traffic_bytes_per_launch"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"vmc_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["no samples"]}
        load = [x for x in sm if smax and x > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_sample(sweeps: int = 1, threads: int = 0):
    """Time the FP64 oracle (explicit inverse + Sherman-Morrison chain) on the host cores:
    one walker per thread (all cores when threads = 0), `sweeps` sweeps of n moves each.
    Returns (record, ratios, seconds)."""
    import numpy as np

    import oracle

    oracle.build()
    threads = threads if threads > 0 else len(os.sched_getaffinity(0))  # every core this process may use
    s = oracle.system(K_LAT, 0, A, KAPPA, RC)
    nw = max(1, threads)
    seeds = list(range(1, nw + 1))
    R0 = np.stack([oracle.initial_positions(s, w, JITTER) for w in seeds])
    t0 = time.perf_counter()
    _, rl, al = oracle.chains(s, seeds, SIGMA, R0, sweeps, solver=oracle.SOLVER_SHERMAN_MORRISON, refresh=0,
                              threads=threads)
    dt = time.perf_counter() - t0
    ratios = nw * sweeps * N
    rec = {"value": ratios / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{nw} walkers x {sweeps * N} moves ({sweeps} sweep(s)) of the same n=1000 workload (FP64 "
                     f"explicit inverse + Sherman-Morrison chain incl. the initial inverse), OpenMP over walkers, "
                     f"{dt:.1f} s"}
    return rec, ratios, dt


def reference_arm(args):
    """One step = one bounded sample of the workload (one sweep of one walker per host core)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_oracle_sample(1)
    total_ratios, total_s, cb = 0, 0.0, None
    for _ in range(args.steps):
        cb, ratios, dt = cpu_oracle_sample(1)
        total_ratios += ratios
        total_s += dt
    v = total_ratios / total_s
    cb["value"] = v
    cb["sample"] = f"per step: {cb['sample'].rsplit(', ', 1)[0]}; {args.steps} steps in {total_s:.1f} s"
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000.0 * total_s / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": N, "walkers_per_gpu": WALKERS,
                      "step": f"one sweep of {cb['cores']} walkers (one per host core) on the CPU"},
           "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-kernels", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    args.warmup = max(3, args.warmup)

    import torch

    from paper_1008_5113_gb300 import vmc
    from paper_1008_5113_gb300.build import build_library

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    if rank == 0 or world == 1:
        build_library()
    if world > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream()
    from paper_1008_5113_gb300 import replicas

    systems = [(K_LAT, 0, A, KAPPA, RC)] * WALKERS
    seeds = replicas.walker_seeds(rank, WALKERS)

    def make(prec, engine, nw=WALKERS):
        ctx = vmc.vmc_create(systems[:nw], vmc.params(precision=prec, engine=engine), stream=stream)
        vmc.vmc_init_positions(ctx, seeds[:nw], JITTER)
        return ctx

    def refactor_mode(ctx):
        lag = vmc.vmc_get_stats(ctx, 0)["async_lag"]
        if lag > 0:
            return (f"background: a factor CTA per walker (cluster of 2) refactors a snapshot, adopted "
                    f"{lag} accepts later")
        return "in line, when the update chain is full"

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    seeds_dev = torch.tensor(seeds, dtype=torch.int64, device="cuda")

    def timed_sweeps(ctx, steps, warmup, keep_state=None):
        for _ in range(warmup):
            vmc.vmc_sweep_async(ctx, 1, SIGMA, seeds_dev)
        vmc.vmc_synchronize(ctx)
        if keep_state is not None:  # walker 0 where the timed sweeps start (for the plain path)
            keep_state["R0"] = vmc.vmc_get_positions(ctx, 0)
            keep_state["sweep"] = vmc.vmc_sweep_count(ctx)
        vmc.vmc_reset_stats(ctx)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            flush.fill_(float(k))                      # L2 flush between timed steps (not timed)
            ev[k][0].record(stream)
            vmc.vmc_sweep_async(ctx, 1, SIGMA, seeds_dev)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        vmc.vmc_synchronize(ctx)
        ms = [a.elapsed_time(b) for a, b in ev]
        return sum(ms), ms, wall

    # ---- headline: batched FP64, persistent engine (one launch per sweep) ------------
    ctx = make(vmc.PREC_FP64, vmc.ENGINE_PERSISTENT)
    refactoring = refactor_mode(ctx)
    state = {}
    kernel_name = "k_sweep_pair" if vmc.vmc_get_stats(ctx, 0)["async_lag"] > 0 else "k_sweep"
    with Clocks(dev) as clk:
        total_ms, per_ms, wall = timed_sweeps(ctx, args.steps, args.warmup, keep_state=state)
    stats = [vmc.vmc_get_stats(ctx, w) for w in range(WALKERS)]
    ratios_local = sum(s["proposals"] for s in stats)
    assert ratios_local == args.steps * WALKERS * N, (ratios_local, args.steps)
    ratios_all, t_max = replicas.reduce_run(ratios_local, total_ms)
    value = replicas.throughput(ratios_all, t_max / 1000.0)
    alg_bytes = sum(s["alg_bytes"] for s in stats)
    vmc.vmc_destroy(ctx)
    # ---- e2e: public host API, host seeds in, host logs out, every step; a fresh context
    #      brought to the same state, so the timed sweeps are the same sweeps as above -----
    ctx = make(vmc.PREC_FP64, vmc.ENGINE_PERSISTENT)
    for _ in range(args.warmup):
        vmc.vmc_sweep_async(ctx, 1, SIGMA, seeds_dev)
    vmc.vmc_synchronize(ctx)
    # the step's inputs and results live in pinned host memory (pageable if pinning fails)
    host_seeds = torch.tensor(seeds, dtype=torch.int64)        # the seeds' uint64 bytes (all positive)
    acc_log = torch.zeros(WALKERS * N, dtype=torch.uint8)
    rat_log = torch.zeros(WALKERS * N, dtype=torch.float64)
    try:
        host_seeds, acc_log, rat_log = host_seeds.pin_memory(), acc_log.pin_memory(), rat_log.pin_memory()
        host_memory = "pinned"
    except RuntimeError:
        host_memory = "pageable"
    lib = vmc.lib()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = lib.vmc_sweep(ctx, 1, SIGMA, vmc._p(host_seeds), vmc._p(acc_log), vmc._p(rat_log))
        assert st == 0, vmc.vmc_last_error(ctx)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_count, e2e_s = replicas.reduce_run(args.steps * WALKERS * N, e2e_s)
    e2e_value = replicas.throughput(e2e_count, e2e_s)
    vmc.vmc_destroy(ctx)

    extra = {}
    if rank == 0:
        # ---- mixed precision, same workload ----------------------------------------------
        ctxm = make(vmc.PREC_MIXED, vmc.ENGINE_PERSISTENT)
        tm, _, _ = timed_sweeps(ctxm, args.steps, args.warmup)
        sm = [vmc.vmc_get_stats(ctxm, w) for w in range(WALKERS)]
        extra["mixed_value"] = sum(s["proposals"] for s in sm) / (tm / 1000.0)
        vmc.vmc_destroy(ctxm)
        # ---- the dense reference point: explicit inverse + Sherman-Morrison (Sec. 1), FP64,
        #      same walkers and sweeps, a fresh inverse every sweep -------------------------
        ctxd = make(vmc.PREC_FP64, vmc.ENGINE_DENSE_SM)
        td, _, _ = timed_sweeps(ctxd, args.steps, args.warmup)
        sd_ = [vmc.vmc_get_stats(ctxd, w) for w in range(WALKERS)]
        extra["dense_sm_fp64_value"] = sum(x["proposals"] for x in sd_) / (td / 1000.0)
        vmc.vmc_destroy(ctxd)
        # ---- plain FP64 one-walker-per-launch path (bounded sample: 1 walker, 1 sweep) ---
        # started from walker 0's configuration at the first timed sweep, with that sweep's
        # random numbers, so that both paths solve equally conditioned matrices
        if not args.no_plain:
            ctxp = make(vmc.PREC_FP64, vmc.ENGINE_PLAIN, nw=1)
            vmc.vmc_set_positions(ctxp, 0, state["R0"])
            vmc.vmc_set_sweep_count(ctxp, state["sweep"])
            sd1 = seeds_dev[:1]
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vmc.vmc_sweep_async(ctxp, 1, SIGMA, sd1)
            e1.record(stream)
            torch.cuda.synchronize()
            vmc.vmc_synchronize(ctxp)
            plain = N / (e0.elapsed_time(e1) / 1000.0)
            vmc.vmc_destroy(ctxp)
            extra["plain_fp64_value"] = plain
            extra["plain_fp64_sample"] = (f"walker 0 from its configuration at sweep {state['sweep']}, "
                                          f"one sweep ({N} launches)")
            extra["speedup_vs_plain"] = value / plain
            extra["speedup_vs_plain_mixed"] = extra["mixed_value"] / plain
    if rank == 0 and not args.no_kernels:
        # ---- per-kernel rooflines at the HBM-sized configurations (CTA per walker; n = 4096
        #      with 256 walkers, n = 32768 with 152 = one per SM): triangular solves and SpMV,
        #      FP32 (mixed mode) ------------------------------------------------------------
        hbm_peak, _ = peaks()
        kr = {}
        # (K, walkers, kappa, r_c): n = 4096 with its configuration's 256 walkers; n = 32768 with
        # 152 walkers, for the kappa = 2 / r_c = 1.5 matrices and for the large configuration's own
        # kappa = 1 / r_c = 2 (about 33 entries a row)
        for K, nwk, kap, rc in ((16, 256, KAPPA, RC), (32, 152, KAPPA, RC), (32, 152, 1.0, 2.0)):
            ctxk = vmc.vmc_create([(K, 0, A, kap, rc)] * nwk, vmc.params(precision=vmc.PREC_MIXED), stream=stream)
            vmc.vmc_init_positions(ctxk, list(range(1, nwk + 1)), JITTER)
            reps = 40 if K == 16 else (10 if kap == KAPPA else 4)
            for which, name in ((0, "trisolve"), (1, "spmv")):
                vmc.vmc_kernel_bench(ctxk, which, 2)
                vmc.vmc_synchronize(ctxk)
                vmc.vmc_reset_stats(ctxk)
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                vmc.vmc_kernel_bench(ctxk, which, reps)
                e1.record(stream)
                torch.cuda.synchronize()
                vmc.vmc_synchronize(ctxk)
                ms = e0.elapsed_time(e1)
                by = sum(vmc.vmc_get_stats(ctxk, w)["alg_bytes"] for w in range(nwk))
                gbs = by / (ms / 1000.0) / 1e9
                tag = "" if kap == KAPPA else f"_k{kap:g}_rc{rc:g}"
                kr[f"{name}_sc{K}_n{K ** 3}{tag}_w{nwk}_f32"] = {
                    "us_per_apply": 1000.0 * ms / reps, "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": gbs / hbm_peak, "bytes_per_apply": by / reps}
            vmc.vmc_destroy(ctxk)
        extra["kernel_rooflines"] = kr
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    hbm, peak_kind = peaks()
    kernel_ms = total_ms / args.steps        # one sweep launch per step
    achieved = alg_bytes / args.steps / (kernel_ms / 1000.0) / 1e9
    its = sum(s["inner_iterations"] for s in stats) / ratios_local
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "walkers_per_gpu": WALKERS, "sweeps_per_step": 1,
                   "engine": "persistent (one launch per sweep, CTA per walker)", "gmres_m": 30,
                   "ilutp": "drop 1e-4, permtol 0.5", "inner_rtol": 1e-10, "refactorisation": refactoring,
                   "l2": "256 MB buffer written between timed steps"},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": host_seeds.numel() * host_seeds.element_size(),
                "d2h_bytes_per_step": acc_log.numel() * acc_log.element_size()
                + rat_log.numel() * rat_log.element_size(),
                "host_memory": host_memory, "api": "vmc_sweep (host seeds in, accept and ratio logs out)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": profiled_traffic(f"{kernel_name}_sc10_n1000_w64_fp64.md"),
                     "note": f"{kernel_name}, algorithmic bytes from the kernel's per-phase counter; peak "
                             f"{peak_kind}"},
        "solver": {"inner_its_per_ratio": its,
                   "accept_rate": sum(s["accepts"] for s in stats) / ratios_local,
                   "reorders": sum(s["reorders"] for s in stats),
                   "refactorizations": sum(s["factorizations"] for s in stats)},
    }
    out.update(extra)
    if not args.no_cpu_baseline and world == 1:  # timed on the host cores at N = 1 only
        try:
            out["cpu_baseline"] = cpu_oracle_sample(6)[0]  # about 10 s on the host cores
            out["cpu_baseline_1core"] = cpu_oracle_sample(2, threads=1)[0]
        except Exception as e:  # the oracle is test infrastructure; report, do not fail
            out["cpu_baseline"] = {"value": None, "error": str(e)}
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
