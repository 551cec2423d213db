"""Benchmark of the sparse determinant-ratio engine (one JSON line on rank 0).

Workload: n = 1000 electrons/orbitals on a 10x10x10 simple-cubic lattice (a = 1),
Gaussian orbitals exp(-2 |r - Z|^2) cut at r_c = 1.5, 64 independent walkers
(seeds 1..64), electrons started at the sites + N(0, 0.1^2), Metropolis steps
N(0, 0.2^2), FP64 arithmetic ("plain FP64 batched").  Synthetic data, nothing read
from disk.

Stationary timed step.  The first sweeps of a chain are a transient: the electrons
leave their start positions and the Slater matrices grow harder to solve (the paper
discards 20 sweeps, Sec. 4).  So the walkers are first taken through S = 20 sweeps
by the engine's dense Sherman-Morrison path (FP64, untimed; the same Markov chain);
their positions and the sweep counter S are the saved state.  The solver layout (CTA
mapping, chain length, ILUTP fill limit) is then picked by the engine's autotuner with
trials from that state.  Every bench step -- warm-up and timed -- restores the state
(vmc_set_positions_all: rows, reordering and a fresh ILUTP per walker;
vmc_set_sweep_count(S)), outside the timed region, and then times one budgeted advance
of the batch by 64 x 250 moves: the walkers claim moves one at a time and each makes them
along its own chain from particle 0 of sweep S, so that the SMs of walkers with cheaper
solves do not idle while the slowest walker finishes.  Every move goes through the whole
hot path (proposal, Slater row, ILUTP-preconditioned GMRES solve with refinement,
stability monitor/reorder/refactor, Metropolis test, row commit and preconditioner
update, background refactorisations).  Every step is the same amount of work.

Reported beside the headline: the end-to-end rate through the host API, the same
sweep in mixed precision, the dense Sherman-Morrison reference point, the plain FP64
one-walker-per-launch path (the metric's denominator) on walker 0's sweep S, the
roofline of the dominant kernel from its algorithmic-byte counter, per-kernel
rooflines of the triangular solves and the SpMV at the HBM-sized configurations, and
the FP64 CPU oracle timed on the host cores.  Legs after the headline are skipped
once the wall-clock budget (--budget-s) is spent; each leg's wall time goes to stderr.

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
EQUIL_SWEEPS = 20  # sweeps discarded before the timed sweep (Sec. 4 discards 20)
MOVES_PER_STEP = 250  # moves per walker in one bench step (particles 0..249 of sweep S)
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


def log(msg: str) -> None:
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--budget-s", type=float, default=900.0,
                    help="wall-clock budget: legs after the headline are skipped once it is spent")
    ap.add_argument("--walkers", type=int, default=WALKERS, help="walkers per GPU (profiling runs use fewer)")
    ap.add_argument("--moves", type=int, default=MOVES_PER_STEP,
                    help="moves per walker in a step: the first moves of sweep S (0: the full sweep)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-kernels", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the larger configurations' legs")
    ap.add_argument("--headline-only", action="store_true", help="skip every leg after the headline")
    ap.add_argument("--no-autotune", action="store_true", help="fixed solver layout instead of the autotuner's")
    ap.add_argument("--layout", default="pairs", choices=["pairs", "inline"],
                    help="with --no-autotune: a factor CTA per walker (background refactorisation) or in-line")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    args.warmup = max(3, args.warmup)
    t_start = time.perf_counter()

    def over_budget() -> bool:
        return time.perf_counter() - t_start > args.budget_s

    import numpy as np
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

    NW = args.walkers
    moves = args.moves if 0 < args.moves < N else N
    systems = [(K_LAT, 0, A, KAPPA, RC)] * NW
    seeds = replicas.walker_seeds(rank, NW)
    seeds_dev = torch.tensor(seeds, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # ---- the saved state: S sweeps of the dense Sherman-Morrison engine (untimed) --------
    t0 = time.perf_counter()
    ctxd = vmc.vmc_create(systems, vmc.params(precision=vmc.PREC_FP64, engine=vmc.ENGINE_DENSE_SM), stream=stream)
    vmc.vmc_init_positions(ctxd, seeds, JITTER)
    vmc.vmc_sweep_async(ctxd, EQUIL_SWEEPS, SIGMA, seeds_dev)
    vmc.vmc_synchronize(ctxd)
    state = np.concatenate([vmc.vmc_get_positions(ctxd, w).reshape(-1) for w in range(NW)])
    vmc.vmc_destroy(ctxd)
    log(f"equilibration: {EQUIL_SWEEPS} dense sweeps of {NW} walkers in {time.perf_counter() - t0:.1f} s")

    def restore(ctx, nw=NW):
        vmc.vmc_set_positions_all(ctx, state[:nw * N * 3])
        vmc.vmc_set_sweep_count(ctx, EQUIL_SWEEPS)

    # ---- solver layout: the autotuner's pick, from the saved state ---------------------
    def tuned(prec):
        base = vmc.params(precision=prec)
        if args.no_autotune:  # the layouts the autotuner picks for this workload (persistent, 256 threads)
            base.lfil_extra = 32
            if args.layout == "pairs":
                base.max_updates, base.refactor_lag = 32, 16
            else:
                base.max_updates, base.refactor_lag = 128, 0
            return base, []
        t1 = time.perf_counter()
        # trials as long as one timed step: shorter ones miss the in-line refactorisations that
        # a chain of 64-128 updates brings every 100-200 moves, and favour the in-line layouts
        p, trials = vmc.vmc_autotune(systems, base, seeds, JITTER, SIGMA, moves, stream=stream, xyz=state,
                                     sweep0=EQUIL_SWEEPS)
        log(f"autotune (precision {prec}): {len(trials)} trials in {time.perf_counter() - t1:.1f} s; picked engine "
            f"{p.engine}, {p.block_threads} threads, chain {p.max_updates}, lag {p.refactor_lag}, lfil {p.lfil_extra}")
        return p, trials

    def with_(p, **kw):
        q = vmc.vmc_solver_params.from_buffer_copy(p)
        for k, v in kw.items():
            setattr(q, k, v)
        return q

    def summed(acc, st):
        if acc is None:
            return st
        for a, b in zip(acc, st):
            for key, v in b.items():
                if isinstance(v, list):
                    a[key] = [x + y for x, y in zip(a[key], v)]
                elif key not in ("status", "factor_set", "async_lag", "max_updates", "n_updates", "levels_L",
                                 "levels_U", "groups_L", "groups_U", "nnz_A", "nnz_LU", "pivots", "chunks_L",
                                 "chunks_U", "N_max_seen"):
                    a[key] += v
                elif key == "N_max_seen":
                    a[key] = max(a[key], v)
        return acc

    def stationary_steps(ctx, steps, warmup, nw=NW, advance=True):
        """warmup + steps times: restore (untimed), flush L2, then time on the stream one
        step: the budgeted advance of nw x moves moves (or, advance = False, one fixed
        sweep).  Returns per-step ms and the statistics summed over the timed steps."""
        ms, acc = [], None
        for k in range(warmup + steps):
            restore(ctx, nw)
            flush.fill_(float(k))                      # L2 flush between timed steps (not timed)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if world > 1 and k == warmup:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            if advance:
                vmc.vmc_advance_async(ctx, nw * moves, SIGMA, seeds_dev[:nw])
            else:
                vmc.vmc_sweep_async(ctx, 1, SIGMA, seeds_dev[:nw])
            e1.record(stream)
            torch.cuda.synchronize()
            vmc.vmc_synchronize(ctx)
            if k >= warmup:
                ms.append(e0.elapsed_time(e1))
                acc = summed(acc, [vmc.vmc_get_stats(ctx, w) for w in range(nw)])
        return ms, acc

    p64, trials64 = tuned(vmc.PREC_FP64)
    # ---- headline: batched FP64, persistent engine, budgeted advance -------------------
    t0 = time.perf_counter()
    ctx = vmc.vmc_create(systems, p64, stream=stream)
    lag = vmc.vmc_get_stats(ctx, 0)["async_lag"]
    refactoring = (f"background: a factor CTA per walker (cluster of 2) refactors a snapshot, adopted {lag} "
                   f"accepts later" if lag > 0 else "in line, when the update chain is full")
    kernel_name = "k_sweep_pair" if lag > 0 else "k_sweep"
    with Clocks(dev) as clk:
        per_ms, stats = stationary_steps(ctx, args.steps, args.warmup)
    total_ms = sum(per_ms)
    ratios_local = sum(s["proposals"] for s in stats)
    assert ratios_local == args.steps * NW * moves, (ratios_local, args.steps)
    ratios_all, t_max = replicas.reduce_run(ratios_local, total_ms)
    value = replicas.throughput(ratios_all, t_max / 1000.0)
    alg_bytes = sum(s["alg_bytes"] for s in stats)
    log(f"headline: {args.warmup}+{args.steps} steps in {time.perf_counter() - t0:.1f} s; "
        f"{value:.0f} ratios/s; per step ms {[round(x) for x in per_ms]}")
    # ---- e2e: public host API (host seeds in, accept counts out, every step), the same
    #      restored steps on the same context ---------------------------------------------
    t0 = time.perf_counter()
    host_seeds = torch.tensor(seeds, dtype=torch.int64)        # the seeds' uint64 bytes (all positive)
    acc_out = torch.zeros(NW, dtype=torch.int64)
    try:
        host_seeds, acc_out = host_seeds.pin_memory(), acc_out.pin_memory()
        host_memory = "pinned"
    except RuntimeError:
        host_memory = "pageable"
    lib = vmc.lib()
    e2e_s = 0.0
    for k in range(args.steps):
        restore(ctx)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        st_ = lib.vmc_advance(ctx, NW * moves, SIGMA, vmc._p(host_seeds), vmc._p(acc_out))
        e2e_s += time.perf_counter() - t1
        assert st_ == 0, vmc.vmc_last_error(ctx)
    e2e_count, e2e_s = replicas.reduce_run(args.steps * NW * moves, e2e_s)
    e2e_value = replicas.throughput(e2e_count, e2e_s)
    vmc.vmc_destroy(ctx)
    log(f"e2e: {args.steps} steps in {time.perf_counter() - t0:.1f} s; {e2e_value:.0f} ratios/s")

    extra, skipped = {}, []
    side_steps = max(1, min(args.steps, 3))   # fixed-size side legs: at most 3 timed + 1 warm-up
    if rank == 0 and not args.headline_only:
        # ---- mixed precision, same restored steps ----------------------------------------
        if not over_budget():
            t0 = time.perf_counter()
            pm, trials_m = tuned(vmc.PREC_MIXED)
            extra["mixed_params"] = {"engine": pm.engine, "block_threads": pm.block_threads,
                                     "max_updates": pm.max_updates, "refactor_lag": pm.refactor_lag,
                                     "lfil_extra": pm.lfil_extra}
            ctxm = vmc.vmc_create(systems, pm, stream=stream)
            ms_m, sm = stationary_steps(ctxm, side_steps, 1)
            extra["mixed_value"] = sum(s["proposals"] for s in sm) / (sum(ms_m) / 1000.0)
            extra["mixed_inner_its_per_ratio"] = sum(s["inner_iterations"] for s in sm) / sum(s["proposals"] for s in sm)
            vmc.vmc_destroy(ctxm)
            log(f"mixed: {time.perf_counter() - t0:.1f} s; {extra['mixed_value']:.0f} ratios/s")
        else:
            skipped.append("mixed")
        # ---- the dense reference point: explicit inverse + Sherman-Morrison (Sec. 1), FP64,
        #      same restored sweep, a fresh inverse at the restore --------------------------
        if not over_budget():
            t0 = time.perf_counter()
            ctxd = vmc.vmc_create(systems, vmc.params(precision=vmc.PREC_FP64, engine=vmc.ENGINE_DENSE_SM),
                                  stream=stream)
            ms_d, sd_ = stationary_steps(ctxd, side_steps, 1, advance=False)  # one full sweep a step
            extra["dense_sm_fp64_value"] = sum(x["proposals"] for x in sd_) / (sum(ms_d) / 1000.0)
            vmc.vmc_destroy(ctxd)
            log(f"dense: {time.perf_counter() - t0:.1f} s; {extra['dense_sm_fp64_value']:.0f} ratios/s")
        else:
            skipped.append("dense")
        # ---- plain FP64 one-walker-per-launch path: walker 0's sweep S from the same state --
        if not args.no_plain and not over_budget():
            t0 = time.perf_counter()
            ctxp = vmc.vmc_create(systems[:1], with_(p64, engine=vmc.ENGINE_PLAIN, sweep_moves=moves),
                                  stream=stream)
            ms_p, sp_ = stationary_steps(ctxp, 1, 1, nw=1, advance=False)
            plain = sp_[0]["proposals"] / (ms_p[0] / 1000.0)
            vmc.vmc_destroy(ctxp)
            extra["plain_fp64_value"] = plain
            extra["plain_fp64_sample"] = (f"walker 0, moves 0..{moves - 1} of sweep {EQUIL_SWEEPS} from the saved "
                                          f"state, one launch per move (graph-replayed), the headline's FP64 "
                                          f"solver parameters")
            extra["speedup_vs_plain"] = value / plain
            if "mixed_value" in extra:
                extra["speedup_vs_plain_mixed"] = extra["mixed_value"] / plain
            log(f"plain: {time.perf_counter() - t0:.1f} s; {plain:.0f} ratios/s")
        elif not args.no_plain:
            skipped.append("plain")
    if rank == 0 and not args.no_configs and not args.headline_only:
        # ---- the larger configurations, mixed precision, budgeted advance: each warmed up
        #      from its start state by a budgeted advance (a few sweeps' worth of moves: 20
        #      sweeps of these batches do not fit a benchmark run), then one timed step,
        #      against the one-walker-per-launch FP64 path at the same size from the same
        #      state (walker 0) -------------------------------------------------------------
        from paper_1008_5113_gb300 import workloads as WLS

        cfg_out = {}
        # fill limit 32 (the autotuner's pick at n = 1000) except for the large matrices of
        # kappa 1, r_c 2, whose rows then outgrow the factorisation's working row: the default
        for wl, warm_moves, step_moves, plain_moves, lfil in ((WLS.MIXED_4096, 2 * 4096, 64, 32, 32),
                                                              (WLS.UNEVEN_320, 1000, 64, 32, 32),
                                                              (WLS.LARGE_32768, 0, 16, 8, -1)):
            if over_budget():
                skipped.append(wl.name)
                continue
            t0 = time.perf_counter()
            csys = wl.systems()
            cnw = len(csys)
            cseeds = wl.seeds()
            csd = torch.tensor(cseeds, dtype=torch.int64, device="cuda")
            pm = vmc.params(precision=vmc.PREC_MIXED, lfil_extra=lfil, trisolve_group=1)
            c = vmc.vmc_create(csys, pm, stream=stream)
            vmc.vmc_init_positions(c, cseeds, wl.jitter)
            if warm_moves:
                vmc.vmc_advance_async(c, cnw * warm_moves, wl.sigma, csd)
                vmc.vmc_synchronize(c)
            prog = [vmc.vmc_get_progress(c, w) for w in range(cnw)]
            xyz = np.concatenate([vmc.vmc_get_positions(c, w).reshape(-1) for w in range(cnw)])
            vmc.vmc_reset_stats(c)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vmc.vmc_advance_async(c, cnw * step_moves, wl.sigma, csd)
            e1.record(stream)
            torch.cuda.synchronize()
            vmc.vmc_synchronize(c)
            ms = e0.elapsed_time(e1)
            cst = [vmc.vmc_get_stats(c, w) for w in range(cnw)]
            vmc.vmc_destroy(c)
            P_ = sum(x["proposals"] for x in cst)
            rec = {"walkers": cnw, "n": sorted({K ** 3 for K in wl.Ks}), "rate": P_ / (ms / 1000.0), "lfil": lfil,
                   "moves_timed": P_, "its_per_ratio": sum(x["inner_iterations"] for x in cst) / P_,
                   "accept_rate": sum(x["accepts"] for x in cst) / P_,
                   "start": f"sweep 0 + a budgeted advance of {warm_moves} moves a walker (walker 0 at sweep "
                            f"{prog[0][0]}, particle {prog[0][1]}); not equilibrated",
                   "its_hist": [sum(x["its_hist"][b] for x in cst) for b in range(40)]}
            # plain FP64 one-walker-per-launch path: walker 0 from the same state
            n0 = wl.Ks[0] ** 3
            pp = vmc.params(precision=vmc.PREC_FP64, engine=vmc.ENGINE_PLAIN, lfil_extra=lfil, sweep_moves=plain_moves)
            cp = vmc.vmc_create(csys[:1], pp, stream=stream)
            vmc.vmc_set_positions_all(cp, xyz[:3 * n0])
            vmc.vmc_set_sweep_count(cp, prog[0][0])
            torch.cuda.synchronize()
            e0.record(stream)
            vmc.vmc_sweep_async(cp, 1, wl.sigma, csd[:1])
            e1.record(stream)
            torch.cuda.synchronize()
            vmc.vmc_synchronize(cp)
            pms = e0.elapsed_time(e1)
            psts = vmc.vmc_get_stats(cp, 0)
            vmc.vmc_destroy(cp)
            rec["plain_fp64_rate"] = psts["proposals"] / (pms / 1000.0)
            rec["plain_fp64_sample"] = f"walker 0 (n = {n0}), {psts['proposals']} moves from particle 0 of its sweep"
            rec["speedup_vs_plain"] = rec["rate"] / rec["plain_fp64_rate"]
            cfg_out[wl.name] = rec
            log(f"config {wl.name}: {time.perf_counter() - t0:.1f} s; {rec['rate']:.0f} ratios/s, plain "
                f"{rec['plain_fp64_rate']:.0f}")
        extra["configs"] = cfg_out
    if rank == 0 and not args.no_kernels and not args.headline_only:
        # ---- per-kernel rooflines at the HBM-sized configurations (CTA per walker; n = 4096
        #      with 256 walkers, n = 32768 with 152 = one per SM): triangular solves and SpMV,
        #      FP32 (mixed mode); fixed repetition counts ----------------------------------
        hbm_peak, _ = peaks()
        kr = {}
        for K, nwk, kap, rc in ((16, 256, KAPPA, RC), (32, 152, KAPPA, RC), (32, 152, 1.0, 2.0)):
            if over_budget():
                skipped.append(f"kernels_sc{K}_k{kap:g}")
                continue
            t0 = time.perf_counter()
            # level-by-level solves: with two walker CTAs an SM (n = 4096) the solves are bound by
            # work, where grouping loses; at n = 32768 two solve vectors do not fit shared memory
            ctxk = vmc.vmc_create([(K, 0, A, kap, rc)] * nwk, vmc.params(precision=vmc.PREC_MIXED, trisolve_group=1),
                                  stream=stream)
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
            log(f"kernel rooflines sc{K} kappa {kap:g}: {time.perf_counter() - t0:.1f} s")
        extra["kernel_rooflines"] = kr
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    hbm, peak_kind = peaks()
    kernel_ms = total_ms / args.steps        # one sweep launch per step
    achieved = alg_bytes / args.steps / (kernel_ms / 1000.0) / 1e9
    nprop = ratios_local
    hist = [sum(s["its_hist"][b] for s in stats) for b in range(64)]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "walkers_per_gpu": NW, "moves_per_step": NW * moves,
                   "step": f"{NW * moves} moves of the batch ({moves} a walker on average), claimed by the walkers "
                           f"one at a time (budgeted advance) from sweep {EQUIL_SWEEPS} of the state after "
                           f"{EQUIL_SWEEPS} discarded sweeps, restored before every step (restore untimed)",
                   "engine": f"persistent, {p64.block_threads} threads a walker CTA, chain {p64.max_updates}",
                   "gmres_m": 30, "ilutp": f"drop 1e-4, permtol 0.5, lfil {p64.lfil_extra}",
                   "solver_layout": f"autotuned from the saved state ({moves} moves a walker a trial)" if trials64 else "fixed (no autotune)",
                   "inner_rtol": 1e-10, "trigger_rtol": 1e-6,
                   "refactorisation": refactoring, "l2": "256 MB buffer written between timed steps",
                   "side_legs": f"mixed: {side_steps} timed + 1 warm-up restored steps (its own autotuned "
                                f"layout); dense: full restored sweeps; plain: one step of walker 0"},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": host_seeds.numel() * host_seeds.element_size(),
                "d2h_bytes_per_step": acc_out.numel() * acc_out.element_size(),
                "host_memory": host_memory,
                "api": "vmc_advance (host seeds in, per-walker accept counts out); the restore is outside the timing"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": profiled_traffic(f"{kernel_name}_sc10_n1000_fp64.md"),
                     "note": f"{kernel_name}, algorithmic bytes from the kernel's per-phase counter; peak "
                             f"{peak_kind}"},
        "solver": {"inner_its_per_ratio": sum(s["inner_iterations"] for s in stats) / nprop,
                   "first_pass_its_per_ratio": sum(s["first_pass_iterations"] for s in stats) / nprop,
                   "its_to_1e-6_per_ratio": sum(s["trigger_iterations"] for s in stats) / nprop,
                   "outer_passes_per_ratio": sum(s["outer_passes"] for s in stats) / nprop,
                   "accept_rate": sum(s["accepts"] for s in stats) / nprop,
                   "reorders_per_1000_moves": 1000.0 * sum(s["reorders"] for s in stats) / nprop,
                   "reorders_skipped_per_1000_moves": 1000.0 * sum(s["reorders_skipped"] for s in stats) / nprop,
                   "factorizations_per_1000_moves": 1000.0 * sum(s["factorizations"] for s in stats) / nprop,
                   "first_pass_its_hist": hist[:max(i for i, h in enumerate(hist) if h) + 1] if any(hist) else []},
        "wall_s": time.perf_counter() - t_start,
    }
    if skipped:
        out["skipped_over_budget"] = skipped
    out["autotune_fp64"] = [{k: t[k] for k in ("engine", "block_threads", "max_updates", "refactor_lag",
                                                  "lfil_extra", "trisolve_group", "ratios_per_s")} for t in trials64]
    out.update(extra)
    if not args.no_cpu_baseline and world == 1 and not args.headline_only:  # host cores, N = 1 only
        try:
            out["cpu_baseline"] = cpu_oracle_sample(6)[0]  # about 10 s on the host cores
            out["cpu_baseline_1core"] = cpu_oracle_sample(2, threads=1)[0]
        except Exception as e:  # the oracle is test infrastructure; report, do not fail
            out["cpu_baseline"] = {"value": None, "error": str(e)}
    out["wall_s"] = time.perf_counter() - t_start
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
