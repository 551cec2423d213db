"""ctypes binding of the C ABI in ``include/vmc.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
computation of its own: the work runs in ``libvmc.so``.  The library must have been
built (``paper_1008_5113_gb300.build.build_library()`` or ``__graft_entry__.build()``);
loading fails loudly otherwise -- there is no fallback path.

Device buffers and streams may be passed as PyTorch CUDA tensors and
``torch.cuda.Stream`` objects (their raw pointers/handles are forwarded).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB

_lock = threading.Lock()
_lib = None

STATUS = {0: "VMC_OK", 1: "VMC_ERR_INVALID", 2: "VMC_ERR_CUDA", 3: "VMC_ERR_OOM", 4: "VMC_ERR_NOCONV",
          5: "VMC_ERR_BREAKDOWN", 6: "VMC_ERR_TIMEOUT", 7: "VMC_ERR_STATE", 8: "VMC_ERR_CAPACITY"}
PREC_FP64, PREC_MIXED, PREC_MIXED_F32ILU = 0, 1, 2
ENGINE_PLAIN, ENGINE_STEP, ENGINE_PERSISTENT, ENGINE_DENSE_SM = 0, 1, 2, 3


class VmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class vmc_system(C.Structure):
    _fields_ = [("K", C.c_int), ("lattice", C.c_int), ("a", C.c_double), ("kappa", C.c_double),
                ("r_c", C.c_double)]


class vmc_solver_params(C.Structure):
    _fields_ = [("drop_tol", C.c_double), ("permtol", C.c_double), ("lfil_extra", C.c_int),
                ("gmres_m", C.c_int), ("max_restarts", C.c_int), ("inner_rtol", C.c_double),
                ("ratio_tol", C.c_double), ("N_max", C.c_double), ("slow_factor", C.c_double),
                ("max_updates", C.c_int), ("precision", C.c_int), ("engine", C.c_int),
                ("block_threads", C.c_int), ("sm_refresh", C.c_int), ("refactor_lag", C.c_int),
                ("refactor_reorder", C.c_int), ("trisolve", C.c_int),
                ("graphs", C.c_int), ("trigger_rtol", C.c_double), ("trigger_its", C.c_int), ("sweep_moves", C.c_int),
                ("ilutp_variant", C.c_int), ("trisolve_warp_rows", C.c_int),
                ("trisolve_group", C.c_int), ("trisolve_row_cap", C.c_int),
                ("trisolve_lane_entries", C.c_int)]


class vmc_stats(C.Structure):
    _fields_ = [("proposals", C.c_int64), ("accepts", C.c_int64), ("solves", C.c_int64),
                ("inner_iterations", C.c_int64), ("first_pass_iterations", C.c_int64),
                ("outer_passes", C.c_int64), ("reorders", C.c_int64), ("reorder_monitor", C.c_int64),
                ("reorder_noconv", C.c_int64), ("reorder_slow", C.c_int64), ("reorder_breakdown", C.c_int64),
                ("refactors_updates", C.c_int64), ("factorizations", C.c_int64), ("pivots", C.c_int64),
                ("N_max_seen", C.c_double), ("N_sum", C.c_double), ("nnz_A", C.c_double), ("nnz_LU", C.c_double),
                ("levels_L", C.c_int), ("levels_U", C.c_int), ("n_updates", C.c_int), ("status", C.c_int),
                ("its_hist", C.c_int64 * 64), ("phase_cycles", C.c_int64 * 16), ("alg_bytes", C.c_double),
                ("ilu_rows", C.c_int64), ("ilu_elims", C.c_int64), ("ilu_cand", C.c_int64),
                ("chunks_L", C.c_int), ("chunks_U", C.c_int), ("refactors_async", C.c_int64),
                ("async_wait_cycles", C.c_int64), ("async_factor_cycles", C.c_int64), ("factor_set", C.c_int),
                ("async_lag", C.c_int), ("max_updates", C.c_int), ("groups_L", C.c_int), ("groups_U", C.c_int),
                ("trigger_iterations", C.c_int64),
                ("reorders_skipped", C.c_int64), ("stream_bytes", C.c_int64)]


class vmc_tune_trial(C.Structure):
    _fields_ = [("engine", C.c_int), ("block_threads", C.c_int), ("max_updates", C.c_int),
                ("refactor_lag", C.c_int), ("ratios_per_s", C.c_double), ("status", C.c_int),
                ("lfil_extra", C.c_int), ("trisolve_group", C.c_int)]


# name -> (restype, argtypes); every symbol the header declares
_SIG = {
    "vmc_default_params": (C.c_int, [C.c_void_p]),
    "vmc_create": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vmc_destroy": (C.c_int, [C.c_void_p]),
    "vmc_init_positions": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double]),
    "vmc_set_positions": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "vmc_set_positions_all": (C.c_int, [C.c_void_p, C.c_void_p]),
    "vmc_get_positions": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "vmc_walker_n": (C.c_int, [C.c_void_p, C.c_int]),
    "vmc_ratio": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "vmc_accept": (C.c_int, [C.c_void_p, C.c_int]),
    "vmc_ratio_grad": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vmc_sweep": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vmc_sweep_async": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vmc_synchronize": (C.c_int, [C.c_void_p]),
    "vmc_advance_async": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p]),
    "vmc_advance": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p]),
    "vmc_get_progress": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "vmc_kinetic_energy": (C.c_int, [C.c_void_p, C.c_void_p]),
    "vmc_get_stats": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "vmc_reset_stats": (C.c_int, [C.c_void_p]),
    "vmc_last_error": (C.c_char_p, [C.c_void_p]),
    "vmc_sweep_count": (C.c_int64, [C.c_void_p]),
    "vmc_set_sweep_count": (C.c_int, [C.c_void_p, C.c_int64]),
    "vmc_get_matrix": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vmc_get_factors": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vmc_apply_preconditioner": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "vmc_refactor": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "vmc_philox_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "vmc_kernel_bench": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "vmc_check_wait_timeout": (C.c_int, [C.c_void_p]),
    "vmc_ratio_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "vmc_noalloc_capacity": (C.c_size_t, []),
    "vmc_noalloc_last_error": (C.c_char_p, []),
    "vmc_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_int,
                               C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "vmc_autotune_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_int64,
                                     C.c_double, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
}


def lib():
    """Load libvmc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"{LIB} is not built; run __graft_entry__.build() (no CPU fallback exists)")
            L = C.CDLL(LIB)
            for name, (res, args) in _SIG.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _check(st: int, ctx=None):
    if st != 0:
        msg = lib().vmc_last_error(ctx).decode(errors="replace") if ctx is not None else ""
        raise VmcError(st, msg)


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def vmc_default_params() -> vmc_solver_params:
    p = vmc_solver_params()
    _check(lib().vmc_default_params(C.byref(p)))
    return p


def vmc_create(systems, params: vmc_solver_params | None = None, stream=None):
    """systems: list of (K, lattice, a, kappa, r_c), one per walker. Returns the context."""
    arr = (vmc_system * len(systems))(*[vmc_system(int(K), int(lat), float(a), float(k), float(rc))
                                        for (K, lat, a, k, rc) in systems])
    ctx = C.c_void_p()
    st = lib().vmc_create(arr, len(systems), C.byref(params) if params is not None else None,
                          _stream_handle(stream), C.byref(ctx))
    if st != 0:
        msg = lib().vmc_last_error(ctx).decode(errors="replace") if ctx.value else ""
        if ctx.value:
            lib().vmc_destroy(ctx)
        raise VmcError(st, msg)
    return ctx


def vmc_destroy(ctx) -> None:
    _check(lib().vmc_destroy(ctx))


def vmc_init_positions(ctx, seeds, jitter: float) -> None:
    s = np.ascontiguousarray(seeds, dtype=np.uint64)
    _check(lib().vmc_init_positions(ctx, _p(s), float(jitter)), ctx)


def vmc_walker_n(ctx, walker: int) -> int:
    return lib().vmc_walker_n(ctx, walker)


def vmc_set_positions(ctx, walker: int, xyz) -> None:
    x = np.ascontiguousarray(xyz, dtype=np.float64)
    _check(lib().vmc_set_positions(ctx, walker, _p(x)), ctx)


def vmc_set_positions_all(ctx, xyz) -> None:
    """xyz: every walker's positions, walker-major (a list of (n_w, 3) arrays or one flat array)."""
    if isinstance(xyz, (list, tuple)):
        xyz = np.concatenate([np.asarray(x, dtype=np.float64).reshape(-1) for x in xyz])
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    _check(lib().vmc_set_positions_all(ctx, _p(x)), ctx)


def vmc_get_positions(ctx, walker: int) -> np.ndarray:
    n = vmc_walker_n(ctx, walker)
    x = np.zeros((n, 3))
    _check(lib().vmc_get_positions(ctx, walker, _p(x)), ctx)
    return x


def vmc_ratio(ctx, walker: int, k: int, r_new) -> float:
    r = np.ascontiguousarray(r_new, dtype=np.float64)
    out = C.c_double(0.0)
    _check(lib().vmc_ratio(ctx, walker, k, _p(r), C.byref(out)), ctx)
    return out.value


def vmc_ratio_grad(ctx, walker: int, k: int, r_new):
    """(ratio, grad ln|det A'|, lap det A' / det A') at the proposed position."""
    r = np.ascontiguousarray(r_new, dtype=np.float64)
    out = C.c_double(0.0)
    g = np.zeros(3)
    lap = C.c_double(0.0)
    _check(lib().vmc_ratio_grad(ctx, walker, k, _p(r), C.byref(out), _p(g), C.byref(lap)), ctx)
    return out.value, g, lap.value


def vmc_accept(ctx, walker: int) -> None:
    _check(lib().vmc_accept(ctx, walker), ctx)


def vmc_sweep(ctx, n_sweeps: int, sigma: float, seeds, logs: bool = True):
    """Host-log sweeps; returns (accept_log bool[], ratio_log float64[]) or (None, None)."""
    s = np.ascontiguousarray(seeds, dtype=np.uint64)
    total = sum(vmc_walker_n(ctx, w) for w in range(len(s))) * n_sweeps
    acc = np.zeros(total, dtype=np.uint8) if logs else None
    rat = np.zeros(total) if logs else None
    _check(lib().vmc_sweep(ctx, n_sweeps, float(sigma), _p(s), _p(acc), _p(rat)), ctx)
    return (acc.astype(bool), rat) if logs else (None, None)


def vmc_sweep_async(ctx, n_sweeps: int, sigma: float, seeds_dev, accept_log_dev=None, ratio_log_dev=None) -> None:
    _check(lib().vmc_sweep_async(ctx, n_sweeps, float(sigma), _p(seeds_dev), _p(accept_log_dev),
                                 _p(ratio_log_dev)), ctx)


def vmc_advance_async(ctx, total_moves: int, sigma: float, seeds_dev) -> None:
    _check(lib().vmc_advance_async(ctx, int(total_moves), float(sigma), _p(seeds_dev)), ctx)


def vmc_advance(ctx, total_moves: int, sigma: float, seeds) -> np.ndarray:
    """Budgeted advance with host seeds; returns every walker's accepted-move count."""
    s = np.ascontiguousarray(seeds, dtype=np.uint64)
    acc = np.zeros(len(s), dtype=np.int64)
    _check(lib().vmc_advance(ctx, int(total_moves), float(sigma), _p(s), _p(acc)), ctx)
    return acc


def vmc_get_progress(ctx, walker: int):
    """(sweep, particle) of walker's next move."""
    sw = C.c_int64(0)
    k = C.c_int(0)
    _check(lib().vmc_get_progress(ctx, walker, C.byref(sw), C.byref(k)), ctx)
    return sw.value, k.value


def vmc_synchronize(ctx) -> None:
    _check(lib().vmc_synchronize(ctx), ctx)


def vmc_kinetic_energy(ctx, n_walkers: int) -> np.ndarray:
    e = np.zeros(n_walkers)
    _check(lib().vmc_kinetic_energy(ctx, _p(e)), ctx)
    return e


def vmc_get_stats(ctx, walker: int) -> dict:
    st = vmc_stats()
    _check(lib().vmc_get_stats(ctx, walker, C.byref(st)), ctx)
    d = {name: getattr(st, name) for name, _ in vmc_stats._fields_ if name not in ("its_hist", "phase_cycles")}
    d["its_hist"] = list(st.its_hist)
    d["phase_cycles"] = list(st.phase_cycles)
    return d


def vmc_reset_stats(ctx) -> None:
    _check(lib().vmc_reset_stats(ctx), ctx)


def vmc_last_error(ctx) -> str:
    return lib().vmc_last_error(ctx).decode(errors="replace")


def vmc_sweep_count(ctx) -> int:
    return lib().vmc_sweep_count(ctx)


def vmc_set_sweep_count(ctx, sweeps: int) -> None:
    _check(lib().vmc_set_sweep_count(ctx, sweeps), ctx)


def vmc_get_matrix(ctx, walker: int):
    n = vmc_walker_n(ctx, walker)
    A = np.zeros((n, n))
    por = np.zeros(n, dtype=np.int32)
    ooc = np.zeros(n, dtype=np.int32)
    _check(lib().vmc_get_matrix(ctx, walker, _p(A), _p(por), _p(ooc)), ctx)
    return A, por, ooc


def vmc_get_factors(ctx, walker: int):
    n = vmc_walker_n(ctx, walker)
    L = np.zeros((n, n))
    U = np.zeros((n, n))
    perm = np.zeros(n, dtype=np.int32)
    _check(lib().vmc_get_factors(ctx, walker, _p(L), _p(U), _p(perm)), ctx)
    return L, U, perm


def vmc_apply_preconditioner(ctx, walker: int, v) -> np.ndarray:
    vv = np.ascontiguousarray(v, dtype=np.float64)
    z = np.zeros_like(vv)
    _check(lib().vmc_apply_preconditioner(ctx, walker, _p(vv), _p(z)), ctx)
    return z


def vmc_refactor(ctx, walker: int, reorder: bool = True) -> None:
    _check(lib().vmc_refactor(ctx, walker, 1 if reorder else 0), ctx)


def vmc_kernel_bench(ctx, which: int, reps: int) -> None:
    _check(lib().vmc_kernel_bench(ctx, which, reps), ctx)


def vmc_check_wait_timeout(ctx) -> int:
    """Status of the bounded-wait check (VMC_ERR_TIMEOUT = 6 expected)."""
    return lib().vmc_check_wait_timeout(ctx)


def vmc_philox_device(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    _check(lib().vmc_philox_device(_p(c), _p(k), _p(out), c.shape[0]))
    return out


def vmc_ratio_noalloc(system, params, xyz_dev, k: int, r_new, ratio_dev, stream=None) -> None:
    """Ratio of one move without device allocation; xyz_dev and ratio_dev are CUDA
    tensors (float64, contiguous, n*3 and 1 element, on the current device) owned by
    the caller.  stream: defaults to the current torch stream of xyz_dev's device, so
    that the call is ordered after the work that produced the positions."""
    import torch

    K, lat, a, kap, rc = system
    n = int(K) ** 3 * (2 if int(lat) == 1 else 1)
    cur = torch.cuda.current_device()
    for name, t, need in (("xyz_dev", xyz_dev, 3 * n), ("ratio_dev", ratio_dev, 1)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise VmcError(1, f"{name} must be a contiguous float64 CUDA tensor")
        if t.device.index != cur:
            raise VmcError(1, f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")
        if t.numel() < need:
            raise VmcError(1, f"{name} holds {t.numel()} doubles, {need} needed")
    if stream is None:
        stream = torch.cuda.current_stream(xyz_dev.device)
    sysc = vmc_system(int(K), int(lat), float(a), float(kap), float(rc))
    r = np.ascontiguousarray(r_new, dtype=np.float64)
    st = lib().vmc_ratio_noalloc(C.byref(sysc), C.byref(params) if params is not None else None, _p(xyz_dev), k,
                                 _p(r), _p(ratio_dev), _stream_handle(stream))
    if st != 0:
        raise VmcError(st, lib().vmc_noalloc_last_error().decode(errors="replace"))


def vmc_noalloc_capacity() -> int:
    return lib().vmc_noalloc_capacity()


def vmc_noalloc_last_error() -> str:
    return lib().vmc_noalloc_last_error().decode(errors="replace")


def params(**kw) -> vmc_solver_params:
    """vmc_default_params() with fields overridden by keyword."""
    p = vmc_default_params()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def vmc_autotune(systems, params: vmc_solver_params, seeds, jitter: float, sigma: float, steps: int, stream=None,
                 xyz=None, sweep0: int = 0):
    """Returns (the tuned parameters, the list of trials as dicts).  xyz: optional start state
    (every walker's positions, walker-major) with its sweep index sweep0."""
    arr = (vmc_system * len(systems))(*[vmc_system(int(K), int(lat), float(a), float(k), float(rc))
                                        for (K, lat, a, k, rc) in systems])
    p = vmc_solver_params.from_buffer_copy(params)
    s = np.ascontiguousarray(seeds, dtype=np.uint64)
    x = None
    if xyz is not None:
        if isinstance(xyz, (list, tuple)):
            xyz = np.concatenate([np.asarray(v, dtype=np.float64).reshape(-1) for v in xyz])
        x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    trials = (vmc_tune_trial * 16)()
    nt = C.c_int(0)
    _check(lib().vmc_autotune_state(arr, len(systems), C.byref(p), _p(s), float(jitter), _p(x), int(sweep0),
                                    float(sigma), int(steps), trials, 16, C.byref(nt), _stream_handle(stream)))
    return p, [{name: getattr(trials[i], name) for name, _ in vmc_tune_trial._fields_} for i in range(nt.value)]
