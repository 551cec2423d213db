"""Plain FP64 CPU oracle for the sparse-VMC determinant ratio (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product path (the CUDA library and its binding) never
does, and the oracle never imports the product package.

The C source (``oracle.c``) is the oracle proper; this module compiles it with gcc
(``-O2 -ffp-contract=off -fopenmp``) into ``liboracle.so`` next to it and wraps it
with ctypes.  Every function cites the passage of Ahuja, Clark, de Sturler,
Ceperley, Kim, "Improved Scaling for Quantum Monte Carlo on Insulators" it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class System(C.Structure):
    """Lattice and orbital parameters (Sec. 2.1 Eq. 3; Sec. 4)."""

    _fields_ = [("K", C.c_int), ("lattice", C.c_int), ("a", C.c_double),
                ("kappa", C.c_double), ("r_c", C.c_double)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, plain C, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            d, i, i64, u32, u64, p = C.c_double, C.c_int, C.c_int64, C.c_uint32, C.c_uint64, C.c_void_p
            sp = C.POINTER(System)
            sig = {
                "orc_philox4x32_10": (None, [p, p, p]),
                "orc_uniform53": (d, [u32, u32]),
                "orc_normal3": (None, [u64, u32, u32, u32, p]),
                "orc_accept_uniform": (d, [u64, u32, u32]),
                "orc_n": (i, [sp]),
                "orc_sites": (None, [sp, p]),
                "orc_initial_positions": (None, [sp, u64, d, p]),
                "orc_propose": (None, [sp, u64, u32, u32, d, p, p]),
                "orc_row_dense": (None, [sp, p, p, p]),
                "orc_slater_dense": (None, [sp, p, p, p]),
                "orc_slater_csr": (C.c_long, [sp, p, p, C.c_long, p, p, p]),
                "orc_lu": (i, [i, p, p, p]),
                "orc_lu_solve": (None, [i, p, p, p, p]),
                "orc_leibniz_det": (d, [i, p]),
                "orc_ratio_dense": (i, [i, p, i, p, p, p]),
                "orc_inverse": (i, [i, p, p]),
                "orc_sm_ratio": (d, [i, p, i, p]),
                "orc_sm_update": (None, [i, p, i, p, d, p]),
                "orc_gmres": (i, [i, p, p, p, p, p, i, i, d]),
                "orc_chain": (C.c_long, [sp, u64, d, i, i, C.c_long, i, i, p, p, p, p]),
                "orc_chains": (C.c_long, [sp, i, p, d, i, i, C.c_long, i, i, p, p, p, i]),
                "orc_max_threads": (i, []),
                "orc_kinetic_energy": (d, [sp, p, p]),
                "orc_ratio_grad_lap": (i, [sp, p, p, i, p, p, p, p]),
                "orc_greedy_pairing": (None, [sp, p, p, p, p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def system(K: int, lattice: int = 0, a: float = 1.0, kappa: float = 2.0, r_c: float = 1.5) -> System:
    return System(K, lattice, a, kappa, r_c)


# ---- RNG --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform53(hi: int, lo: int) -> float:
    return lib().orc_uniform53(hi, lo)


def normal3(seed: int, sweep: int, particle: int, purpose: int) -> np.ndarray:
    z = np.zeros(3)
    lib().orc_normal3(seed, sweep, particle, purpose, _ptr(z))
    return z


def accept_uniform(seed: int, sweep: int, particle: int) -> float:
    return lib().orc_accept_uniform(seed, sweep, particle)


# ---- geometry ---------------------------------------------------------------------
def n_of(s: System) -> int:
    return lib().orc_n(C.byref(s))


def sites(s: System) -> np.ndarray:
    Z = np.zeros((n_of(s), 3))
    lib().orc_sites(C.byref(s), _ptr(Z))
    return Z


def initial_positions(s: System, seed: int, jitter: float) -> np.ndarray:
    R = np.zeros((n_of(s), 3))
    lib().orc_initial_positions(C.byref(s), seed, jitter, _ptr(R))
    return R


def propose(s: System, seed: int, sweep: int, particle: int, sigma: float, r_old) -> np.ndarray:
    r0 = np.ascontiguousarray(r_old, dtype=np.float64)
    r1 = np.zeros(3)
    lib().orc_propose(C.byref(s), seed, sweep, particle, sigma, _ptr(r0), _ptr(r1))
    return r1


def row_dense(s: System, Z: np.ndarray, r) -> np.ndarray:
    rr = np.ascontiguousarray(r, dtype=np.float64)
    row = np.zeros(n_of(s))
    lib().orc_row_dense(C.byref(s), _ptr(Z), _ptr(rr), _ptr(row))
    return row


def slater_dense(s: System, Z: np.ndarray, R: np.ndarray) -> np.ndarray:
    n = n_of(s)
    A = np.zeros((n, n))
    lib().orc_slater_dense(C.byref(s), _ptr(Z), _ptr(np.ascontiguousarray(R)), _ptr(A))
    return A


def slater_csr(s: System, Z: np.ndarray, R: np.ndarray, cap: int | None = None):
    n = n_of(s)
    cap = cap or n * 64
    rp = np.zeros(n + 1, dtype=np.int64)
    ci = np.zeros(cap, dtype=np.int32)
    cv = np.zeros(cap)
    nnz = lib().orc_slater_csr(C.byref(s), _ptr(Z), _ptr(np.ascontiguousarray(R)), cap,
                               _ptr(rp), _ptr(ci), _ptr(cv))
    if nnz < 0:
        raise ValueError("CSR capacity too small")
    return rp, ci[:nnz].copy(), cv[:nnz].copy()


# ---- dense linear algebra -----------------------------------------------------------
def leibniz_det(A: np.ndarray) -> float:
    A = np.ascontiguousarray(A, dtype=np.float64)
    if A.shape[0] > 9:
        raise ValueError("Leibniz sum limited to n <= 9")
    return lib().orc_leibniz_det(A.shape[0], _ptr(A))


def lu(A: np.ndarray):
    LU = np.ascontiguousarray(A, dtype=np.float64).copy()
    n = LU.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    sign = C.c_int(0)
    rc = lib().orc_lu(n, _ptr(LU), _ptr(piv), C.byref(sign))
    if rc:
        raise np.linalg.LinAlgError("singular")
    return LU, piv, sign.value


def lu_solve(LU, piv, b) -> np.ndarray:
    bb = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(bb)
    lib().orc_lu_solve(LU.shape[0], _ptr(LU), _ptr(piv), _ptr(bb), _ptr(x))
    return x


def ratio_dense(A: np.ndarray, i: int, a_new) -> tuple[float, float]:
    """det(A')/det(A) = 1 + u^T A^{-1} e_i (Eq. 13), and the log-det cross-check."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    an = np.ascontiguousarray(a_new, dtype=np.float64)
    r = C.c_double(0.0)
    rl = C.c_double(0.0)
    rc = lib().orc_ratio_dense(A.shape[0], _ptr(A), i, _ptr(an), C.byref(r), C.byref(rl))
    if rc:
        raise np.linalg.LinAlgError("singular")
    return r.value, rl.value


def inverse(A: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.zeros_like(A)
    if lib().orc_inverse(A.shape[0], _ptr(A), _ptr(B)):
        raise np.linalg.LinAlgError("singular")
    return B


def sm_ratio(B: np.ndarray, i: int, u) -> float:
    uu = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_sm_ratio(B.shape[0], _ptr(B), i, _ptr(uu))


def sm_update(B: np.ndarray, i: int, u, ratio: float) -> None:
    uu = np.ascontiguousarray(u, dtype=np.float64)
    work = np.zeros(2 * B.shape[0])
    lib().orc_sm_update(B.shape[0], _ptr(B), i, _ptr(uu), ratio, _ptr(work))


def gmres(rowptr, col, val, b, restart=200, max_iter=20000, tol=1e-14):
    n = len(rowptr) - 1
    x = np.zeros(n)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    its = lib().orc_gmres(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(bb), _ptr(x), restart, max_iter, tol)
    return x, its


# ---- chains ---------------------------------------------------------------------------
SOLVER_DENSE_LU, SOLVER_SHERMAN_MORRISON, SOLVER_GMRES = 0, 1, 2


def chain(s: System, seed: int, sigma: float, R0: np.ndarray, n_sweeps: int, first_sweep: int = 0,
          max_steps: int = -1, solver: int = SOLVER_DENSE_LU, refresh: int = 0):
    """Independent Metropolis chain of one walker (Sec. 2.2): returns (R, ratios, accepts, U)."""
    n = n_of(s)
    R = np.ascontiguousarray(R0, dtype=np.float64).copy()
    steps = n_sweeps * n if max_steps < 0 else min(max_steps, n_sweeps * n)
    rl = np.zeros(steps)
    al = np.zeros(steps, dtype=np.uint8)
    ul = np.zeros(steps)
    got = lib().orc_chain(C.byref(s), seed, sigma, first_sweep, n_sweeps, max_steps, solver, refresh,
                          _ptr(R), _ptr(rl), _ptr(al), _ptr(ul))
    if got < 0:
        raise np.linalg.LinAlgError("singular Slater matrix in chain")
    return R, rl[:got], al[:got].astype(bool), ul[:got]


def chains(s: System, seeds, sigma: float, R0: np.ndarray, n_sweeps: int, first_sweep: int = 0,
           max_steps: int = -1, solver: int = SOLVER_SHERMAN_MORRISON, refresh: int = 0, threads: int = 0):
    """Several independent walkers, OpenMP across walkers."""
    n = n_of(s)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    W = len(seeds)
    R = np.ascontiguousarray(R0, dtype=np.float64).reshape(W, n, 3).copy()
    per = n_sweeps * n if max_steps < 0 else min(max_steps, n_sweeps * n)
    rl = np.zeros((W, per))
    al = np.zeros((W, per), dtype=np.uint8)
    got = lib().orc_chains(C.byref(s), W, _ptr(seeds), sigma, first_sweep, n_sweeps, max_steps, solver,
                           refresh, _ptr(R), _ptr(rl), _ptr(al), threads)
    if got < 0:
        raise np.linalg.LinAlgError("singular Slater matrix in chain")
    return R, rl, al.astype(bool)


def max_threads() -> int:
    return lib().orc_max_threads()


def greedy_pairing(s: System, R: np.ndarray, Z: np.ndarray, P, Q):
    """The greedy particle/orbital reordering of Sec. 3.1; returns the new (P, Q)."""
    PP = np.ascontiguousarray(P, dtype=np.int32).copy()
    QQ = np.ascontiguousarray(Q, dtype=np.int32).copy()
    lib().orc_greedy_pairing(C.byref(s), _ptr(np.ascontiguousarray(R)), _ptr(np.ascontiguousarray(Z)),
                             _ptr(PP), _ptr(QQ))
    return PP, QQ


def kinetic_energy(s: System, Z: np.ndarray, R: np.ndarray) -> float:
    """Kinetic-energy estimator of Eq. 21 (hbar = mass = 1)."""
    return lib().orc_kinetic_energy(C.byref(s), _ptr(Z), _ptr(np.ascontiguousarray(R)))


def ratio_grad_lap(s: System, Z: np.ndarray, R: np.ndarray, i: int, r_new):
    """(ratio, grad ln|det A'| at r_new, lap det A' / det A' at r_new) for moving particle i."""
    rn = np.ascontiguousarray(r_new, dtype=np.float64)
    ratio = C.c_double(0.0)
    g = np.zeros(3)
    lap = C.c_double(0.0)
    rc = lib().orc_ratio_grad_lap(C.byref(s), _ptr(Z), _ptr(np.ascontiguousarray(R)), int(i), _ptr(rn),
                                  C.byref(ratio), _ptr(g), C.byref(lap))
    if rc:
        raise RuntimeError("singular Slater matrix")
    return ratio.value, g, lap.value
