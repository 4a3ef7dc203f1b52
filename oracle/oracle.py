"""ctypes front end of the plain C SSQA oracle (``ssqa_oracle.c``).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module; the product library
never does.  Every function is a thin marshalling wrapper; the arithmetic is
in the C file, which cites the paper passage each function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ssqa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libssqa_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32), ("R", ctypes.c_int32), ("cycles", ctypes.c_int32),
        ("I0", ctypes.c_int32), ("alpha", ctypes.c_int32), ("n_rnd", ctypes.c_int32),
        ("jperp_min", ctypes.c_int32), ("jperp_max", ctypes.c_int32),
        ("beta", ctypes.c_int32), ("tau", ctypes.c_int32), ("delay", ctypes.c_int32),
        ("coupling_both", ctypes.c_int32), ("init_mode", ctypes.c_int32),
        ("start_cycle", ctypes.c_int32), ("seed", ctypes.c_uint64),
        ("i0_max", ctypes.c_int32), ("i0_mult", ctypes.c_int32), ("i0_tau", ctypes.c_int32),
    ]


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u8p = i8p = i32p = i64p = u32p = ctypes.c_void_p
            L.or_splitmix64_next.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
            L.or_splitmix64_next.restype = ctypes.c_uint64
            L.or_gen_er_graph.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, u8p]
            L.or_permute_graph.argtypes = [ctypes.c_int, u8p, ctypes.c_uint64, u8p, i32p]
            L.or_gi_hamiltonian.argtypes = [ctypes.c_int, u8p, u8p, ctypes.c_int64, ctypes.c_int64, u8p]
            L.or_gi_hamiltonian.restype = ctypes.c_int64
            L.or_gi_qubo.argtypes = [ctypes.c_int, u8p, u8p, ctypes.c_int64, ctypes.c_int64, i64p, i64p]
            L.or_qubo_value.argtypes = [ctypes.c_int, i64p, ctypes.c_int64, u8p]
            L.or_qubo_value.restype = ctypes.c_int64
            L.or_qubo_to_ising.argtypes = [ctypes.c_int, i64p, ctypes.c_int64, ctypes.c_int64, i64p, i64p, i64p]
            L.or_ising_energy.argtypes = [ctypes.c_int, i64p, i64p, i8p]
            L.or_ising_energy.restype = ctypes.c_int64
            L.or_ising_energy_batch.argtypes = [ctypes.c_int, i64p, i64p, i8p, ctypes.c_int64, i64p]
            L.or_ising_energy_batch.restype = None
            L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.or_philox4x32_10.restype = None
            L.or_noise_bit.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
            L.or_jperp.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
            L.or_jperp.restype = ctypes.c_int32
            L.or_iterations.argtypes = [ctypes.c_double] * 4
            L.or_iterations.restype = ctypes.c_double
            L.or_tts.argtypes = [ctypes.c_double] * 3
            L.or_tts.restype = ctypes.c_double
            L.or_anneal.argtypes = [ctypes.POINTER(Params), i64p, i64p, ctypes.c_int32, ctypes.c_uint32,
                                    i8p, i8p, i32p, i64p, i64p, i32p, i64p]
            L.or_ssa_i0.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
            L.or_ssa_i0.restype = ctypes.c_int32
            L.or_ssa_trial.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_uint64, ctypes.c_uint32, i8p, i32p]
            _lib = L
    return _lib


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with {rc}")


# --------------------------------------------------------------------------
# graphs and instance construction (Sec. 4.1-4.2)
# --------------------------------------------------------------------------
def splitmix64(seed: int, count: int) -> np.ndarray:
    st = ctypes.c_uint64(seed)
    return np.array([lib().or_splitmix64_next(ctypes.byref(st)) for _ in range(count)], dtype=np.uint64)


def gen_er_graph(n: int, p_q32: int, seed: int) -> np.ndarray:
    adj = np.zeros((n, n), dtype=np.uint8)
    _check(lib().or_gen_er_graph(n, p_q32, seed, _p(adj)), "gen_er_graph")
    return adj


def permute_graph(adj: np.ndarray, seed: int):
    n = adj.shape[0]
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    out = np.zeros_like(adj)
    perm = np.zeros(n, dtype=np.int32)
    _check(lib().or_permute_graph(n, _p(adj), seed, _p(out), _p(perm)), "permute_graph")
    return out, perm


def gi_hamiltonian(adj1, adj2, C1: int, C2: int, x) -> int:
    n = adj1.shape[0]
    a1 = np.ascontiguousarray(adj1, dtype=np.uint8)
    a2 = np.ascontiguousarray(adj2, dtype=np.uint8)
    xx = np.ascontiguousarray(x, dtype=np.uint8).reshape(-1)
    return int(lib().or_gi_hamiltonian(n, _p(a1), _p(a2), C1, C2, _p(xx)))


def gi_qubo(adj1, adj2, C1: int = 1, C2: int = 1):
    n = adj1.shape[0]
    N = n * n
    a1 = np.ascontiguousarray(adj1, dtype=np.uint8)
    a2 = np.ascontiguousarray(adj2, dtype=np.uint8)
    Q = np.zeros((N, N), dtype=np.int64)
    c = np.zeros(1, dtype=np.int64)
    _check(lib().or_gi_qubo(n, _p(a1), _p(a2), C1, C2, _p(Q), _p(c)), "gi_qubo")
    return Q, int(c[0])


def qubo_value(Q, const_term: int, x) -> int:
    Q = np.ascontiguousarray(Q, dtype=np.int64)
    xx = np.ascontiguousarray(x, dtype=np.uint8).reshape(-1)
    return int(lib().or_qubo_value(Q.shape[0], _p(Q), const_term, _p(xx)))


def qubo_to_ising(Q, const_term: int, S: int = 12):
    Q = np.ascontiguousarray(Q, dtype=np.int64)
    N = Q.shape[0]
    h = np.zeros(N, dtype=np.int64)
    J = np.zeros((N, N), dtype=np.int64)
    off = np.zeros(1, dtype=np.int64)
    _check(lib().or_qubo_to_ising(N, _p(Q), const_term, S, _p(h), _p(J), _p(off)), "qubo_to_ising")
    return h, J, int(off[0])


def build_gi_ising(adj1, adj2, C1: int = 1, C2: int = 1, S: int = 12):
    """Eq. 8 -> Q -> (h', J', offset').  Ground energy of an isomorphic pair
    is -offset' (Eq. 8 vanishes exactly on isomorphisms)."""
    Q, c = gi_qubo(adj1, adj2, C1, C2)
    return qubo_to_ising(Q, c, S)


def ising_energy(h, J, sigma) -> np.ndarray:
    h = np.ascontiguousarray(h, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    s = np.ascontiguousarray(sigma, dtype=np.int8)
    N = h.shape[0]
    flat = s.reshape(-1, N)
    E = np.zeros(flat.shape[0], dtype=np.int64)
    lib().or_ising_energy_batch(N, _p(h), _p(J), _p(flat), flat.shape[0], _p(E))
    return E.reshape(s.shape[:-1])


# --------------------------------------------------------------------------
# Philox, schedules, TTS
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def noise_bit(seed: int, i: int, k: int, trial: int, t: int) -> int:
    return int(lib().or_noise_bit(seed, i, k, trial, t & 0xFFFFFFFF))


def jperp(t: int, jmin: int, jmax: int, beta: int, tau: int) -> int:
    return int(lib().or_jperp(t, jmin, jmax, beta, tau))


def iterations(EC, R, tau, beta) -> float:
    return float(lib().or_iterations(EC, R, tau, beta))


def tts(t: float, p_s: float, p_target: float = 0.99) -> float:
    return float(lib().or_tts(t, p_s, p_target))


def ssa_i0(t, i0_min, i0_max, i0_mult, tau) -> int:
    return int(lib().or_ssa_i0(t, i0_min, i0_max, i0_mult, tau))


# --------------------------------------------------------------------------
# SSQA / SSA anneals (Eq. 6, Eq. 2)
# --------------------------------------------------------------------------
PAPER_DEFAULTS = dict(I0=24, alpha=1, n_rnd=12, jperp_min=0, jperp_max=6, beta=3, tau=100,
                      delay=1, coupling_both=0, init_mode=0, start_cycle=0, i0_max=0, i0_mult=2, i0_tau=10)
"""Table 2 (J_perp 0..0.5, beta 3, d 1, I0 2, n_rnd 1) scaled by S = 12."""


def anneal(h, J, *, R: int, cycles: int, trials: int, seed: int, trial_offset: int = 0,
           track_best: bool = False, state=None, trace: bool = False, **kw):
    """Run Eq. 6 for `trials` trials; returns a dict of numpy arrays.

    state: optional dict(sigma [T,R,N] int8, hist [T,d,R,N] int8, Is [T,R,N] int32)
    used with init_mode=2 (resume).  trace: also return E_trace [cycles,T,R],
    the energy of every replica after every cycle (Fig. 6)."""
    h = np.ascontiguousarray(h, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    N = h.shape[0]
    cfg = dict(PAPER_DEFAULTS)
    cfg.update(kw)
    p = Params(N=N, R=R, cycles=cycles, seed=seed, **cfg)
    d = p.delay
    sigma = np.zeros((trials, R, N), dtype=np.int8)
    hist = np.zeros((trials, d, R, N), dtype=np.int8)
    Is = np.zeros((trials, R, N), dtype=np.int32)
    if state is not None:
        sigma[...] = state["sigma"]
        Is[...] = state["Is"]
        if d:
            hist[...] = state["hist"]
    E_final = np.zeros((trials, R), dtype=np.int64)
    E_best = np.zeros((trials, R), dtype=np.int64) if track_best else None
    best_cycle = np.zeros((trials, R), dtype=np.int32) if track_best else None
    E_trace = np.zeros((cycles, trials, R), dtype=np.int64) if trace else None
    rc = lib().or_anneal(ctypes.byref(p), _p(h), _p(J), trials, trial_offset, _p(sigma),
                         _p(hist), _p(Is), _p(E_final), _p(E_best), _p(best_cycle), _p(E_trace))
    _check(rc, "anneal")
    out = dict(sigma=sigma, hist=hist, Is=Is, E_final=E_final)
    if track_best:
        out.update(E_best=E_best, best_cycle=best_cycle)
    if trace:
        out["E_trace"] = E_trace
    return out


def ssa(h, J, *, cycles: int, seed: int, trial: int = 0, i0_min: int, i0_max: int,
        i0_mult: int = 2, tau: int = 10, alpha: int = 1, n_rnd: int):
    h = np.ascontiguousarray(h, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    N = h.shape[0]
    sigma = np.zeros(N, dtype=np.int8)
    Is = np.zeros(N, dtype=np.int32)
    _check(lib().or_ssa_trial(N, _p(h), _p(J), cycles, i0_min, i0_max, i0_mult, tau, alpha, n_rnd,
                              seed, trial, _p(sigma), _p(Is)), "ssa")
    return sigma, Is
