"""Python binding of the SSQA C-ABI library (include/ssqa.h).

Argument marshalling only: every step of an anneal runs in the CUDA kernels
of ``libssqa.so``.  The library must have been built (``build.build()``);
there is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libssqa.so")

OK, PENDING = 0, 1
ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_BUDGET, ERR_TIMEOUT, ERR_DEVICE, ERR_NOT_FOUND = -1, -2, -3, -4, -5, -6, -7
COUPLING_UPPER, COUPLING_BOTH = 0, 1
INIT_RANDOM, INIT_ALL_MINUS, INIT_FROM_STATE = 0, 1, 2
ALGO_AUTO, ALGO_PLAIN, ALGO_TENSOR, ALGO_DELTA, ALGO_STREAMED = 0, 1, 2, 3, 4
FLAG_TRACK_BEST, FLAG_DEVICE_PTRS = 1, 2


class SSQAError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ssqa error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("R", ctypes.c_int32), ("cycles", ctypes.c_int32), ("trials", ctypes.c_int32),
        ("I0", ctypes.c_int32), ("alpha", ctypes.c_int32), ("n_rnd", ctypes.c_int32),
        ("jperp_min", ctypes.c_int32), ("jperp_max", ctypes.c_int32), ("beta", ctypes.c_int32),
        ("tau", ctypes.c_int32), ("delay", ctypes.c_int32), ("coupling", ctypes.c_int32),
        ("init_mode", ctypes.c_int32), ("algo", ctypes.c_int32), ("flags", ctypes.c_uint32),
        ("start_cycle", ctypes.c_int32), ("trial_offset", ctypes.c_uint32), ("seed", ctypes.c_uint64),
        ("i0_max", ctypes.c_int32), ("i0_mult", ctypes.c_int32), ("i0_tau", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("sigma", ctypes.c_void_p), ("sigma_hist", ctypes.c_void_p), ("is_state", ctypes.c_void_p),
        ("e_final", ctypes.c_void_p), ("e_best", ctypes.c_void_p), ("best_cycle", ctypes.c_void_p),
        ("e_trace", ctypes.c_void_p),
    ]


_lib = None


def lib():
    """Load libssqa.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2302_12454_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, u32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64
        L.ssqa_gen_er_graph.argtypes = [i32, u32, u64, vp]
        L.ssqa_permute_graph.argtypes = [i32, vp, u64, vp, vp]
        L.ssqa_build_gi_ising.argtypes = [i32, vp, vp, i32, i32, i32, ctypes.POINTER(vp)]
        L.ssqa_ising_from_dense.argtypes = [i32, vp, vp, i64, ctypes.POINTER(vp)]
        L.ssqa_ising_free.argtypes = [vp]
        L.ssqa_ising_free.restype = None
        L.ssqa_ising_export.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), vp, vp]
        L.ssqa_params_default.argtypes = [ctypes.POINTER(Params)]
        L.ssqa_params_default.restype = None
        L.ssqa_anneal.argtypes = [vp, ctypes.POINTER(Params), ctypes.POINTER(Result), vp]
        L.ssqa_energy.argtypes = [vp, vp, i64, vp, u32, vp]
        L.ssqa_plan.argtypes = [vp, ctypes.POINTER(Params), ctypes.c_char_p, ctypes.c_size_t]
        L.ssqa_anneal_batch.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(Params), ctypes.POINTER(Result),
                                        ctypes.POINTER(i32), vp]
        L.ssqa_anneal_noalloc.argtypes = [i32, vp, vp, ctypes.POINTER(Params), ctypes.POINTER(Result), vp]
        L.ssqa_set_wait_limit.argtypes = [i64]
        L.ssqa_tts.argtypes = [ctypes.c_double] * 3
        L.ssqa_tts.restype = ctypes.c_double
        L.ssqa_last_error.argtypes = []
        L.ssqa_last_error.restype = ctypes.c_char_p
        L.ssqa_server_create.argtypes = [ctypes.c_size_t, i32, i32, ctypes.POINTER(vp)]
        L.ssqa_server_destroy.argtypes = [vp]
        L.ssqa_server_destroy.restype = None
        L.ssqa_submit.argtypes = [vp, vp, ctypes.POINTER(Params), ctypes.POINTER(u64)]
        L.ssqa_poll.argtypes = [vp, u64, ctypes.POINTER(Result), i32, ctypes.POINTER(ctypes.c_double)]
        _lib = L
    return _lib


def last_error() -> str:
    return lib().ssqa_last_error().decode()


def _check(rc: int, what: str):
    if rc < 0:
        raise SSQAError(rc, f"{what}: {last_error()}")
    return rc


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())  # torch tensor


# ---------------------------------------------------------------- instances
def gen_er_graph(n: int, p_q32: int, seed: int) -> np.ndarray:
    adj = np.zeros((n, n), np.uint8)
    _check(lib().ssqa_gen_er_graph(n, p_q32, seed, _ptr(adj)), "gen_er_graph")
    return adj


def permute_graph(adj: np.ndarray, seed: int):
    adj = np.ascontiguousarray(adj, np.uint8)
    out = np.zeros_like(adj)
    perm = np.zeros(adj.shape[0], np.int32)
    _check(lib().ssqa_permute_graph(adj.shape[0], _ptr(adj), seed, _ptr(out), _ptr(perm)), "permute_graph")
    return out, perm


class Ising:
    """Library-owned Ising instance (freed with the Python object)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @classmethod
    def gi(cls, adj1, adj2, C1: int = 1, C2: int = 1, scale: int = 12) -> "Ising":
        a1 = np.ascontiguousarray(adj1, np.uint8)
        a2 = np.ascontiguousarray(adj2, np.uint8)
        out = ctypes.c_void_p()
        _check(lib().ssqa_build_gi_ising(a1.shape[0], _ptr(a1), _ptr(a2), C1, C2, scale, ctypes.byref(out)),
               "build_gi_ising")
        return cls(out.value)

    @classmethod
    def dense(cls, J, h, e_offset: int = 0) -> "Ising":
        J = np.ascontiguousarray(J, np.int8)
        h = np.ascontiguousarray(h, np.int32)
        out = ctypes.c_void_p()
        _check(lib().ssqa_ising_from_dense(h.shape[0], _ptr(J), _ptr(h), e_offset, ctypes.byref(out)),
               "ising_from_dense")
        return cls(out.value)

    @property
    def handle(self):
        return self._h

    def export(self):
        N = ctypes.c_int32()
        off = ctypes.c_int64()
        _check(lib().ssqa_ising_export(self._h, ctypes.byref(N), ctypes.byref(off), None, None), "export")
        h = np.zeros(N.value, np.int32)
        J = np.zeros((N.value, N.value), np.int8)
        _check(lib().ssqa_ising_export(self._h, None, None, _ptr(h), _ptr(J)), "export")
        return h, J, off.value

    @property
    def N(self) -> int:
        N = ctypes.c_int32()
        _check(lib().ssqa_ising_export(self._h, ctypes.byref(N), None, None, None), "export")
        return N.value

    def __del__(self):
        if getattr(self, "_h", None) is not None and self._h.value and _lib is not None:
            _lib.ssqa_ising_free(self._h)
            self._h = None


# ------------------------------------------------------------------ anneal
PAPER_DEFAULTS = dict(I0=24, alpha=1, n_rnd=12, jperp_min=0, jperp_max=6, beta=3, tau=100, delay=1,
                      coupling=COUPLING_UPPER, init_mode=INIT_RANDOM, algo=ALGO_AUTO)


def make_params(*, R: int, cycles: int, trials: int, seed: int, **kw) -> Params:
    p = Params()
    lib().ssqa_params_default(ctypes.byref(p))
    p.R, p.cycles, p.trials, p.seed = R, cycles, trials, seed
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def anneal(ising: Ising, *, R: int, cycles: int, trials: int, seed: int, track_best: bool = False,
           state=None, want_hist: bool = False, want_trace: bool = False, want_state: bool = True, stream=None,
           out=None, **kw):
    """Anneal with host buffers; returns numpy arrays (sigma, Is, E_final, ...).
    want_trace (implies track_best): E_trace [cycles, trials, R], the energy of
    every replica after every cycle.  want_state=False: the counters Is are not
    returned (nor copied back); needed only to resume.  out: optional dict of
    caller-owned result arrays to fill instead of fresh ones (sigma int8
    [T,R,N], Is int32 [T,R,N], E_final int64 [T,R]), e.g. pinned buffers
    reused across calls."""
    track_best = track_best or want_trace
    N = ising.N
    p = make_params(R=R, cycles=cycles, trials=trials, seed=seed, **kw)
    if track_best:
        p.flags |= FLAG_TRACK_BEST
    d = p.delay

    def _buf(key, shape, dtype):
        if out is not None and key in out:
            a = out[key]
            if a.shape != shape or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"out[{key!r}] must be a C-contiguous {np.dtype(dtype)} array of shape {shape}")
            return a
        return np.zeros(shape, dtype)

    sigma = _buf("sigma", (trials, R, N), np.int8)
    if state is not None and not want_state:
        raise ValueError("resuming (state=...) needs want_state=True")
    Is = _buf("Is", (trials, R, N), np.int32) if want_state else None
    hist = np.zeros((trials, d, R, N), np.int8) if (d and (want_hist or state is not None)) else None
    if state is not None:
        sigma[...] = state["sigma"]
        Is[...] = state["Is"]
        if hist is not None:
            hist[...] = state["hist"]
    E = _buf("E_final", (trials, R), np.int64)
    Eb = np.zeros((trials, R), np.int64) if track_best else None
    bc = np.zeros((trials, R), np.int32) if track_best else None
    tr = np.zeros((cycles, trials, R), np.int64) if want_trace else None
    r = Result(_ptr(sigma), _ptr(hist), _ptr(Is), _ptr(E), _ptr(Eb), _ptr(bc), _ptr(tr))
    st = None if stream is None else ctypes.c_void_p(int(stream))
    _check(lib().ssqa_anneal(ising.handle, ctypes.byref(p), ctypes.byref(r), st), "anneal")
    out = dict(sigma=sigma, E_final=E)
    if want_state:
        out["Is"] = Is
    if hist is not None:
        out["hist"] = hist
    if track_best:
        out.update(E_best=Eb, best_cycle=bc)
    if want_trace:
        out["E_trace"] = tr
    return out


def anneal_device(ising: Ising, params: Params, sigma, Is, e_final=None, hist=None, e_best=None, best_cycle=None,
                  stream=None, e_trace=None):
    """Anneal on device buffers (torch CUDA tensors); enqueued on `stream`
    (a torch.cuda.Stream or raw handle, default: torch's current stream)."""
    import torch

    p = Params.from_buffer_copy(params)
    p.flags |= FLAG_DEVICE_PTRS
    if e_best is not None:
        p.flags |= FLAG_TRACK_BEST
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    r = Result(_ptr(sigma), _ptr(hist), _ptr(Is), _ptr(e_final), _ptr(e_best), _ptr(best_cycle), _ptr(e_trace))
    _check(lib().ssqa_anneal(ising.handle, ctypes.byref(p), ctypes.byref(r), ctypes.c_void_p(handle)), "anneal")


def plan(ising: Ising, *, R: int, cycles: int, trials: int, seed: int = 0, track_best: bool = False, **kw):
    """(algo, description) of the kernel path ssqa_anneal would take (host only)."""
    p = make_params(R=R, cycles=cycles, trials=trials, seed=seed, **kw)
    if track_best:
        p.flags |= FLAG_TRACK_BEST
    buf = ctypes.create_string_buffer(512)
    rc = _check(lib().ssqa_plan(ising.handle, ctypes.byref(p), buf, 512), "plan")
    return rc, buf.value.decode()


def anneal_batch(items, stream=None) -> int:
    """Several device-buffer anneals in as few launches as possible
    (ssqa_anneal_batch).  items: list of (ising, params, buffers) with buffers a
    dict of torch CUDA tensors (sigma, Is, and optionally hist, e_final,
    e_best, best_cycle, e_trace).  Returns the number of kernel launches."""
    import torch

    n = len(items)
    isings = (ctypes.c_void_p * n)(*[it[0].handle.value for it in items])
    ps = (Params * n)()
    rs = (Result * n)()
    for k, (ising, params, buf) in enumerate(items):
        p = Params.from_buffer_copy(params)
        p.flags |= FLAG_DEVICE_PTRS
        if buf.get("e_best") is not None:
            p.flags |= FLAG_TRACK_BEST
        ps[k] = p
        rs[k] = Result(_ptr(buf["sigma"]), _ptr(buf.get("hist")), _ptr(buf["Is"]), _ptr(buf.get("e_final")),
                       _ptr(buf.get("e_best")), _ptr(buf.get("best_cycle")), _ptr(buf.get("e_trace")))
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    launches = ctypes.c_int32()
    _check(lib().ssqa_anneal_batch(n, isings, ps, rs, ctypes.byref(launches), ctypes.c_void_p(handle)),
           "anneal_batch")
    return launches.value


def energy(ising: Ising, sigma) -> np.ndarray:
    s = np.ascontiguousarray(sigma, np.int8)
    N = ising.N
    flat = s.reshape(-1, N)
    E = np.zeros(flat.shape[0], np.int64)
    _check(lib().ssqa_energy(ising.handle, _ptr(flat), flat.shape[0], _ptr(E), 0, None), "energy")
    return E.reshape(s.shape[:-1])


def set_wait_limit(clocks: int) -> None:
    """Bound of the tensor-core kernels' device waits in SM clocks (0: default)."""
    _check(lib().ssqa_set_wait_limit(int(clocks)), "set_wait_limit")


def tts(t: float, p_s: float, p_target: float = 0.99) -> float:
    return float(lib().ssqa_tts(t, p_s, p_target))


# ----------------------------------------------------------------- serving
class Server:
    """Continuous-batching server (ssqa_server_*): submit anneals, poll results."""

    def __init__(self, hbm_budget: int, max_slots: int = 4, device: int = 0):
        self._s = ctypes.c_void_p()
        _check(lib().ssqa_server_create(hbm_budget, max_slots, device, ctypes.byref(self._s)), "server_create")
        self._pending = {}

    def submit(self, ising: Ising, *, R: int, cycles: int, trials: int, seed: int, track_best: bool = False,
               **kw) -> int:
        p = make_params(R=R, cycles=cycles, trials=trials, seed=seed, **kw)
        if track_best:
            p.flags |= FLAG_TRACK_BEST
        t = ctypes.c_uint64()
        _check(lib().ssqa_submit(self._s, ising.handle, ctypes.byref(p), ctypes.byref(t)), "submit")
        self._pending[t.value] = (ising, p)  # keeps the instance alive until polled
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """Returns None while pending, else (result dict, latency in seconds)."""
        ising, p = self._pending[ticket]
        N, T, R, d = ising.N, p.trials, p.R, p.delay
        out = dict(sigma=np.zeros((T, R, N), np.int8), Is=np.zeros((T, R, N), np.int32),
                   E_final=np.zeros((T, R), np.int64))
        if d:
            out["hist"] = np.zeros((T, d, R, N), np.int8)
        tb = p.flags & FLAG_TRACK_BEST
        if tb:
            out["E_best"] = np.zeros((T, R), np.int64)
            out["best_cycle"] = np.zeros((T, R), np.int32)
        r = Result(_ptr(out["sigma"]), _ptr(out.get("hist")), _ptr(out["Is"]), _ptr(out["E_final"]),
                   _ptr(out.get("E_best")), _ptr(out.get("best_cycle")))
        lat = ctypes.c_double()
        rc = lib().ssqa_poll(self._s, ticket, ctypes.byref(r), timeout_ms, ctypes.byref(lat))
        if rc == PENDING:
            return None
        del self._pending[ticket]
        _check(rc, "poll")
        return out, lat.value * 1e-6

    def close(self):
        if self._s is not None and self._s.value:
            lib().ssqa_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
