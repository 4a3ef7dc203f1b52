"""CPU tests of the C ABI: the library builds and loads, exports every
declared entry point, and its host-side logic (graph generation, GI
instance construction, TTS, argument checking) agrees with the oracle.
No compute call is made here (they need a GPU)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_2302_12454_gb300 as S
from paper_2302_12454_gb300 import build as B
from paper_2302_12454_gb300 import workloads as W
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "ssqa.h")).read()
    return sorted(set(re.findall(r"\b(ssqa_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 15
    L = ctypes.CDLL(S.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("n,p,seed", [(1, 0.5, 0), (6, 0.5, 1), (20, 0.5, 11), (50, 0.3, 21), (50, 0.7, 23), (33, 0.9, 5)])
def test_graph_generators_match_oracle(n, p, seed):
    a = S.gen_er_graph(n, W.p_q32(p), seed)
    assert np.array_equal(a, O.gen_er_graph(n, W.p_q32(p), seed))
    b, perm = S.permute_graph(a, seed + 1)
    ob, operm = O.permute_graph(a, seed + 1)
    assert np.array_equal(b, ob) and np.array_equal(perm, operm)


@pytest.mark.parametrize("n,C1,C2,scale", [(3, 1, 1, 12), (6, 1, 1, 12), (7, 2, 3, 4), (10, 1, 1, 12), (12, 3, 1, 8)])
def test_gi_builder_matches_oracle(n, C1, C2, scale):
    a = O.gen_er_graph(n, W.p_q32(0.5), n)
    b, _ = O.permute_graph(a, n + 7)
    b = b.copy()
    if n > 3:
        b[0, 2] ^= 1
        b[2, 0] ^= 1
    I = S.Ising.gi(a, b, C1, C2, scale)
    h, J, off = I.export()
    oh, oJ, ooff = O.build_gi_ising(a, b, C1, C2, scale)
    assert np.array_equal(h, oh) and np.array_equal(J, oJ) and off == ooff


def test_dense_instance_roundtrip_and_checks():
    J = W.sk_couplings(64, 5)
    h = np.arange(64, dtype=np.int32) - 30
    I = S.Ising.dense(J, h, 17)
    h2, J2, off = I.export()
    assert np.array_equal(J, J2) and np.array_equal(h, h2) and off == 17
    bad = J.copy()
    bad[0, 1] = 3
    with pytest.raises(S.SSQAError) as e:
        S.Ising.dense(bad, h)
    assert e.value.code == S.ERR_INVALID_ARG
    bad = J.copy()
    bad[3, 3] = 1
    with pytest.raises(S.SSQAError):
        S.Ising.dense(bad, h)


def test_dense_instance_symmetry_checked_in_every_tile():
    """The symmetry check runs over 32 x 32 tiles; a single asymmetric pair
    anywhere (corner tiles, the ragged last tile of N = 77, either triangle)
    is rejected, and the symmetric instance is accepted."""
    N = 77
    J = W.sk_couplings(N, 9)
    h = np.zeros(N, np.int32)
    S.Ising.dense(J, h)
    for i, j in ((76, 0), (0, 76), (40, 70), (33, 65), (31, 32), (64, 76), (75, 74)):
        bad = J.copy()
        bad[i, j] = -bad[i, j] if bad[i, j] else 12
        with pytest.raises(S.SSQAError) as e:
            S.Ising.dense(bad, h)
        assert e.value.code == S.ERR_INVALID_ARG, (i, j)


def test_gi_builder_rejects_bad_graphs():
    a = np.zeros((4, 4), np.uint8)
    a[0, 1] = 1  # asymmetric
    with pytest.raises(S.SSQAError):
        S.Ising.gi(a, np.zeros((4, 4), np.uint8))
    with pytest.raises(S.SSQAError):
        S.Ising.gi(np.zeros((4, 4), np.uint8), np.zeros((4, 4), np.uint8), 1, 1, 3)  # non-integral


def test_tts_matches_oracle_and_limits():
    for t, p in ((5.42, 0.95), (22.7, 0.51), (46.4, 0.41), (1.0, 0.5)):
        assert math.isclose(S.tts(t, p), O.tts(t, p), rel_tol=1e-12)
    assert S.tts(1.0, 1.0) == 0.0
    assert math.isinf(S.tts(1.0, 0.0))
    assert math.isnan(S.tts(1.0, 0.5, 1.5))


@pytest.mark.parametrize("bad", [dict(R=0), dict(R=129), dict(I0=0), dict(alpha=0), dict(alpha=49),
                                 dict(beta=0), dict(tau=0), dict(delay=4), dict(jperp_max=5),
                                 dict(coupling=2), dict(init_mode=3), dict(algo=7), dict(flags=64)])
def test_anneal_argument_checks(bad):
    a = O.gen_er_graph(4, W.p_q32(0.5), 1)
    I = S.Ising.gi(a, a)
    kw = dict(R=4, cycles=5, trials=2, seed=1)
    kw.update(bad)
    with pytest.raises(S.SSQAError) as e:
        S.anneal(I, **kw)
    assert e.value.code == S.ERR_INVALID_ARG


def test_counters_are_required_only_to_resume_or_on_device():
    """is_state may be NULL for a fresh anneal into host buffers; with device
    pointers or when resuming it is required, which is checked before any
    device work."""
    import torch
    a = O.gen_er_graph(4, W.p_q32(0.5), 1)
    I = S.Ising.gi(a, a)
    sig = np.zeros((2, 3, 16), np.int8)
    for flags, init in ((S.FLAG_DEVICE_PTRS, S.INIT_RANDOM), (0, S.INIT_FROM_STATE)):
        p = S.make_params(R=3, cycles=1, trials=2, seed=1, init_mode=init, delay=0)
        p.flags |= flags
        r = S.Result(S._ptr(sig), None, None, None, None, None, None)
        assert S.lib().ssqa_anneal(I.handle, ctypes.byref(p), ctypes.byref(r), None) == S.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        S.anneal(I, R=3, cycles=1, trials=2, seed=1, delay=0, want_state=False,
                 init_mode=S.INIT_FROM_STATE, state={"sigma": sig, "Is": np.zeros((2, 3, 16), np.int32)})
    if not torch.cuda.is_available():
        with pytest.raises(S.SSQAError) as e:  # accepted by validation, then no device
            S.anneal(I, R=3, cycles=1, trials=2, seed=1, want_state=False)
        assert e.value.code == S.ERR_DEVICE


def test_compute_calls_fail_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    a = O.gen_er_graph(4, W.p_q32(0.5), 1)
    I = S.Ising.gi(a, a)
    with pytest.raises(S.SSQAError) as e:
        S.anneal(I, R=2, cycles=3, trials=1, seed=1)
    assert e.value.code == S.ERR_DEVICE
    with pytest.raises(S.SSQAError) as e:
        S.energy(I, np.ones((1, 16), np.int8))
    assert e.value.code == S.ERR_DEVICE
    srv = ctypes.c_void_p()
    assert S.lib().ssqa_server_create(1 << 30, 2, 0, ctypes.byref(srv)) == S.ERR_DEVICE


def test_params_default_is_table2():
    p = S.make_params(R=25, cycles=1600, trials=100, seed=0)
    assert (p.I0, p.alpha, p.n_rnd, p.jperp_min, p.jperp_max, p.beta, p.tau, p.delay) == (24, 1, 12, 0, 6, 3, 100, 1)


def test_anneal_out_buffers_are_checked():
    """Caller-owned result arrays (out=) must have the result's shape, dtype
    and layout; a mismatch is rejected before any device work."""
    a = S.gen_er_graph(4, W.p_q32(0.5), 1)
    b, _ = S.permute_graph(a, 2)
    I = S.Ising.gi(a, b)
    for bad in ({"sigma": np.zeros((2, 3, 15), np.int8)}, {"Is": np.zeros((2, 3, 16), np.int64)},
                {"E_final": np.zeros((3, 2), np.int64)}, {"sigma": np.zeros((2, 16, 3), np.int8).transpose(0, 2, 1)}):
        with pytest.raises(ValueError):
            S.anneal(I, R=3, cycles=1, trials=2, seed=1, out=bad)


def test_noalloc_rejects_misaligned_pointers_before_any_launch():
    """ssqa_anneal_noalloc checks the alignment of every caller pointer on
    the host.  The pointers here are fake device addresses that are never
    dereferenced: each call must return SSQA_ERR_INVALID_ARG before touching
    the device.  (Skipped where a GPU is present, so that a checking bug can
    never turn into a launch on fake addresses.)"""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("host-only check; runs where no GPU is present")
    L = S.lib()
    p = S.make_params(R=4, cycles=3, trials=2, seed=1)
    p.flags = S.FLAG_DEVICE_PTRS | S.FLAG_TRACK_BEST
    base = dict(J=0x10000, h=0x20000, sigma=0x30000, hist=0x40000, Is=0x50000, E=0x60000, Eb=0x70000,
                bc=0x80000, tr=0x90000)
    for key, off in (("J", 8), ("J", 1), ("h", 2), ("Is", 1), ("bc", 2), ("E", 4), ("Eb", 2), ("tr", 4)):
        ptr = dict(base)
        ptr[key] += off
        r = S.Result(ptr["sigma"], ptr["hist"], ptr["Is"], ptr["E"], ptr["Eb"], ptr["bc"], ptr["tr"])
        rc = L.ssqa_anneal_noalloc(36, ctypes.c_void_p(ptr["J"]), ctypes.c_void_p(ptr["h"]), ctypes.byref(p),
                                   ctypes.byref(r), None)
        assert rc == S.ERR_INVALID_ARG, (key, off, rc)
        assert "aligned" in S.last_error(), S.last_error()
