"""GPU parity of the per-cycle energy trace (the waveform of Fig. 6):
E_trace[c] = E(sigma(t0 + c + 1)) of every replica, from every anneal path,
bit-exact against the oracle's trace."""
import numpy as np
import pytest

import paper_2302_12454_gb300 as S
from paper_2302_12454_gb300 import build as B
from paper_2302_12454_gb300 import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def gi(n, gseed, pseed):
    a = S.gen_er_graph(n, W.p_q32(0.5), gseed)
    b, _ = S.permute_graph(a, pseed)
    return S.Ising.gi(a, b)


@pytest.mark.parametrize("algo,n", [(S.ALGO_TENSOR, 9), (S.ALGO_PLAIN, 9), (S.ALGO_DELTA, 9),
                                    (S.ALGO_STREAMED, 17), (S.ALGO_TENSOR, 20)])
def test_trace_bit_exact(algo, n):
    I = gi(n, 90 + n, 91 + n)
    h, J, off = I.export()
    kw = dict(R=6, cycles=33, trials=5, seed=92, tau=4, trial_offset=3, start_cycle=7)
    g = S.anneal(I, algo=algo, want_trace=True, **kw)
    o = O.anneal(h, J, track_best=True, trace=True, **kw)
    assert g["E_trace"].shape == (33, 5, 6)
    np.testing.assert_array_equal(g["E_trace"], o["E_trace"])
    np.testing.assert_array_equal(g["E_best"], o["E_best"])
    np.testing.assert_array_equal(g["best_cycle"], o["best_cycle"])
    np.testing.assert_array_equal(g["E_trace"][-1], g["E_final"])


def test_trace_needs_tracking():
    I = gi(6, 1, 2)
    p = S.make_params(R=2, cycles=3, trials=1, seed=1)
    sig = np.zeros((1, 2, 36), np.int8)
    Is = np.zeros((1, 2, 36), np.int32)
    tr = np.zeros((3, 1, 2), np.int64)
    r = S.Result(S._ptr(sig), None, S._ptr(Is), None, None, None, S._ptr(tr))
    import ctypes
    rc = S.lib().ssqa_anneal(I.handle, ctypes.byref(p), ctypes.byref(r), None)
    assert rc == S.ERR_INVALID_ARG
