"""A bounded device wait made to run out, on the GPU, without a fault.

Every wait of the tensor-core kernels (for the tensor cores, the bulk copies
or another warp) gives up after ssqa_set_wait_limit clocks: the kernel stops
its work, lets its own MMAs and copies in flight finish, frees its tensor
memory and returns, and the call reports SSQA_ERR_TIMEOUT.  With a limit of
100 SM clocks -- far shorter than one chunk of MMAs or one copy -- a resident
(N = 400) and a streamed (N = 529) anneal must return SSQA_ERR_TIMEOUT; after
the default is restored the same calls run in the same CUDA context and match
the oracle bit for bit."""
import numpy as np
import pytest

import paper_2302_12454_gb300 as S
from paper_2302_12454_gb300 import build as B
from paper_2302_12454_gb300 import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _gi(n, gseed, pseed):
    a = S.gen_er_graph(n, W.p_q32(0.5), gseed)
    b, _ = S.permute_graph(a, pseed)
    return S.Ising.gi(a, b)


def test_wait_limit_runs_out_then_recovers():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    cases = [(_gi(20, 3, 4), S.ALGO_TENSOR), (_gi(23, 5, 6), S.ALGO_STREAMED)]
    kw = dict(R=16, cycles=6, trials=8, seed=21, tau=3)
    S.set_wait_limit(100)
    try:
        for I, algo in cases:
            with pytest.raises(S.SSQAError) as e:
                S.anneal(I, algo=algo, **kw)
            assert e.value.code == S.ERR_TIMEOUT, (algo, str(e.value))
    finally:
        S.set_wait_limit(0)
    for I, algo in cases:
        g = S.anneal(I, algo=algo, track_best=True, **kw)
        h, J, _ = I.export()
        o = O.anneal(h, J, track_best=True, **kw)
        for k in ("sigma", "Is", "E_final", "E_best", "best_cycle"):
            np.testing.assert_array_equal(g[k], o[k], err_msg=f"{k} algo {algo}")
    with pytest.raises(S.SSQAError):
        S.set_wait_limit(-1)
