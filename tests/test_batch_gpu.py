"""Uneven problems in one launch (ssqa_anneal_batch): every problem's result
equals the same anneal made alone, bit for bit, and the problems the
resident kernel takes run as the column groups of one launch per kernel
variant.  The mix differs in instance and size (N = 36 .. 400 on the resident
kernel, N = 1000 on the streamed path), replicas, trials, cycles, seeds,
coupling mode and energy tracking."""
import numpy as np
import pytest

import paper_2302_12454_gb300 as S
from paper_2302_12454_gb300 import build as B
from paper_2302_12454_gb300 import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _gi(n, gseed):
    a = S.gen_er_graph(n, W.p_q32(0.5), gseed)
    b, _ = S.permute_graph(a, gseed + 1)
    return S.Ising.gi(a, b)


def _problems():
    sk250 = S.Ising.dense(W.sk_couplings(250, 5), np.zeros(250, np.int32))
    sk1000 = S.Ising.dense(W.sk_couplings(1000, 6), np.zeros(1000, np.int32))
    return [
        (_gi(6, 1), dict(R=8, trials=5, cycles=60, seed=1, tau=7), False),
        (_gi(9, 3), dict(R=16, trials=9, cycles=45, seed=2, tau=5), False),
        (_gi(17, 5), dict(R=4, trials=33, cycles=30, seed=3, tau=4), False),   # two MMA chunks
        (_gi(20, 7), dict(R=16, trials=12, cycles=40, seed=4, tau=6), False),  # N = 400
        (_gi(12, 9), dict(R=32, trials=3, cycles=80, seed=5, tau=9), False),
        (sk250, dict(R=8, trials=7, cycles=25, seed=6, tau=3), False),
        (_gi(7, 11), dict(R=16, trials=6, cycles=50, seed=7, tau=5), True),    # energy tracking
        (_gi(8, 13), dict(R=25, trials=4, cycles=40, seed=8, tau=5), False),   # R = 25: no batched variant
        (sk1000, dict(R=8, trials=3, cycles=12, seed=9, tau=3), False),        # streamed path
        (_gi(10, 15), dict(R=8, trials=5, cycles=35, seed=10, tau=4, coupling=S.COUPLING_BOTH), False),
    ]


def test_batch_equals_each_alone():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    probs = _problems()
    items, expect_groups, singles = [], set(), 0
    for I, kw, track in probs:
        N, T, R, C = I.N, kw["trials"], kw["R"], kw["cycles"]
        dev = torch.device("cuda")
        buf = dict(sigma=torch.zeros((T, R, N), dtype=torch.int8, device=dev),
                   Is=torch.zeros((T, R, N), dtype=torch.int32, device=dev),
                   hist=torch.zeros((T, 1, R, N), dtype=torch.int8, device=dev),
                   e_final=torch.zeros((T, R), dtype=torch.int64, device=dev))
        if track:
            buf.update(e_best=torch.zeros((T, R), dtype=torch.int64, device=dev),
                       best_cycle=torch.zeros((T, R), dtype=torch.int32, device=dev),
                       e_trace=torch.zeros((C, T, R), dtype=torch.int64, device=dev))
        items.append((I, S.make_params(**kw), buf))
        algo, desc = S.plan(I, track_best=track, **kw)
        if algo == S.ALGO_TENSOR and "shuffle" in desc and "byte" in desc:
            expect_groups.add((desc, track, kw.get("coupling", 0)))
        else:
            singles += 1
    launches = S.anneal_batch(items)
    torch.cuda.synchronize()
    assert launches == len(expect_groups) + singles < len(items), (launches, expect_groups, singles)
    for (I, kw, track), (_, _, buf) in zip(probs, items):
        ref = S.anneal(I, track_best=track, want_trace=track, want_hist=True, **kw)
        got = {k: v.cpu().numpy() for k, v in buf.items()}
        np.testing.assert_array_equal(got["sigma"], ref["sigma"])
        np.testing.assert_array_equal(got["Is"], ref["Is"])
        np.testing.assert_array_equal(got["hist"], ref["hist"])
        np.testing.assert_array_equal(got["e_final"], ref["E_final"])
        if track:
            np.testing.assert_array_equal(got["e_best"], ref["E_best"])
            np.testing.assert_array_equal(got["best_cycle"], ref["best_cycle"])
            np.testing.assert_array_equal(got["e_trace"], ref["E_trace"])
    # two of the batched problems against the oracle directly
    for j in (0, 3):
        I, kw, _ = probs[j]
        h, J, _ = I.export()
        o = O.anneal(h, J, **kw)
        got = items[j][2]
        np.testing.assert_array_equal(got["sigma"].cpu().numpy(), o["sigma"])
        np.testing.assert_array_equal(got["e_final"].cpu().numpy(), o["E_final"])


def test_batch_rejects_host_pointers():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    I = _gi(6, 1)
    buf = dict(sigma=torch.zeros((2, 8, 36), dtype=torch.int8, device="cuda"),
               Is=torch.zeros((2, 8, 36), dtype=torch.int32, device="cuda"))
    p = S.make_params(R=8, trials=2, cycles=3, seed=1)
    import ctypes
    isings = (ctypes.c_void_p * 1)(I.handle.value)
    ps = (S.Params * 1)(p)
    rs = (S.Result * 1)(S.Result(buf["sigma"].data_ptr(), None, buf["Is"].data_ptr(), None, None, None, None))
    rc = S.lib().ssqa_anneal_batch(1, isings, ps, rs, None, None)
    assert rc == S.ERR_INVALID_ARG and "DEVICE_PTRS" in S.last_error()
