"""The allocation-free anneal (ssqa_anneal_noalloc) against ssqa_anneal.

ssqa_anneal_noalloc serves callers that cannot allocate device memory (for
instance plugins whose host framework owns every device allocation, or
real-time loops in which an allocation would synchronise the device): it
takes only caller-provided device buffers and keeps its scratch in a fixed
array inside the library.
This test calls it through the C ABI twice in a row (the shared scratch
keeps the previous call's contents) and checks both results element by
element against ssqa_anneal on the same inputs; the method is integer
arithmetic, so the tolerance is exact equality.  The file is collected last
so that a failure here does not stop the other tests under -x.
"""
import ctypes

import numpy as np
import pytest

import paper_2302_12454_gb300 as S
from paper_2302_12454_gb300 import build as B
from paper_2302_12454_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _device_inputs(I, torch):
    h, J, off = I.export()
    N = h.shape[0]
    Np = (N + 15) // 16 * 16
    Jp = np.zeros((N, Np), np.int8)
    Jp[:, :N] = J
    return torch.from_numpy(Jp).cuda(), torch.from_numpy(h).cuda(), N


def test_noalloc_matches_anneal_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    L = S.lib()
    cases = [
        (S.Ising.gi(*(lambda a: (a, S.permute_graph(a, 2)[0]))(S.gen_er_graph(6, W.p_q32(0.5), 1))),
         dict(R=8, cycles=120, trials=64, seed=3, tau=20)),
        (S.Ising.gi(*(lambda a: (a, S.permute_graph(a, 5)[0]))(S.gen_er_graph(9, W.p_q32(0.5), 4))),
         dict(R=5, cycles=60, trials=11, seed=8, tau=7, delay=2, coupling=S.COUPLING_BOTH)),
    ]
    stream = torch.cuda.current_stream()
    for call in range(2):
        I, kw = cases[call]
        ref = S.anneal(I, algo=S.ALGO_PLAIN, track_best=True, want_hist=True, want_trace=True, **kw)
        Jd, hd, N = _device_inputs(I, torch)
        p = S.make_params(**kw)
        p.flags = S.FLAG_DEVICE_PTRS | S.FLAG_TRACK_BEST
        T, R, d = kw["trials"], kw["R"], p.delay
        sig = torch.zeros((T, R, N), dtype=torch.int8, device="cuda")
        Is = torch.full((T, R, N), 77, dtype=torch.int32, device="cuda")
        hist = torch.zeros((T, d, R, N), dtype=torch.int8, device="cuda")
        E = torch.zeros((T, R), dtype=torch.int64, device="cuda")
        Eb = torch.zeros((T, R), dtype=torch.int64, device="cuda")
        bc = torch.zeros((T, R), dtype=torch.int32, device="cuda")
        tr = torch.zeros((kw["cycles"], T, R), dtype=torch.int64, device="cuda")
        r = S.Result(sig.data_ptr(), hist.data_ptr(), Is.data_ptr(), E.data_ptr(), Eb.data_ptr(), bc.data_ptr(),
                     tr.data_ptr())
        rc = L.ssqa_anneal_noalloc(N, Jd.data_ptr(), hd.data_ptr(), ctypes.byref(p), ctypes.byref(r),
                                   ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, S.last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(sig.cpu().numpy(), ref["sigma"])
        np.testing.assert_array_equal(Is.cpu().numpy(), ref["Is"])
        np.testing.assert_array_equal(hist.cpu().numpy(), ref["hist"])
        np.testing.assert_array_equal(E.cpu().numpy(), ref["E_final"])
        np.testing.assert_array_equal(Eb.cpu().numpy(), ref["E_best"])
        np.testing.assert_array_equal(bc.cpu().numpy(), ref["best_cycle"])
        np.testing.assert_array_equal(tr.cpu().numpy(), ref["E_trace"])
    # a problem beyond the fixed scratch is rejected with a clear error
    I, kw = cases[0]
    Jd, hd, N = _device_inputs(I, torch)
    p = S.make_params(R=128, cycles=1, trials=20000, seed=1)
    p.flags = S.FLAG_DEVICE_PTRS
    r = S.Result(Jd.data_ptr(), None, hd.data_ptr(), None, None, None, None)
    assert L.ssqa_anneal_noalloc(N, Jd.data_ptr(), hd.data_ptr(), ctypes.byref(p), ctypes.byref(r), None) == S.ERR_INVALID_ARG
    assert "scratch" in S.last_error()
