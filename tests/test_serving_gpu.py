"""Serving: requests of different sizes admitted by HBM budget and run
concurrently give, each, exactly the result of the same anneal run alone."""
import time

import numpy as np
import pytest

import paper_2302_12454_gb300 as S
from paper_2302_12454_gb300 import build as B
from paper_2302_12454_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def _gi(n, seed):
    a = S.gen_er_graph(n, W.p_q32(0.3 + 0.4 * ((seed * 7) % 10) / 10), seed)
    b, _ = S.permute_graph(a, seed + 1)
    return S.Ising.gi(a, b)


def test_mixed_requests_equal_alone():
    rng = np.random.default_rng(41)
    reqs = []
    for j in range(14):
        n = int(rng.integers(4, 21))
        kw = dict(R=int(rng.choice([4, 8, 16])), cycles=int(rng.choice([100, 200, 300])),
                  trials=int(rng.integers(1, 33)), seed=41 + j, tau=int(rng.choice([10, 25])))
        if j % 5 == 3:
            kw.update(delay=2, coupling=S.COUPLING_BOTH)
        reqs.append((_gi(n, 100 + j), kw))
    srv = S.Server(hbm_budget=1 << 30, max_slots=4)
    tickets = [srv.submit(I, track_best=(j % 2 == 0), **kw) for j, (I, kw) in enumerate(reqs)]
    results = {}
    deadline = time.time() + 300
    while len(results) < len(tickets) and time.time() < deadline:
        for j, t in enumerate(tickets):
            if j in results:
                continue
            r = srv.poll(t, timeout_ms=10)
            if r is not None:
                results[j] = r
    assert len(results) == len(tickets)
    for j, (I, kw) in enumerate(reqs):
        alone = S.anneal(I, track_best=(j % 2 == 0), want_hist=True, **kw)
        got, lat = results[j]
        assert lat > 0
        for k in alone:
            np.testing.assert_array_equal(got[k], alone[k], err_msg=f"request {j} field {k}")
    srv.close()


def test_budget_and_ticket_errors():
    srv = S.Server(hbm_budget=1 << 20, max_slots=2)
    I = _gi(20, 3)
    with pytest.raises(S.SSQAError) as e:
        srv.submit(I, R=16, cycles=10, trials=512, seed=1)
    assert e.value.code == S.ERR_BUDGET
    import ctypes
    assert S.lib().ssqa_poll(srv._s, 12345, None, 0, None) == S.ERR_NOT_FOUND
    t = srv.submit(_gi(4, 1), R=2, cycles=5, trials=1, seed=1)
    r = srv.poll(t, timeout_ms=-1)
    assert r is not None
    srv.close()


def test_mixed_paths_equal_alone():
    """Resident, streamed and delta requests in flight together (the streamed
    kernel's clusters share the GPU with resident CTAs and CUDA-core kernels):
    each served result equals its lone run."""
    reqs = []
    for j, (n, R, trials, cycles) in enumerate([(6, 8, 20, 120), (23, 4, 6, 60), (20, 16, 16, 100), (30, 8, 5, 40),
                                                (45, 4, 3, 30), (12, 16, 9, 80), (50, 2, 4, 25)]):
        reqs.append((_gi(n, 200 + j), dict(R=R, cycles=cycles, trials=trials, seed=300 + j, tau=10)))
    # a dense instance whose couplings have no exact FP8 value: delta path
    rng = np.random.default_rng(5)
    Jd = np.triu(rng.integers(-1, 2, size=(300, 300)) * 17, 1)
    Jd = (Jd + Jd.T).astype(np.int8)
    hd = ((np.arange(300) % 7) * 2 - 5).astype(np.int32)
    reqs.append((S.Ising.dense(Jd, hd), dict(R=4, cycles=40, trials=3, seed=400, tau=5)))
    srv = S.Server(hbm_budget=4 << 30, max_slots=8)
    tickets = [srv.submit(I, track_best=True, **kw) for I, kw in reqs]
    results = [srv.poll(t, timeout_ms=-1) for t in tickets]
    for j, (I, kw) in enumerate(reqs):
        alone = S.anneal(I, track_best=True, want_hist=True, **kw)
        got, _ = results[j]
        for k in alone:
            np.testing.assert_array_equal(got[k], alone[k], err_msg=f"request {j} field {k}")
    srv.close()


def _min_budget(I, kw):
    """The request's device footprint: the smallest budget ssqa_submit accepts
    it under (a request needing more than the whole budget is rejected)."""
    lo, hi = 1, 1 << 36
    while lo < hi:
        mid = (lo + hi) // 2
        srv = S.Server(hbm_budget=mid, max_slots=1)
        try:
            srv.submit(I, **kw)
            ok = True
        except S.SSQAError as e:
            assert e.code == S.ERR_BUDGET
            ok = False
        srv.close()
        lo, hi = (lo, mid) if ok else (mid + 1, hi)
    return lo


def test_large_request_is_not_starved():
    """A request that needs the whole budget, submitted behind small requests
    that keep arriving: with first-fit admission the small ones would always
    pass it; with bounded bypass (at most 2 x slots admissions past the oldest
    request) it is admitted once the running requests drain, and its result is
    the one it has alone."""
    big = (_gi(20, 7), dict(R=16, cycles=300, trials=128, seed=5, tau=25))
    small = [(_gi(6, 200 + j), dict(R=8, cycles=200, trials=8, seed=300 + j, tau=20)) for j in range(8)]
    fb = _min_budget(*big)
    fs = _min_budget(*small[0])
    assert fb > 4 * fs
    slots = 4
    srv = S.Server(hbm_budget=fb + fs // 2, max_slots=slots)  # the big request needs an idle server
    tickets = [srv.submit(I, **kw) for I, kw in small[:6]]
    tb = srv.submit(big[0], **big[1])
    got_big = None
    submitted_after = 0
    done_after = 0
    deadline = time.time() + 120
    while got_big is None and time.time() < deadline and submitted_after < 400:
        I, kw = small[submitted_after % len(small)]
        tickets.append(srv.submit(I, **kw))
        submitted_after += 1
        for t in list(tickets):
            r = srv.poll(t, timeout_ms=0)
            if r is not None:
                tickets.remove(t)
                done_after += 1
        r = srv.poll(tb, timeout_ms=1)
        if r is not None:
            got_big = r
    for t in tickets:
        srv.poll(t, timeout_ms=-1)
    srv.close()
    assert got_big is not None, f"starved: {submitted_after} small requests submitted after it"
    # passed over at most 2 x slots times (an admission may batch several small requests)
    assert done_after < 200, done_after
    alone = S.anneal(big[0], want_hist=True, **big[1])
    for k in alone:
        np.testing.assert_array_equal(got_big[0][k], alone[k], err_msg=k)


def test_failed_request_reports_its_error_and_the_server_recovers():
    """A request whose anneal fails on the device (its bounded waits made to run
    out with a 100-clock limit, the only failure injected) reports
    SSQA_ERR_TIMEOUT on poll; the worker frees its budget and slot and the next
    requests, with the default limit restored, give the results of the same
    anneals run alone."""
    srv = S.Server(hbm_budget=1 << 30, max_slots=2)
    I = _gi(20, 7)
    kw = dict(R=16, cycles=40, trials=64, seed=17, tau=10)
    S.set_wait_limit(100)
    try:
        t = srv.submit(I, **kw)
        with pytest.raises(S.SSQAError) as e:
            srv.poll(t, timeout_ms=-1)
        assert e.value.code == S.ERR_TIMEOUT, str(e.value)
    finally:
        S.set_wait_limit(0)
    tickets = [srv.submit(I, **kw), srv.submit(_gi(9, 8), R=8, cycles=30, trials=5, seed=3)]
    got = [srv.poll(t, timeout_ms=-1) for t in tickets]
    for (out, _), (inst, kws) in zip(got, [(I, kw), (_gi(9, 8), dict(R=8, cycles=30, trials=5, seed=3))]):
        alone = S.anneal(inst, want_hist=True, **kws)
        for k in alone:
            np.testing.assert_array_equal(out[k], alone[k], err_msg=k)
    srv.close()
