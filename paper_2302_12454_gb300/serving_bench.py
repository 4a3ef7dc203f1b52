"""Served-latency benchmark for the continuous-batching server.

A seeded stream of GI requests (n uniform in [n_min, n_max], edge
probability uniform in [0.3, 0.7], R = 16 replicas, 32 trials, cycles drawn
from a set; request j's draws come from its own generator keyed by (seed, j))
is run four ways on one GPU:
  1. one at a time through ssqa_anneal (host buffers) on a bounded sample of
     the stream, the baseline;
  2. the same with the plain CUDA-core path on a smaller sample;
  3. closed loop through the server (a sample submitted at once) to measure
     its capacity in requests per second;
  4. open loop with Poisson arrivals at `load` x that capacity over the whole
     stream, recording the submit-to-completion latency of every request
     (p50 / p99).  Instances are built by a thread pool a bounded window
     ahead of their arrival and freed after completion, so that streams of
     thousands of requests (up to 2500 spins each) fit in memory.
Throughput is spin updates per second (N R trials cycles per request).
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time

import numpy as np


def request_spec(j, n_min, n_max, cycles_set, seed):
    """(n, p, cycles, seed) of request j (its own generator)."""
    rng = np.random.default_rng([seed, j])
    n = int(rng.integers(n_min, n_max + 1))
    p = float(rng.uniform(0.3, 0.7))
    cycles = int(rng.choice(cycles_set))
    return n, p, cycles, seed + j


def build_request(S, W, j, n_min, n_max, cycles_set, seed):
    n, p, cycles, s = request_spec(j, n_min, n_max, cycles_set, seed)
    a = S.gen_er_graph(n, W.p_q32(p), s)
    b, _ = S.permute_graph(a, s + 10007)
    I = S.Ising.gi(a, b)
    kw = dict(R=16, trials=32, cycles=cycles, seed=s, tau=100)
    return I, kw, n * n * 16 * 32 * cycles


def make_requests(S, W, count, n_min, n_max, cycles_set, seed=41, threads=8):
    with cf.ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda j: build_request(S, W, j, n_min, n_max, cycles_set, seed), range(count)))


def _one_at_a_time(S, reqs, **extra):
    t0 = time.perf_counter()
    for I, kw, _ in reqs:
        S.anneal(I, **kw, **extra)
    t = time.perf_counter() - t0
    return float(sum(u for _, _, u in reqs)) / t, t


def run(S, W, count=200, n_min=8, n_max=20, cycles_set=(1000, 2000, 5000), slots=32, load=0.8,
        budget=8 << 30, seed=41, plain_sample=16, seq_sample=200, capacity_sample=400, build_threads=8,
        lookahead=256):
    seq_n = max(1, min(seq_sample, count))
    cap_n = max(1, min(capacity_sample, count))
    head = make_requests(S, W, max(seq_n, cap_n), n_min, n_max, cycles_set, seed, build_threads)
    # warm the kernels and the first instances' device copies
    for I, kw, _ in head[: min(4, len(head))]:
        S.anneal(I, **{**kw, "cycles": 10})
    # 1-2. one at a time: tensor path where it applies, plain CUDA-core path
    seq_rate, t_seq = _one_at_a_time(S, head[:seq_n])
    plain_n = max(1, min(plain_sample, count))
    plain_rate, _ = _one_at_a_time(S, head[:plain_n], algo=S.ALGO_PLAIN)
    srv = S.Server(hbm_budget=budget, max_slots=slots)
    # 3. closed loop capacity on the first cap_n requests
    caps = head[:cap_n]
    t0 = time.perf_counter()
    tickets = [srv.submit(I, **kw) for I, kw, _ in caps]
    for t in tickets:
        srv.poll(t, timeout_ms=-1)
    t_closed = time.perf_counter() - t0
    capacity = cap_n / t_closed
    closed_rate = float(sum(u for _, _, u in caps)) / t_closed
    del caps, tickets
    head = head[: min(len(head), lookahead)]
    # 4. Poisson arrivals at load x capacity over the whole stream
    rate = load * capacity
    arrivals = np.cumsum(np.random.default_rng(seed + 1).exponential(1.0 / rate, size=count))
    pool = cf.ThreadPoolExecutor(build_threads)
    futs = collections.OrderedDict()
    for j in range(count):
        if j < len(head):
            f = cf.Future()
            f.set_result(head[j])
            futs[j] = f
        elif len(futs) < lookahead:
            futs[j] = pool.submit(build_request, S, W, j, n_min, n_max, cycles_set, seed)
        else:
            break
    head = None
    lat = np.zeros(count)
    done_t = np.zeros(count)
    updates = np.zeros(count)
    inflight = {}  # ticket -> (j, instance)
    lock = threading.Lock()
    cond = threading.Condition(lock)
    next_build = len(futs)
    start = time.perf_counter()
    submit_err = []

    def submitter():
        nonlocal next_build
        try:
            for j in range(count):
                with lock:
                    f = futs.pop(j)
                    if next_build < count:
                        futs[next_build] = pool.submit(build_request, S, W, next_build, n_min, n_max, cycles_set,
                                                       seed)
                        next_build += 1
                I, kw, u = f.result()
                d = start + arrivals[j] - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tk = srv.submit(I, **kw)
                with cond:
                    inflight[tk] = (j, I)
                    updates[j] = u
                    cond.notify()
        except Exception as e:  # reported by the main thread
            submit_err.append(e)
            with cond:
                cond.notify()

    th = threading.Thread(target=submitter)
    th.start()
    finished = 0
    while finished < count and not submit_err:
        with cond:
            if not inflight:
                cond.wait(0.01)
            items = list(inflight.items())
        for tk, (j, _) in items:
            r = srv.poll(tk, timeout_ms=0)
            if r is not None:
                lat[j] = r[1]
                done_t[j] = time.perf_counter()
                finished += 1
                with cond:
                    inflight.pop(tk)  # drops the instance
        time.sleep(0.0005)
    th.join()
    pool.shutdown()
    if submit_err:
        raise submit_err[0]
    t_open = float(done_t.max() - start)
    srv.close()
    return {
        "requests": count, "n_range": [n_min, n_max], "p_range": [0.3, 0.7], "cycles_set": list(cycles_set), "R": 16,
        "trials": 32, "slots": slots, "load": load,
        "one_at_a_time": {"value": seq_rate, "unit": "spin-updates/s", "seconds": t_seq, "requests": seq_n},
        "served_closed_loop": {"value": closed_rate, "unit": "spin-updates/s", "seconds": t_closed,
                               "requests": cap_n, "requests_per_s": capacity},
        "served_poisson": {"value": float(updates.sum()) / t_open, "unit": "spin-updates/s", "seconds": t_open,
                           "requests": count, "arrival_rate_per_s": rate,
                           "p50_ms": float(np.percentile(lat, 50) * 1e3),
                           "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)},
        "speedup_vs_one_at_a_time": closed_rate / seq_rate,
        "plain_one_at_a_time": {"value": plain_rate, "unit": "spin-updates/s", "requests": plain_n},
        "speedup_vs_plain_one_at_a_time": closed_rate / plain_rate,
    }
