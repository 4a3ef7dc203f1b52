"""Served-latency benchmark for the continuous-batching server.

A seeded stream of GI requests (n uniform in [n_min, n_max], edge
probability uniform in [0.3, 0.7], R = 16 replicas, 32 trials, cycles drawn
from a set) is run three ways on one GPU:
  1. one at a time through ssqa_anneal (host buffers), the baseline, also
     with the plain CUDA-core path on a sample of the requests;
  2. closed loop through the server (all submitted at once) to measure its
     capacity in requests per second;
  3. open loop with Poisson arrivals at `load` x that capacity, recording the
     submit-to-completion latency of every request (p50 / p99).
Throughput is spin updates per second (N R trials cycles per request).
"""
from __future__ import annotations

import threading
import time

import numpy as np


def make_requests(S, W, count, n_min, n_max, cycles_set, seed=41):
    rng = np.random.default_rng(seed)
    reqs = []
    for j in range(count):
        n = int(rng.integers(n_min, n_max + 1))
        p = float(rng.uniform(0.3, 0.7))
        a = S.gen_er_graph(n, W.p_q32(p), seed + j)
        b, _ = S.permute_graph(a, seed + 10007 + j)
        I = S.Ising.gi(a, b)
        kw = dict(R=16, trials=32, cycles=int(rng.choice(cycles_set)), seed=seed + j, tau=100)
        reqs.append((I, kw, n * n * 16 * 32 * kw["cycles"]))
    return reqs


def run(S, W, count=200, n_min=8, n_max=20, cycles_set=(1000, 2000, 5000), slots=32, load=0.8,
        budget=8 << 30, seed=41, plain_sample=16):
    reqs = make_requests(S, W, count, n_min, n_max, cycles_set, seed)
    total_updates = float(sum(u for _, _, u in reqs))
    # warm every instance's device copy and the kernels
    for I, kw, _ in reqs[: min(4, count)]:
        S.anneal(I, **{**kw, "cycles": 10})
    # 1. one at a time (tensor path where it applies), and the plain CUDA-core
    #    path one at a time on the first `plain_sample` requests
    t0 = time.perf_counter()
    for I, kw, _ in reqs:
        S.anneal(I, **kw)
    t_seq = time.perf_counter() - t0
    ps = reqs[: max(1, min(plain_sample, count))]
    t0 = time.perf_counter()
    for I, kw, _ in ps:
        S.anneal(I, algo=S.ALGO_PLAIN, **kw)
    t_plain = time.perf_counter() - t0
    plain_rate = float(sum(u for _, _, u in ps)) / t_plain
    srv = S.Server(hbm_budget=budget, max_slots=slots)
    # 2. closed loop capacity
    t0 = time.perf_counter()
    tickets = [srv.submit(I, **kw) for I, kw, _ in reqs]
    for t in tickets:
        srv.poll(t, timeout_ms=-1)
    t_closed = time.perf_counter() - t0
    capacity = count / t_closed
    # 3. Poisson arrivals at `load` x capacity
    rate = load * capacity
    gaps = np.random.default_rng(seed + 1).exponential(1.0 / rate, size=count)
    arrivals = np.cumsum(gaps)
    lat = [None] * count
    tickets = [None] * count
    done_t = [0.0] * count
    lock = threading.Lock()
    start = time.perf_counter()

    def submitter():
        for j, (I, kw, _) in enumerate(reqs):
            d = start + arrivals[j] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tk = srv.submit(I, **kw)
            with lock:
                tickets[j] = tk

    th = threading.Thread(target=submitter)
    th.start()
    remaining = set(range(count))
    while remaining:
        for j in list(remaining):
            with lock:
                tk = tickets[j]
            if tk is None:
                continue
            r = srv.poll(tk, timeout_ms=0)
            if r is not None:
                lat[j] = r[1]
                done_t[j] = time.perf_counter()
                remaining.discard(j)
        time.sleep(0.0005)
    th.join()
    t_open = max(done_t) - start
    srv.close()
    lat = np.array(lat)
    return {
        "requests": count, "n_range": [n_min, n_max], "cycles_set": list(cycles_set), "R": 16, "trials": 32,
        "slots": slots, "load": load,
        "one_at_a_time": {"value": total_updates / t_seq, "unit": "spin-updates/s", "seconds": t_seq},
        "served_closed_loop": {"value": total_updates / t_closed, "unit": "spin-updates/s", "seconds": t_closed,
                               "requests_per_s": capacity},
        "served_poisson": {"value": total_updates / t_open, "unit": "spin-updates/s", "seconds": t_open,
                           "arrival_rate_per_s": rate, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                           "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)},
        "speedup_vs_one_at_a_time": t_seq / t_closed,
        "plain_one_at_a_time": {"value": plain_rate, "unit": "spin-updates/s", "requests": len(ps)},
        "speedup_vs_plain_one_at_a_time": (total_updates / t_closed) / plain_rate,
    }
