"""Benchmark: SSQA spin-updates/s on the batched GI workload (N = 400 spins,
R = 16 replicas, 2000 cycles, 1024 trials per GPU), one JSON line on stdout.

A step is one full anneal of the whole batch (every cycle of Eq. 6 for all
spins x replicas x trials) through ssqa_anneal with device-resident buffers.
`e2e` repeats the step through the same C ABI with host buffers (instance
upload, anneal, result download inside the timed region).  `--impl
reference` times the C oracle on the host cores on a bounded sample of the
same workload.  Multi-GPU runs shard trials across ranks (weak scaling, no
collective on the data path).
"""
from __future__ import annotations

import argparse
import datetime
import json
import math
import multiprocessing as mp
import os
import platform
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "batched_gi_n20"
PLAIN_CYCLES = 200


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------ oracle (CPU)
def _oracle_trial(args):
    h, J, kw, tr = args
    from oracle import oracle as O

    t0 = time.perf_counter()
    O.anneal(h, J, trial_offset=tr, **kw)
    return time.perf_counter() - t0


def _oracle_warm(_):
    from oracle import oracle as O

    O.lib()
    return os.getpid()


def host_info():
    """Core count and CPU model of this host (for the CPU-side lines)."""
    model = platform.processor() or ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() == "Model name" and v.strip():
                return {"cpu_count": os.cpu_count(), "cpu_model": v.strip(), "machine": platform.machine()}
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k, _, v = ln.partition(":")
                if k.strip() in ("model name", "Model", "CPU part") and v.strip():
                    model = v.strip() if k.strip() != "CPU part" else f"{platform.machine()} CPU part {v.strip()}"
                    break
    except OSError:
        pass
    return {"cpu_count": os.cpu_count(), "cpu_model": model or platform.machine(), "machine": platform.machine()}


class OraclePool:
    """Single-threaded oracle processes, one per core, started (spawn) and
    warmed once, so that timed maps measure the oracle and not process start-up."""

    def __init__(self, cores):
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores) if cores > 1 else None
        if self.pool is not None:
            self.pool.map(_oracle_warm, range(cores))
        else:
            _oracle_warm(0)

    def map(self, jobs):
        if self.pool is not None:
            return self.pool.map(_oracle_trial, jobs, chunksize=1)
        return [_oracle_trial(j) for j in jobs]

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None


def oracle_rate(pool, h, J, cfg, cycles, ntrials):
    """Spin-updates/s of the oracle: `ntrials` single-trial anneals of
    `cycles` cycles spread over the pool's worker processes."""
    kw = dict(R=cfg["R"], cycles=cycles, trials=1, seed=cfg["seed"], tau=cfg["tau"])
    jobs = [(h, J, kw, tr) for tr in range(ntrials)]
    t0 = time.perf_counter()
    pool.map(jobs)
    wall = time.perf_counter() - t0
    return h.shape[0] * cfg["R"] * cycles * ntrials / wall, wall


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self, dev=0):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9 or f[0] != str(dev):
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons)}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- our arm
def streamed_shape(desc):
    """The launch shape in a streamed-path plan description (`ssqa_plan`), and
    the operand bytes that launch moves into the SMs per cycle: every (column
    group, 256-spin chunk) pair streams its A blocks (4 KB per K-block) and each
    CTA the chunk's B blocks (8 KB per K-block; two groups per CTA share them in
    dual mode).  None for the other paths."""
    shape = {k: int(v) for k, v in re.findall(r"(groups|KB|NCH|CS|dual|CTAs) (\d+)", desc)}
    if not shape:
        return None
    g, kb, nch, dual = (shape[k] for k in ("groups", "KB", "NCH", "dual"))
    ctas_per_rank = (g + 1) // 2 if dual else g
    return shape, kb * nch * (g * 4096 + ctas_per_rank * 8192)


def large_workloads(S, W, torch, stream, pool=None):
    """The large configurations (GI n = 50 at p = 0.5, 0.3 and 0.7, SK N =
    8192; one anneal each, default path = the streamed tensor kernel), timed
    with CUDA events after a warm-up call that uploads the instance.  Informational: the headline is the batched N = 400
    workload.  With `cores`, also the oracle's rate on a bounded sample of the
    same instance (one trial per core, a few cycles), per spin update."""
    res = {}
    for name in ("large_gi_n50", "large_gi_n50_p03", "large_gi_n50_p07", "sk_n8192"):
        cfg = dict(W.CONFIGS[name])
        if cfg["kind"] == "gi":
            a = S.gen_er_graph(cfg["n"], W.p_q32(cfg["p"]), cfg["graph_seed"])
            b, _ = S.permute_graph(a, cfg["perm_seed"])
            I = S.Ising.gi(a, b)
        else:
            I = S.Ising.dense(W.sk_couplings(cfg["N"], cfg["j_seed"]), np.zeros(cfg["N"], np.int32))
        h, J, off = I.export()
        N, R, T, C = h.shape[0], cfg["R"], cfg["trials"], cfg["cycles"]
        dev = torch.device("cuda")
        sig = torch.empty((T, R, N), dtype=torch.int8, device=dev)
        Is = torch.empty((T, R, N), dtype=torch.int32, device=dev)
        E = torch.empty((T, R), dtype=torch.int64, device=dev)
        warm = S.make_params(R=R, cycles=10, trials=T, seed=cfg["seed"], tau=cfg["tau"], algo=S.ALGO_AUTO)
        S.anneal_device(I, warm, sig, Is, e_final=E, stream=stream)
        p = S.make_params(R=R, cycles=C, trials=T, seed=cfg["seed"], tau=cfg["tau"], algo=S.ALGO_AUTO)
        torch.cuda.synchronize()
        # two timed anneals (mean), SM clocks sampled meanwhile
        clk = ClockSampler(os.path.join(tempfile.gettempdir(), f"ssqa_clocks_{name}.csv"))
        ts = []
        with clk:
            for _ in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                S.anneal_device(I, p, sig, Is, e_final=E, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
        t = float(np.mean(ts))
        algo, desc = S.plan(I, R=R, cycles=C, trials=T, seed=cfg["seed"], tau=cfg["tau"])
        tflops = 2.0 * N * N * R * T * C / t / 1e12
        r = {"N": N, "R": R, "trials": T, "cycles": C, "seconds": t, "runs": ts, "value": N * R * T * C / t,
             "unit": "spin-updates/s", "path": desc, "tflops": tflops, "clocks": clk.summary()}
        sh = streamed_shape(desc)
        if sh:
            shape, per_cycle = sh
            # one launch of a quarter second or more at full tensor load runs
            # under the power cap, so the sustained figure is the peak
            peaks, src = _peaks()
            fp8 = 2.0 * peaks["bf16_tflops_sustained"]
            fp8b = 2.0 * peaks["bf16_tflops"]
            r["roofline"] = {"bound": "tensor", "achieved": tflops, "peak": fp8, "unit": "TFLOP/s",
                             "frac": tflops / fp8, "frac_of_burst": tflops / fp8b, "traffic": None,
                             "peak_source": f"{src}: 2 x bf16_tflops_sustained (FP8 dense / BF16 dense = 2); "
                                            f"burst 2 x bf16_tflops = {fp8b:.1f}",
                             "operand_bytes_per_cycle": per_cycle,
                             "operand_TBps_into_SMs": per_cycle * C / t / 1e12,
                             "shape": shape}
        if cfg["kind"] == "gi":
            r["p_s"] = float((E.min(dim=1).values.cpu().numpy() == -off).mean())
        if pool is not None:
            oc = 2 if cfg["kind"] == "gi" else 1
            rate, wall = oracle_rate(pool, h.astype(np.int64), J.astype(np.int64), cfg, oc, pool.cores)
            r["oracle"] = {"value": rate, "unit": "spin-updates/s", "cores": pool.cores,
                           "sample": f"{pool.cores} trials x {oc} cycles ({wall:.1f} s)", "ratio": r["value"] / rate}
        res[name] = r
        del I
    return res


def row_timings(S, torch, stream, I, cfg, sigma, Is, E, base_ms):
    """The rows the headline step leaves out, timed on the same instance and
    batch (CUDA events, best of three after a warm-up call):
    - energy tracking: lowest energy and its cycle per replica, from the
      energy fused into every cycle's epilogue;
    - energy trace: the same plus every replica's energy after every cycle
      ([cycles][trials * R] int64 written to device memory);
    - SSA mode: R = 1 with the I0 schedule (I0' = 12 .. 192 doubling every 10
      cycles, n_rnd' = 12, no J_perp), one column per trial, same column count;
    - ssqa_energy on the final spins of the headline step (every column),
      checked against the anneal's own final energies."""
    import ctypes

    N, R, T, C = I.N, cfg["R"], cfg["trials"], cfg["cycles"]
    cols = T * R
    dev = sigma.device

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best

    def row(ms, updates, what):
        return {"ms": ms, "value": updates / (ms / 1e3), "unit": "spin-updates/s", "vs_headline_step": ms / base_ms,
                "what": what}

    out = {}
    Eb = torch.empty((T, R), dtype=torch.int64, device=dev)
    bc = torch.empty((T, R), dtype=torch.int32, device=dev)
    pt = S.make_params(R=R, cycles=C, trials=T, seed=cfg["seed"], tau=cfg["tau"], algo=S.ALGO_TENSOR)
    ms = timed(lambda: S.anneal_device(I, pt, sigma, Is, e_final=E, e_best=Eb, best_cycle=bc, stream=stream))
    out["energy_tracking"] = row(ms, N * cols * C, "headline anneal + per-cycle energy, best energy and cycle")
    tr = torch.empty((C, cols), dtype=torch.int64, device=dev)
    ms = timed(lambda: S.anneal_device(I, pt, sigma, Is, e_final=E, e_best=Eb, best_cycle=bc, stream=stream,
                                       e_trace=tr))
    out["energy_trace"] = row(ms, N * cols * C, f"as energy_tracking + trace of {C} x {cols} energies "
                                                f"({tr.numel() * 8 / 1e6:.0f} MB)")
    assert torch.equal(tr.min(dim=0).values.view(T, R), Eb)
    del tr
    ps = S.make_params(R=1, cycles=C, trials=cols, seed=cfg["seed"], tau=10, beta=3, jperp_min=0, jperp_max=0,
                       I0=12, i0_max=192, i0_mult=2, i0_tau=10, n_rnd=12, algo=S.ALGO_TENSOR)
    s1, i1, e1 = sigma.view(cols, 1, N), Is.view(cols, 1, N), E.view(cols, 1)
    ms = timed(lambda: S.anneal_device(I, ps, s1, i1, e_final=e1, stream=stream))
    out["ssa"] = row(ms, N * cols * C, f"SSA (R = 1, I0 schedule), {cols} trials x {C} cycles")
    # final spins and energies of one headline step, then ssqa_energy on them
    S.anneal_device(I, pt, sigma, Is, e_final=E, e_best=Eb, best_cycle=bc, stream=stream)
    E2 = torch.empty(cols, dtype=torch.int64, device=dev)
    h = ctypes.c_void_p(stream.cuda_stream)
    call = lambda: S._check(S.lib().ssqa_energy(I.handle, ctypes.c_void_p(sigma.data_ptr()), cols,  # noqa: E731
                                                 ctypes.c_void_p(E2.data_ptr()), S.FLAG_DEVICE_PTRS, h), "energy")
    ms = timed(call)
    assert torch.equal(E2.view(T, R), E)
    out["energy_call"] = {"ms": ms, "value": cols / (ms / 1e3), "unit": "configurations/s",
                          "what": f"ssqa_energy of {cols} spin vectors of N = {N} (device pointers)"}
    return out


def run_ours(args, rank, world):
    import torch

    import paper_2302_12454_gb300 as S
    from paper_2302_12454_gb300 import build as B
    from paper_2302_12454_gb300 import workloads as W

    B.build()
    cfg = dict(W.CONFIGS[WORKLOAD])
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dist = None
    if world > 1:
        import torch.distributed as dist

        # a rank that dies or never joins ends the others' next collective with an
        # error after this bound instead of holding their GPUs
        dist.init_process_group("nccl", timeout=datetime.timedelta(minutes=10))
    n, R, cycles, trials = cfg["n"], cfg["R"], cfg["cycles"], cfg["trials"]
    a = S.gen_er_graph(n, W.p_q32(cfg["p"]), cfg["graph_seed"])
    b, _ = S.permute_graph(a, cfg["perm_seed"])
    I = S.Ising.gi(a, b)
    h, J, off = I.export()
    N = n * n
    cols = trials * R
    offset = rank * trials  # weak scaling: each rank anneals its own trial range
    params = S.make_params(R=R, cycles=cycles, trials=trials, seed=cfg["seed"], tau=cfg["tau"],
                           trial_offset=offset, algo=S.ALGO_TENSOR)
    dev = torch.device("cuda")
    sigma = torch.empty((trials, R, N), dtype=torch.int8, device=dev)
    Is = torch.empty((trials, R, N), dtype=torch.int32, device=dev)
    E = torch.empty((trials, R), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        S.anneal_device(I, params, sigma, Is, e_final=E, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(args.clocks_csv.replace("{rank}", str(rank)) if args.clocks_csv
                       else os.path.join(tempfile.gettempdir(), f"ssqa_clocks_r{rank}.csv"))
    wall0 = time.perf_counter()
    with clk:
        for k in range(args.steps):
            flush.fill_(k & 0xFF)  # L2 flush between timed steps (outside the events)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    t_total = sum(ms) / 1e3
    if dist:
        tt = torch.tensor([t_total], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_total = float(tt.item())
    updates_per_step = N * R * cycles * trials
    value = updates_per_step * args.steps * world / t_total
    ms_per_step = t_total / args.steps * 1e3

    # results of the last step: success probability and time to solution
    e_min = E.min(dim=1).values.cpu().numpy()
    p_s = float((e_min == -off).mean())
    t_trial = t_total / args.steps / trials
    tts = S.tts(t_trial, p_s, 0.99)

    # end to end through the C ABI with host buffers: instance upload,
    # anneal, result download inside the timed region (pinned host memory)
    hJ = torch.from_numpy(J).pin_memory().numpy()
    hh = torch.from_numpy(h).pin_memory().numpy()
    # result buffers: pinned host memory, allocated once and reused by every
    # call; the step's result is the final spins and energies (the counters
    # Is are only needed to resume and are not read back)
    hout = {"sigma": torch.empty((trials, R, N), dtype=torch.int8, pin_memory=True).numpy(),
            "E_final": torch.empty((trials, R), dtype=torch.int64, pin_memory=True).numpy()}
    e2e_t = []
    for k in range(max(1, min(args.steps, 3)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ik = S.Ising.dense(hJ, hh, off)
        outk = S.anneal(Ik, R=R, cycles=cycles, trials=trials, seed=cfg["seed"], tau=cfg["tau"],
                        trial_offset=offset, algo=S.ALGO_TENSOR, want_state=False, out=hout)
        e2e_t.append(time.perf_counter() - t0)
        del Ik
    e2e_t = e2e_t[1:]  # first call includes one-time context and allocator set-up
    e2e_val = updates_per_step * world / float(np.mean(e2e_t))
    h2d = J.nbytes + h.nbytes  # the step's inputs: couplings and biases (device images derive from them)
    d2h = outk["sigma"].nbytes + outk["E_final"].nbytes
    assert np.array_equal(outk["E_final"].min(axis=1) == -off, e_min == -off)

    # plain GPU path (one kernel launch per cycle, CUDA-core dot products) on
    # the same instance and batch: its per-update rate over the first
    # PLAIN_CYCLES cycles (each cycle costs the same, so the rate carries over)
    Ip = S.Ising.gi(a, b)
    pp = S.make_params(R=R, cycles=PLAIN_CYCLES, trials=trials, seed=cfg["seed"], tau=cfg["tau"],
                       trial_offset=offset, algo=S.ALGO_PLAIN)
    S.anneal_device(Ip, pp, sigma, Is, e_final=E, stream=stream)  # warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    S.anneal_device(Ip, pp, sigma, Is, e_final=E, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_s = e0.elapsed_time(e1) / 1e3
    plain_val = N * R * PLAIN_CYCLES * trials / plain_s

    peaks, src = _peaks()
    fp8_peak = 2.0 * peaks["bf16_tflops"]  # FP8 dense = 2x BF16 (nominal 4.5 / 2.25 PF)
    flop = 2.0 * N * updates_per_step  # 2N FLOP (N MACs) per spin update
    achieved = flop / (t_total / args.steps) / 1e12
    traffic = None
    prof = os.path.join(ROOT, "profiles", "dram_traffic_per_launch.json")
    if os.path.exists(prof):
        try:
            traffic = json.load(open(prof)).get("ssqa_tc_kernel_batched_gi_n20", {}).get("bytes")
        except Exception:
            traffic = None
    out = {
        "metric": "spin-updates/sec",
        "value": value,
        "unit": "spin-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "fp8",
        "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: GI n={n} (N={N} spins), ER p=0.5, planted permutation; R={R}, "
                               f"{cycles} cycles, {trials} trials per GPU, one persistent launch",
                   "N": N, "R": R, "cycles": cycles, "trials_per_gpu": trials,
                   "l2": "flushed between timed steps (256 MiB write outside the timed events)"},
        "gpu_launches": args.steps,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": fp8_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp8_peak, "traffic": traffic,
                     "peak_source": f"{src}: 2 x bf16_tflops (FP8 dense / BF16 dense = 2)"},
        "e2e": {"value": e2e_val, "unit": "spin-updates/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "tts_s": tts, "p_s": p_s, "t_per_trial_s": t_trial,
        "plain_gpu": {"value": plain_val, "unit": "spin-updates/s", "ratio": value / world / plain_val,
                      "note": f"one kernel launch per cycle, CUDA cores (dp4a), same instance and batch, "
                              f"first {PLAIN_CYCLES} cycles, 1 GPU"},
        "wall_s": wall,
    }
    if rank == 0:
        out["clocks"] = clk.summary(int(os.environ.get("LOCAL_RANK", 0)))
        # served latency: a seeded Poisson stream of GI requests with the
        # serving workload's distributions (n in [8, 50], i.e. 64 to 2500
        # spins, p in [0.3, 0.7], R = 16, 32 trials, cycles in {1000, 2000,
        # 5000}); 400 requests, a bounded sample of its 10 000
        from paper_2302_12454_gb300 import serving_bench as SB

        out["served"] = SB.run(S, W, count=400, n_min=8, n_max=50, cycles_set=(1000, 2000, 5000), slots=32,
                               plain_sample=8, seq_sample=100, capacity_sample=200)
        out["rows"] = row_timings(S, torch, stream, I, cfg, sigma, Is, E, ms_per_step)
        pool = None if args.no_cpu_baseline else OraclePool(min(64, os.cpu_count() or 1))
        if not args.no_large:
            out["large_workloads"] = large_workloads(S, W, torch, stream, pool)
        if pool is not None:
            cores = pool.cores
            rate, cwall = oracle_rate(pool, h.astype(np.int64), J.astype(np.int64), cfg, cycles, 2 * cores)
            pool1 = OraclePool(1)
            rate1, wall1 = oracle_rate(pool1, h.astype(np.int64), J.astype(np.int64), cfg, 500, 1)
            pool.close()
            out["cpu_baseline"] = {"value": rate, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                                   "sample": f"{2 * cores} trials x {cycles} cycles of the same workload, one "
                                             f"single-threaded oracle process per core ({cwall:.1f} s)",
                                   "host": host_info(),
                                   "single_core": {"value": rate1, "sample": f"1 trial x 500 cycles ({wall1:.1f} s)"}}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2302_12454_gb300 import workloads as W
    from oracle import oracle as O

    O.build()
    cfg = dict(W.CONFIGS[WORKLOAD])
    a = O.gen_er_graph(cfg["n"], W.p_q32(cfg["p"]), cfg["graph_seed"])
    b, _ = O.permute_graph(a, cfg["perm_seed"])
    h, J, off = O.build_gi_ising(a, b)
    cores = min(64, os.cpu_count() or 1)
    cycles = 100
    pool = OraclePool(cores)  # started and warmed outside the timed steps
    for _ in range(args.warmup):
        oracle_rate(pool, h, J, cfg, 20, cores)
    rates, walls = [], []
    for _ in range(args.steps):
        r, w = oracle_rate(pool, h, J, cfg, cycles, cores)
        rates.append(r)
        walls.append(w)
    pool.close()
    value = float(cycles * cores * h.shape[0] * cfg["R"] * len(walls) / sum(walls))
    sample = f"{cores} trials x {cycles} cycles per step (one single-threaded oracle process per core)"
    out = {"impl": "reference", "metric": "spin-updates/sec", "value": value, "unit": "spin-updates/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": sum(walls) / len(walls) * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": f"{WORKLOAD} (bounded sample: {sample})"},
           "cpu_baseline": {"value": value, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                            "sample": sample, "host": host_info()},
           "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the two large-instance timings")
    ap.add_argument("--clocks-csv", default="", help="where to keep the nvidia-smi clock samples ({rank} = rank)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if "RANK" in os.environ else 1))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
