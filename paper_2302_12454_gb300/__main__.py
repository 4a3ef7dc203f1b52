"""Command line: run SSQA anneals on a named synthetic workload, or measure
served latency.

  python -m paper_2302_12454_gb300 anneal --workload batched_gi_n20 \\
      [--cycles C] [--trials T] [--algo tensor|plain|delta|auto] [--repeat K]
  python -m paper_2302_12454_gb300 serve-bench [--requests 200] [--n-min 8]
      [--n-max 20] [--cycles 1000,2000,5000] [--slots 32] [--load 0.8]
      [--seq-sample 200] [--capacity-sample 400] [--plain-sample 16]

Prints one line per run: device time of the anneal (CUDA events on the
launching stream), spin-updates/s, success probability P_s (any replica at
the ground energy -e_offset, GI workloads) and the time to solution of
Eq. 10.  Buffers stay on the device; nothing is copied back except the
final energies.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


def _instance(S, W, cfg):
    if cfg["kind"] == "gi":
        a = S.gen_er_graph(cfg["n"], W.p_q32(cfg["p"]), cfg["graph_seed"])
        b, _ = S.permute_graph(a, cfg["perm_seed"])
        return S.Ising.gi(a, b), True
    N = cfg["N"]
    return S.Ising.dense(W.sk_couplings(N, cfg["j_seed"]), np.zeros(N, np.int32)), False


def cmd_anneal(args):
    import torch

    import paper_2302_12454_gb300 as S
    from paper_2302_12454_gb300 import build as B
    from paper_2302_12454_gb300 import workloads as W

    B.build()
    cfg = dict(W.CONFIGS[args.workload])
    if args.cycles is not None:
        cfg["cycles"] = args.cycles
    if args.trials is not None:
        cfg["trials"] = args.trials
    I, has_ground = _instance(S, W, cfg)
    h, J, off = I.export()
    N, R, T = h.shape[0], cfg["R"], cfg["trials"]
    algo = {"auto": S.ALGO_AUTO, "tensor": S.ALGO_TENSOR, "plain": S.ALGO_PLAIN, "delta": S.ALGO_DELTA,
            "streamed": S.ALGO_STREAMED}[args.algo]
    p = S.make_params(R=R, cycles=cfg["cycles"], trials=T, seed=cfg["seed"], tau=cfg["tau"], algo=algo)
    sig = torch.empty((T, R, N), dtype=torch.int8, device="cuda")
    Is = torch.empty((T, R, N), dtype=torch.int32, device="cuda")
    E = torch.empty((T, R), dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream()
    for k in range(args.repeat):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        S.anneal_device(I, p, sig, Is, e_final=E, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        rec = dict(run=k, workload=args.workload, N=N, R=R, cycles=cfg["cycles"], trials=T, algo=args.algo,
                   seconds=t, spin_updates_per_s=N * R * T * cfg["cycles"] / t)
        if has_ground:
            ps = float((E.min(dim=1).values.cpu().numpy() == -off).mean())
            rec.update(p_s=ps, tts_s=S.tts(t / T, ps, 0.99))
        print(json.dumps(rec), flush=True)


def cmd_serve(args):
    import json as _json

    import paper_2302_12454_gb300 as S
    from paper_2302_12454_gb300 import build as B
    from paper_2302_12454_gb300 import serving_bench as SB
    from paper_2302_12454_gb300 import workloads as W

    B.build()
    out = SB.run(S, W, count=args.requests, n_min=args.n_min, n_max=args.n_max,
                 cycles_set=tuple(int(c) for c in args.cycles.split(",")), slots=args.slots, load=args.load,
                 seq_sample=args.seq_sample, capacity_sample=args.capacity_sample, plain_sample=args.plain_sample,
                 build_threads=args.build_threads)
    print(_json.dumps(out), flush=True)


def cmd_sweep(args):
    import json

    import torch

    import paper_2302_12454_gb300 as S
    from paper_2302_12454_gb300 import build as B
    from paper_2302_12454_gb300 import sweep as SW
    from paper_2302_12454_gb300 import workloads as W

    B.build()
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
    if args.table == 4:
        sizes = tuple(int(x) for x in args.sizes.split(",")) if args.sizes else SW.TABLE4_N
        rows = SW.table4(S, W, torch, sizes=sizes, trials=args.trials, with_ssa=not args.no_ssa,
                         ssqa_alpha=args.ssqa_alpha, ssa_alpha=args.ssa_alpha, log=log)
    else:
        sizes = tuple(int(x) for x in args.sizes.split(",")) if args.sizes else SW.TABLE3_N
        rows = SW.table3(S, W, torch, sizes=sizes, trials=args.trials, alpha=args.ssqa_alpha, log=log)
    for r in rows:
        print(json.dumps(r), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2302_12454_gb300")
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("anneal", help="run anneals of a named workload on cuda:0")
    from paper_2302_12454_gb300 import workloads as W

    a.add_argument("--workload", default="batched_gi_n20", choices=sorted(W.CONFIGS))
    a.add_argument("--cycles", type=int)
    a.add_argument("--trials", type=int)
    a.add_argument("--algo", default="auto", choices=["auto", "tensor", "plain", "delta", "streamed"])
    a.add_argument("--repeat", type=int, default=1)
    sv = sub.add_parser("serve-bench", help="served p50/p99 latency under Poisson arrivals on cuda:0")
    sv.add_argument("--requests", type=int, default=200)
    sv.add_argument("--n-min", type=int, default=8)
    sv.add_argument("--n-max", type=int, default=20)
    sv.add_argument("--cycles", default="1000,2000,5000")
    sv.add_argument("--slots", type=int, default=32)
    sv.add_argument("--load", type=float, default=0.8)
    sv.add_argument("--seq-sample", type=int, default=200, help="requests timed one at a time")
    sv.add_argument("--capacity-sample", type=int, default=400, help="requests of the closed-loop capacity run")
    sv.add_argument("--plain-sample", type=int, default=16, help="requests timed on the plain path")
    sv.add_argument("--build-threads", type=int, default=8, help="threads building instances ahead of arrival")
    sw = sub.add_parser("sweep", help="P_s / TTS sweep on synthetic GI (Table 4 sizes or Table 3 cases) on cuda:0")
    sw.add_argument("--table", type=int, default=4, choices=[3, 4])
    sw.add_argument("--trials", type=int, default=100)
    sw.add_argument("--sizes", default="", help="comma-separated N (squares of the graph sizes)")
    sw.add_argument("--no-ssa", action="store_true", help="Table 4 without the SSA arm")
    sw.add_argument("--ssqa-alpha", type=int, default=1, help="SSQA counter resolution alpha' (scaled units)")
    sw.add_argument("--ssa-alpha", type=int, default=1, help="SSA counter resolution alpha' (scaled units)")
    args = ap.parse_args(argv)
    if args.cmd == "anneal":
        cmd_anneal(args)
    elif args.cmd == "serve-bench":
        cmd_serve(args)
    elif args.cmd == "sweep":
        cmd_sweep(args)


if __name__ == "__main__":
    sys.exit(main())
