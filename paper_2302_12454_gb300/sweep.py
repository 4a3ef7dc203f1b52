"""P_s / TTS sweeps on synthetic GI instances (the trend of Table 4 and of the
cases of Table 3; Sec. 4.3-4.4).

Every instance is an Erdos-Renyi graph G1 (p = 0.5) and a relabelled copy G2,
so the ground energy is known: -e_offset (Eq. 7-8).  For each size the batch
of trials runs as one anneal on the GPU; a trial succeeds when any replica's
final energy is the ground energy (`p_s`), or when any replica reached it at
some cycle (`p_s_best`).  The time per trial t is the batch's device time
divided by the number of trials (all trials run concurrently), and TTS is
Eq. 10 with P_T = 0.99.  The paper's values come from other instances (its
graphs and several constants are not given), so only the trend compares.

SSQA uses Table 2 at integer scale S = 12 (I0' = 24, n_rnd' = 12, J_perp'
0..6 in beta = 3 steps, d = 1).  SSA (Eq. 2) is the R = 1, J_perp = 0 anneal
with the I0 schedule of Sec. 4.4: I0 = 1 .. 16 doubling every tau = 10 cycles
and n_rnd = 1, in units of the unscaled Hamiltonian (scaled by S: I0' = 12 ..
192, n_rnd' = 12).  The counter resolution alpha is not given for either
method; alpha' (scaled units) is a parameter of both arms: 1 is one least
significant unit, S is alpha = 1 in unscaled units.
"""
from __future__ import annotations

import math
import time

# Table 4: problem sizes N = n^2 of the GI comparisons
TABLE4_N = (25, 100, 400, 625, 1225, 2025, 2500)
# Table 3: (EC, tau) of the five SSQA cases, R = 25
TABLE3_CASES = ((10000, 50), (10000, 100), (20000, 50), (20000, 100), (40000, 100))
TABLE3_N = (900, 1600, 2500)

S_SCALE = 12


def success(e_final, e_best, ground):
    """Per-trial success (any replica at the ground energy): final and ever."""
    fin = [min(row) == ground for row in e_final]
    best = [min(row) == ground for row in e_best]
    return sum(fin) / len(fin), sum(best) / len(best)


def tts(S, t, p):
    return S.tts(t, p, 0.99)


def _gi(S, W, n, seed):
    a = S.gen_er_graph(n, W.p_q32(0.5), 1000 + seed)
    b, _ = S.permute_graph(a, 2000 + seed)
    return S.Ising.gi(a, b)


def _timed_anneal(S, torch, I, trials, **kw):
    """One batched anneal on cuda:0 (device buffers), timed with CUDA events."""
    h, _, _ = I.export()
    N, R = h.shape[0], kw["R"]
    dev = torch.device("cuda")
    sig = torch.empty((trials, R, N), dtype=torch.int8, device=dev)
    Is = torch.empty((trials, R, N), dtype=torch.int32, device=dev)
    E = torch.empty((trials, R), dtype=torch.int64, device=dev)
    Eb = torch.empty((trials, R), dtype=torch.int64, device=dev)
    bc = torch.empty((trials, R), dtype=torch.int32, device=dev)
    p = S.make_params(trials=trials, **kw)
    p.flags |= S.FLAG_TRACK_BEST
    st = torch.cuda.current_stream()
    warm = S.make_params(trials=trials, **dict(kw, cycles=2))
    warm.flags |= S.FLAG_TRACK_BEST
    S.anneal_device(I, warm, sig, Is, e_final=E, e_best=Eb, best_cycle=bc, stream=st)  # instance upload
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    S.anneal_device(I, p, sig, Is, e_final=E, e_best=Eb, best_cycle=bc, stream=st)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, E.cpu().numpy(), Eb.cpu().numpy()


def ssqa_point(S, W, torch, n, *, trials=100, R=25, cycles=1600, tau=100, seed=0, alpha=1):
    I = _gi(S, W, n, seed)
    _, _, off = I.export()
    t, E, Eb = _timed_anneal(S, torch, I, trials, R=R, cycles=cycles, seed=7 + seed, tau=tau,
                             **dict(W.TABLE2, alpha=alpha))
    ps, psb = success(E.tolist(), Eb.tolist(), -off)
    return {"method": "SSQA", "N": n * n, "R": R, "cycles": cycles, "tau": tau, "trials": trials, "alpha": alpha,
            "p_s": ps, "p_s_best": psb, "batch_s": t, "t_per_trial_s": t / trials,
            "tts_s": tts(S, t / trials, ps), "tts_best_s": tts(S, t / trials, psb)}


def ssa_point(S, W, torch, n, *, trials=100, cycles=40000, seed=0, alpha=1):
    I = _gi(S, W, n, seed)
    _, _, off = I.export()
    t, E, Eb = _timed_anneal(S, torch, I, trials, R=1, cycles=cycles, seed=9 + seed, tau=10, beta=3,
                             jperp_min=0, jperp_max=0, delay=1, I0=S_SCALE, i0_max=16 * S_SCALE, i0_mult=2,
                             i0_tau=10, n_rnd=S_SCALE, alpha=alpha)
    ps, psb = success(E.tolist(), Eb.tolist(), -off)
    return {"method": "SSA", "N": n * n, "R": 1, "cycles": cycles, "trials": trials, "alpha": alpha, "p_s": ps,
            "p_s_best": psb, "batch_s": t, "t_per_trial_s": t / trials, "tts_s": tts(S, t / trials, ps),
            "tts_best_s": tts(S, t / trials, psb)}


def table4(S, W, torch, *, sizes=TABLE4_N, trials=100, with_ssa=True, ssqa_alpha=1, ssa_alpha=1, log=None):
    """SSQA (SC = 1600, R = 25, tau = 100) and SSA (40000 cycles) per size."""
    rows = []
    for N in sizes:
        n = int(round(math.sqrt(N)))
        t0 = time.perf_counter()
        rows.append(ssqa_point(S, W, torch, n, trials=trials, alpha=ssqa_alpha))
        if with_ssa:
            rows.append(ssa_point(S, W, torch, n, trials=trials, alpha=ssa_alpha))
        if log:
            log(f"N={N}: {time.perf_counter() - t0:.1f} s")
    return rows


def table3(S, W, torch, *, sizes=TABLE3_N, trials=100, R=25, alpha=1, log=None):
    """The five (EC, tau) cases of Table 3 with SC = EC / R."""
    rows = []
    for N in sizes:
        n = int(round(math.sqrt(N)))
        for case, (ec, tau) in enumerate(TABLE3_CASES, 1):
            r = ssqa_point(S, W, torch, n, trials=trials, R=R, cycles=ec // R, tau=tau, alpha=alpha)
            r.update(case=case, EC=ec, iterations=(ec // R) // (tau * 4))
            rows.append(r)
        if log:
            log(f"N={N} done")
    return rows
