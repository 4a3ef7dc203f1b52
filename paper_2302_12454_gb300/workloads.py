"""Seeded synthetic workloads (sizes, seeds and input generators only).

Shared by the tests, the benchmark and the oracle comparisons; nothing here
computes any part of the method.  GI instances follow Sec. 4.2 of the paper
(random graph with edge probability p, second graph a relabelled copy); the
fully connected +-1 (SK-type) instance is a dense random Ising model.
"""
from __future__ import annotations

import numpy as np

# Table 2 at integer scale S = 12 (I0 = 2, n_rnd = 1, J_perp 0 .. 0.5 in
# beta = 3 steps, d = 1, alpha = one least-significant unit)
S = 12
TABLE2 = dict(I0=24, alpha=1, n_rnd=12, jperp_min=0, jperp_max=6, beta=3, delay=1)

CONFIGS = {
    "plain_gi_n6": dict(kind="gi", n=6, p=0.5, graph_seed=1, perm_seed=2, seed=3, R=8, cycles=500, trials=64,
                        tau=100),
    "batched_gi_n20": dict(kind="gi", n=20, p=0.5, graph_seed=11, perm_seed=12, seed=13, R=16, cycles=2000,
                           trials=1024, tau=100),
    "large_gi_n50": dict(kind="gi", n=50, p=0.5, graph_seed=21, perm_seed=22, seed=23, R=32, cycles=5000,
                         trials=256, tau=100),
    # the same size at the other two edge densities of the large GI workload
    "large_gi_n50_p03": dict(kind="gi", n=50, p=0.3, graph_seed=24, perm_seed=25, seed=26, R=32, cycles=5000,
                             trials=256, tau=100),
    "large_gi_n50_p07": dict(kind="gi", n=50, p=0.7, graph_seed=27, perm_seed=28, seed=29, R=32, cycles=5000,
                             trials=256, tau=100),
    "sk_n8192": dict(kind="sk", N=8192, j_seed=31, seed=33, R=32, cycles=2000, trials=64, tau=100),
}


def p_q32(p: float) -> int:
    """Edge probability as the 32-bit threshold used by the graph generator."""
    return min(int(round(p * 2**32)), 2**32 - 1)


def sk_couplings(N: int, seed: int, scale: int = S) -> np.ndarray:
    """Symmetric +-scale couplings with zero diagonal (int8), PCG64-seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.integers(0, 2, size=(N, N), dtype=np.int8) * 2 - 1
    J = np.triu(u, 1)
    J = (J + J.T).astype(np.int8) * np.int8(scale)
    return J


def random_spins(shape, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.integers(0, 2, size=shape, dtype=np.int8) * 2 - 1).astype(np.int8)
