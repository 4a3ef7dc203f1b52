"""GPU parity: the CUDA paths of ssqa_anneal / ssqa_energy against the C
oracle, element by element (sigma, Is, energies, history, best energies).
Every comparison is bit-exact: the method is integer arithmetic."""
import numpy as np
import pytest

import paper_2302_12454_gb300 as S
from paper_2302_12454_gb300 import build as B
from paper_2302_12454_gb300 import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def gi(n, p=0.5, gseed=1, pseed=2, toggle=False):
    a = S.gen_er_graph(n, W.p_q32(p), gseed)
    b, perm = S.permute_graph(a, pseed)
    if toggle:
        b = b.copy()
        b[0, n - 1] ^= 1
        b[n - 1, 0] ^= 1
    return S.Ising.gi(a, b)


def both_runs(I, algo, *, R, cycles, trials, seed, track=False, trial_offset=0, state=None, **kw):
    """Run the library and the oracle with the same parameters."""
    h, J, off = I.export()
    lib_kw = dict(kw)
    ora_kw = dict(kw)
    if "coupling" in kw:
        ora_kw["coupling_both"] = ora_kw.pop("coupling")
    g = S.anneal(I, R=R, cycles=cycles, trials=trials, seed=seed, algo=algo, track_best=track,
                 trial_offset=trial_offset, state=state, want_hist=True, **lib_kw)
    o = O.anneal(h, J, R=R, cycles=cycles, trials=trials, seed=seed, track_best=track,
                 trial_offset=trial_offset, state=state, **ora_kw)
    return g, o


def assert_same(g, o, track=False):
    np.testing.assert_array_equal(g["sigma"], o["sigma"])
    np.testing.assert_array_equal(g["Is"], o["Is"])
    np.testing.assert_array_equal(g["E_final"], o["E_final"])
    if "hist" in g:
        np.testing.assert_array_equal(g["hist"], o["hist"])
    if track:
        np.testing.assert_array_equal(g["E_best"], o["E_best"])
        np.testing.assert_array_equal(g["best_cycle"], o["best_cycle"])


# ------------------------------------------------------------ full config 1
@pytest.mark.parametrize("algo", [S.ALGO_TENSOR, S.ALGO_PLAIN, S.ALGO_DELTA])
def test_plain_gi_n6_full_bit_exact(algo):
    c = W.CONFIGS["plain_gi_n6"]
    I = gi(c["n"], c["p"], c["graph_seed"], c["perm_seed"])
    g, o = both_runs(I, algo, R=c["R"], cycles=c["cycles"], trials=c["trials"], seed=c["seed"], tau=c["tau"],
                     track=True)
    assert_same(g, o, track=True)
    h, J, off = I.export()
    assert (g["E_final"] >= -off).all()


# --------------------------------------------- variants, ragged sizes, modes
VARIANTS = [
    # n, R, trials, cycles, extra
    (3, 1, 3, 40, dict(tau=5)),
    (5, 3, 7, 60, dict(tau=7, delay=0)),
    (7, 5, 13, 80, dict(tau=9, delay=2, coupling=1)),
    (8, 8, 17, 50, dict(tau=4, delay=3)),
    (9, 25, 6, 45, dict(tau=5, alpha=3, I0=20)),
    (11, 16, 9, 40, dict(tau=3, jperp_min=-4, jperp_max=8, beta=4, n_rnd=7)),
    (13, 32, 5, 30, dict(tau=6, init_mode=S.INIT_ALL_MINUS)),
    (16, 4, 33, 25, dict(tau=5, delay=1, coupling=1, alpha=2)),
    (17, 2, 65, 20, dict(tau=3)),          # N = 289: two MMA chunks
    (19, 16, 10, 20, dict(tau=2, delay=0, coupling=1)),
    (20, 16, 12, 25, dict(tau=4)),         # N = 400, the batched size
]


@pytest.mark.parametrize("algo", [S.ALGO_TENSOR, S.ALGO_PLAIN, S.ALGO_DELTA])
@pytest.mark.parametrize("n,R,trials,cycles,extra", VARIANTS)
def test_variants_bit_exact(algo, n, R, trials, cycles, extra):
    I = gi(n, 0.5, n, n + 1, toggle=(n % 2 == 1))
    g, o = both_runs(I, algo, R=R, cycles=cycles, trials=trials, seed=1000 + n, track=True, trial_offset=n, **extra)
    assert_same(g, o, track=True)


@pytest.mark.parametrize("algo", [S.ALGO_TENSOR, S.ALGO_PLAIN, S.ALGO_DELTA])
def test_zero_cycles_and_no_noise(algo):
    I = gi(6)
    g, o = both_runs(I, algo, R=4, cycles=0, trials=3, seed=5)
    assert_same(g, o)
    g, o = both_runs(I, algo, R=4, cycles=30, trials=3, seed=5, n_rnd=0, tau=5)
    assert_same(g, o)


@pytest.mark.parametrize("algo", [S.ALGO_TENSOR, S.ALGO_PLAIN, S.ALGO_DELTA])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_resume_equals_straight_run(algo, d):
    I = gi(8, 0.5, 4, 5)
    full = S.anneal(I, R=6, cycles=70, trials=9, seed=7, tau=6, delay=d, algo=algo, want_hist=True)
    part = S.anneal(I, R=6, cycles=25, trials=9, seed=7, tau=6, delay=d, algo=algo, want_hist=True)
    rest = S.anneal(I, R=6, cycles=45, trials=9, seed=7, tau=6, delay=d, algo=algo, want_hist=True,
                    init_mode=S.INIT_FROM_STATE, start_cycle=25, state=part)
    for k in ("sigma", "Is", "E_final") + (("hist",) if d else ()):
        np.testing.assert_array_equal(full[k], rest[k])
    h, J, off = I.export()
    o = O.anneal(h, J, R=6, cycles=45, trials=9, seed=7, tau=6, delay=d, init_mode=2, start_cycle=25,
                 state=dict(sigma=part["sigma"], Is=part["Is"], hist=part.get("hist")))
    np.testing.assert_array_equal(rest["sigma"], o["sigma"])


def test_tensor_equals_plain_and_trial_split():
    I = gi(12, 0.5, 3, 4)
    kw = dict(R=10, cycles=90, trials=40, seed=99, tau=10)
    t = S.anneal(I, algo=S.ALGO_TENSOR, **kw)
    p = S.anneal(I, algo=S.ALGO_PLAIN, **kw)
    for k in ("sigma", "Is", "E_final"):
        np.testing.assert_array_equal(t[k], p[k])
    # the same trials in two calls (trial_offset) equal one call
    kw2 = dict(kw)
    kw2["trials"] = 15
    a = S.anneal(I, algo=S.ALGO_TENSOR, **kw2)
    kw2["trials"] = 25
    b = S.anneal(I, algo=S.ALGO_TENSOR, trial_offset=15, **kw2)
    np.testing.assert_array_equal(np.concatenate([a["sigma"], b["sigma"]]), t["sigma"])


# -------------------------------------------------------------- SK instances
@pytest.mark.parametrize("N", [64, 250, 400])
def test_sk_pm1_bit_exact(N):
    J = W.sk_couplings(N, 31)
    I = S.Ising.dense(J, np.zeros(N, np.int32))
    g, o = both_runs(I, S.ALGO_AUTO, R=8, cycles=20, trials=3, seed=33, tau=5)
    assert_same(g, o)


def test_ferromagnet_accumulation_extremes():
    # all couplings -1 (unit) with large fields: partial sums reach N - 1,
    # the accumulator bound of the FP8 tensor path is exercised at both signs
    N = 400
    J = -np.ones((N, N), np.int8) * 6
    np.fill_diagonal(J, 0)
    h = (np.arange(N, dtype=np.int32) % 7 - 3) * 600
    I = S.Ising.dense(J, h)
    for init in (S.INIT_ALL_MINUS, S.INIT_RANDOM):
        g, o = both_runs(I, S.ALGO_TENSOR, R=16, cycles=12, trials=9, seed=1, tau=3, init_mode=init)
        assert_same(g, o)


# -------------------------------------------------------------------- energy
@pytest.mark.parametrize("N,seed", [(36, 1), (400, 2), (2500, 3), (1000, 4)])
def test_energy_matches_oracle(N, seed):
    if N in (36, 400, 2500):
        n = int(round(N ** 0.5))
        I = gi(n, 0.5, seed, seed + 1)
    else:
        I = S.Ising.dense(W.sk_couplings(N, seed), np.arange(N, dtype=np.int32) - N // 2)
    h, J, off = I.export()
    s = W.random_spins((37, N), seed)
    np.testing.assert_array_equal(S.energy(I, s), O.ising_energy(h, J, s))


# ---------------------------------------- batched GI (N = 400) at full size
def test_batched_gi_n20_full_size_sampled_trials():
    c = W.CONFIGS["batched_gi_n20"]
    I = gi(c["n"], c["p"], c["graph_seed"], c["perm_seed"])
    kw = dict(R=c["R"], cycles=c["cycles"], trials=c["trials"], seed=c["seed"], tau=c["tau"])
    g = S.anneal(I, algo=S.ALGO_TENSOR, **kw)
    h, J, off = I.export()
    for tr in (0, 513, c["trials"] - 1):
        kwo = dict(kw)
        kwo["trials"] = 1
        o = O.anneal(h, J, trial_offset=tr, **kwo)
        np.testing.assert_array_equal(g["sigma"][tr], o["sigma"][0])
        np.testing.assert_array_equal(g["Is"][tr], o["Is"][0])
        np.testing.assert_array_equal(g["E_final"][tr], o["E_final"][0])
    # every trial: the plain CUDA path (per-cycle launches, int8 dot products)
    # gives the same states, and energies match the returned spins
    pl = S.anneal(I, algo=S.ALGO_PLAIN, **kw)
    de = S.anneal(I, algo=S.ALGO_DELTA, **kw)
    for k in ("sigma", "Is", "E_final"):
        np.testing.assert_array_equal(g[k], pl[k])
        np.testing.assert_array_equal(g[k], de[k])
    np.testing.assert_array_equal(S.energy(I, g["sigma"]), g["E_final"])
    assert (g["E_final"] >= -off).all()
    assert (g["Is"] >= -24).all() and (g["Is"] <= 23).all()
    assert ((g["Is"] >= 0) == (g["sigma"] == 1)).all()


# ----------------------------------- large instances: one-cycle transitions
@pytest.mark.parametrize("kind", ["large_gi_n50", "large_gi_n50_p03", "large_gi_n50_p07", "sk_n8192"])
def test_large_instances_transition_sampled(kind):
    c = W.CONFIGS[kind]
    if c["kind"] == "gi":
        I = gi(c["n"], c["p"], c["graph_seed"], c["perm_seed"])
    else:
        I = S.Ising.dense(W.sk_couplings(c["N"], c["j_seed"]), np.zeros(c["N"], np.int32))
    h, J, off = I.export()
    trials = 4
    kw = dict(R=c["R"], trials=trials, seed=c["seed"], tau=c["tau"])
    first = S.anneal(I, cycles=150, want_hist=True, **kw)
    nxt = S.anneal(I, cycles=2, want_hist=True, init_mode=S.INIT_FROM_STATE, start_cycle=150, state=first, **kw)
    straight = S.anneal(I, cycles=152, **kw)
    np.testing.assert_array_equal(nxt["sigma"], straight["sigma"])
    tr = 2
    st = dict(sigma=first["sigma"][tr:tr + 1], Is=first["Is"][tr:tr + 1], hist=first["hist"][tr:tr + 1])
    o = O.anneal(h, J, R=c["R"], cycles=2, trials=1, seed=c["seed"], tau=c["tau"], trial_offset=tr, init_mode=2,
                 start_cycle=150, state=st)
    np.testing.assert_array_equal(nxt["sigma"][tr], o["sigma"][0])
    np.testing.assert_array_equal(nxt["Is"][tr], o["Is"][0])
    np.testing.assert_array_equal(nxt["E_final"][tr], o["E_final"][0])


# ------------------------------------------------- SSA mode (Eq. 2, Sec. 4.4)
@pytest.mark.parametrize("algo", [S.ALGO_TENSOR, S.ALGO_PLAIN, S.ALGO_DELTA])
def test_ssa_mode_matches_eq2(algo):
    # R = 1, J_perp = 0, I0 from 1 to 16 doubling every 10 cycles (scale 4)
    a = S.gen_er_graph(8, W.p_q32(0.5), 51)
    b, _ = S.permute_graph(a, 52)
    I = S.Ising.gi(a, b, 1, 1, 4)
    h, J, off = I.export()
    g = S.anneal(I, R=1, cycles=300, trials=6, seed=53, algo=algo, jperp_max=0, I0=4, alpha=1, n_rnd=4,
                 i0_max=64, i0_mult=2, i0_tau=10)
    for tr in range(6):
        s, Is = O.ssa(h, J, cycles=300, seed=53, trial=tr, i0_min=4, i0_max=64, i0_mult=2, tau=10, alpha=1,
                      n_rnd=4)
        np.testing.assert_array_equal(g["sigma"][tr, 0], s)
        np.testing.assert_array_equal(g["Is"][tr, 0], Is)


@pytest.mark.parametrize("algo", [S.ALGO_TENSOR, S.ALGO_PLAIN, S.ALGO_DELTA])
def test_ssqa_with_i0_schedule_bit_exact(algo):
    I = gi(9, 0.5, 61, 62)
    g, o = both_runs(I, algo, R=8, cycles=120, trials=5, seed=63, tau=7, I0=12, i0_max=96, i0_mult=2, i0_tau=9,
                     track=True)
    assert_same(g, o, track=True)


def test_resume_with_counters_beyond_a_byte():
    # a state from a run with I0' = 400 holds counters outside -128..127: the
    # resident kernel then keeps them as half2 (byte counters otherwise)
    I = gi(9, 0.5, 71, 72)
    h, J, off = I.export()
    big = S.anneal(I, R=4, cycles=40, trials=3, seed=2, algo=S.ALGO_DELTA, I0=400, n_rnd=300, want_hist=True)
    assert np.abs(big["Is"]).max() > 127
    kw = dict(R=4, cycles=20, trials=3, seed=2, tau=5, start_cycle=40)
    g = S.anneal(I, algo=S.ALGO_TENSOR, init_mode=S.INIT_FROM_STATE, state=big, want_hist=True, **kw)
    o = O.anneal(h, J, init_mode=2, state=dict(sigma=big["sigma"], Is=big["Is"], hist=big["hist"]), **kw)
    for k in ("sigma", "Is", "E_final", "hist"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
