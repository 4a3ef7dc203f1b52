"""GPU parity of the streamed tensor-core path (SSQA_ALGO_STREAMED): J kept
in L2 and streamed in 256-spin chunks, clusters of CTAs sharing the chunks of
one group of 128 spin columns.  Every comparison with the C oracle is
bit-exact (Eq. 6a-6c are integer arithmetic); at the full sizes of the large
workloads all trials are compared with the delta CUDA-core path and sampled
trials with the oracle."""
import numpy as np
import pytest

import paper_2302_12454_gb300 as S
from paper_2302_12454_gb300 import build as B
from paper_2302_12454_gb300 import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu
ST = S.ALGO_STREAMED


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def gi(n, p=0.5, gseed=1, pseed=2, toggle=False):
    a = S.gen_er_graph(n, W.p_q32(p), gseed)
    b, _ = S.permute_graph(a, pseed)
    if toggle:
        b = b.copy()
        b[0, n - 1] ^= 1
        b[n - 1, 0] ^= 1
    return S.Ising.gi(a, b)


def sk(N, seed, hscale=0):
    h = ((np.arange(N, dtype=np.int64) * 7919) % 23 - 11).astype(np.int32) * hscale
    return S.Ising.dense(W.sk_couplings(N, seed), h)


def both(I, *, R, cycles, trials, seed, track=True, **kw):
    h, J, _ = I.export()
    g = S.anneal(I, R=R, cycles=cycles, trials=trials, seed=seed, algo=ST, track_best=track, want_hist=True, **kw)
    okw = dict(kw)
    if "coupling" in okw:
        okw["coupling_both"] = okw.pop("coupling")
    o = O.anneal(h, J, R=R, cycles=cycles, trials=trials, seed=seed, track_best=track, **okw)
    return g, o


def same(g, o, track=True, rows=slice(None)):
    for k in ("sigma", "Is", "E_final") + (("hist",) if "hist" in g and "hist" in o else ()):
        np.testing.assert_array_equal(g[k][rows], o[k], err_msg=k)
    if track:
        np.testing.assert_array_equal(g["E_best"][rows], o["E_best"], err_msg="E_best")
        np.testing.assert_array_equal(g["best_cycle"][rows], o["best_cycle"], err_msg="best_cycle")


CASES = [
    # instance, R, trials, cycles, extra
    ("gi17", 2, 65, 30, dict(tau=3, trial_offset=5)),                       # N 289: 2 chunks, ragged group
    ("gi20", 16, 12, 25, dict(tau=4)),                                      # N 400
    ("gi23", 25, 11, 20, dict(tau=5, delay=2, coupling=1)),                 # N 529: 3 chunks, R not dividing 128
    ("sk1000h", 8, 17, 20, dict(tau=3, delay=3, alpha=3, I0=20)),           # h digit columns
    ("sk300", 128, 3, 30, dict(tau=6, jperp_min=-4, jperp_max=8, beta=4, n_rnd=7)),
    ("sk300", 7, 40, 25, dict(tau=2, delay=0, init_mode=S.INIT_ALL_MINUS)),
    ("gi19", 1, 9, 60, dict(tau=5, jperp_max=0, I0=4, n_rnd=4, i0_max=64, i0_mult=2, i0_tau=10)),  # SSA mode
    ("gi18", 8, 10, 40, dict(tau=7, I0=12, i0_max=96, i0_mult=2, i0_tau=9)),
]


def instance(name):
    if name.startswith("gi"):
        n = int(name[2:])
        return gi(n, 0.5, n, n + 1, toggle=(n % 2 == 1))
    if name == "sk1000h":
        return sk(1000, 4, hscale=12)
    return sk(int(name[2:]), 5)


@pytest.mark.parametrize("name,R,trials,cycles,extra", CASES)
def test_streamed_bit_exact(name, R, trials, cycles, extra):
    I = instance(name)
    g, o = both(I, R=R, cycles=cycles, trials=trials, seed=700 + R, **extra)
    same(g, o)


def test_streamed_zero_cycles_and_no_noise():
    I = gi(17, 0.5, 3, 4)
    g, o = both(I, R=4, cycles=0, trials=3, seed=5)
    same(g, o)
    assert (g["best_cycle"] == -1).all()
    g, o = both(I, R=4, cycles=30, trials=3, seed=5, n_rnd=0, tau=5)
    same(g, o)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_streamed_resume_equals_straight_run(d):
    I = gi(18, 0.5, 4, 5)
    kw = dict(R=6, trials=9, seed=7, tau=6, delay=d, algo=ST, want_hist=True)
    full = S.anneal(I, cycles=70, **kw)
    part = S.anneal(I, cycles=25, **kw)
    rest = S.anneal(I, cycles=45, init_mode=S.INIT_FROM_STATE, start_cycle=25, state=part, **kw)
    for k in ("sigma", "Is", "E_final") + (("hist",) if d else ()):
        np.testing.assert_array_equal(full[k], rest[k])


def test_streamed_ferromagnet_accumulation_extremes():
    # all couplings -6 (one unit) and fields up to 6 * 2400: field sums reach
    # |D| near the 2^14 accumulator bound at both signs; four h digit columns
    N = 1000
    J = -np.ones((N, N), np.int8) * 6
    np.fill_diagonal(J, 0)
    h = (np.arange(N, dtype=np.int32) % 9 - 4) * 3600
    I = S.Ising.dense(J, h)
    for init in (S.INIT_ALL_MINUS, S.INIT_RANDOM):
        g, o = both(I, R=16, cycles=8, trials=9, seed=1, tau=3, init_mode=init)
        same(g, o)


def test_streamed_rejects_small_and_out_of_range_state():
    with pytest.raises(S.SSQAError):
        S.anneal(gi(9), R=4, cycles=5, trials=2, seed=1, algo=ST)   # N = 81: resident sizes only
    I = gi(17, 0.5, 8, 9)
    big = S.anneal(I, R=4, cycles=40, trials=3, seed=2, algo=S.ALGO_DELTA, I0=400, n_rnd=300, want_hist=True)
    assert np.abs(big["Is"]).max() > 127
    kw = dict(R=4, cycles=20, trials=3, seed=2, init_mode=S.INIT_FROM_STATE, start_cycle=40, state=big,
              want_hist=True)
    with pytest.raises(S.SSQAError):
        S.anneal(I, algo=ST, **kw)
    auto = S.anneal(I, algo=S.ALGO_AUTO, **kw)
    delta = S.anneal(I, algo=S.ALGO_DELTA, **kw)
    for k in ("sigma", "Is", "E_final"):
        np.testing.assert_array_equal(auto[k], delta[k])


def test_large_gi_n50_full_trials():
    c = W.CONFIGS["large_gi_n50"]
    I = gi(c["n"], c["p"], c["graph_seed"], c["perm_seed"])
    kw = dict(R=c["R"], cycles=30, trials=c["trials"], seed=c["seed"], tau=c["tau"], track_best=True)
    g = S.anneal(I, algo=S.ALGO_AUTO, **kw)
    de = S.anneal(I, algo=S.ALGO_DELTA, **kw)
    for k in ("sigma", "Is", "E_final", "E_best", "best_cycle"):
        np.testing.assert_array_equal(g[k], de[k], err_msg=k)
    h, J, _ = I.export()
    for tr in (0, 85, 170, c["trials"] - 1):
        o = O.anneal(h, J, R=c["R"], cycles=30, trials=1, seed=c["seed"], tau=c["tau"], trial_offset=tr,
                     track_best=True)
        for k in ("sigma", "Is", "E_final", "E_best", "best_cycle"):
            np.testing.assert_array_equal(g[k][tr:tr + 1], o[k], err_msg=k)


def test_sk_n8192_full_trials():
    c = W.CONFIGS["sk_n8192"]
    I = S.Ising.dense(W.sk_couplings(c["N"], c["j_seed"]), np.zeros(c["N"], np.int32))
    kw = dict(R=c["R"], cycles=3, trials=c["trials"], seed=c["seed"], tau=c["tau"])
    g = S.anneal(I, algo=S.ALGO_AUTO, **kw)
    de = S.anneal(I, algo=S.ALGO_DELTA, **kw)
    for k in ("sigma", "Is", "E_final"):
        np.testing.assert_array_equal(g[k], de[k], err_msg=k)
    h, J, _ = I.export()
    for tr in (0, 21, 42, c["trials"] - 1):
        o = O.anneal(h, J, R=c["R"], cycles=3, trials=1, seed=c["seed"], tau=c["tau"], trial_offset=tr)
        for k in ("sigma", "Is", "E_final"):
            np.testing.assert_array_equal(g[k][tr:tr + 1], o[k], err_msg=k)


@pytest.mark.parametrize("case", ["dummy_steps", "padded_groups"])
def test_streamed_cluster_shapes(case):
    # On a 152-SM device: N = 1100 has 5 chunks over 4 ranks (ranks with fewer
    # chunks run dummy steps); 17 groups of R = 32 columns pad to 18 for 2-group
    # clusters.  All trials equal the delta path; sampled trials equal the oracle.
    if case == "dummy_steps":
        I = sk(1100, 7, hscale=12)
        kw = dict(R=16, cycles=20, trials=256, seed=81, tau=4, delay=2)
        sample = (0, 255)
    else:
        I = gi(45, 0.5, 45, 46)
        kw = dict(R=32, cycles=15, trials=65, seed=82, tau=3, coupling=1)
        sample = (64,)
    g = S.anneal(I, algo=ST, track_best=True, **kw)
    de = S.anneal(I, algo=S.ALGO_DELTA, track_best=True, **kw)
    for k in ("sigma", "Is", "E_final", "E_best", "best_cycle"):
        np.testing.assert_array_equal(g[k], de[k], err_msg=k)
    h, J, _ = I.export()
    okw = dict(kw)
    if "coupling" in okw:
        okw["coupling_both"] = okw.pop("coupling")
    okw["trials"] = 1
    for tr in sample:
        o = O.anneal(h, J, trial_offset=tr, track_best=True, **okw)
        for k in ("sigma", "Is", "E_final", "E_best", "best_cycle"):
            np.testing.assert_array_equal(g[k][tr:tr + 1], o[k], err_msg=k)


def test_two_column_groups_per_cta():
    """From 160 K-blocks per chunk (N = 5152 here) a CTA serves two groups of
    128 columns whose MMAs share each B block.  R = 32 and 10 trials make
    three groups (4 + 4 + 2 trials): one CTA pair with both groups, one with
    a single, partial group.  A trial of each group against the oracle."""
    N, R, trials, cycles = 5152, 32, 10, 4
    I = sk(N, 41, hscale=12)
    h, J, _ = I.export()
    g = S.anneal(I, R=R, cycles=cycles, trials=trials, seed=43, tau=2, algo=ST, track_best=True)
    for tr in (1, 6, 9):
        o = O.anneal(h, J, R=R, cycles=cycles, trials=1, seed=43, tau=2, trial_offset=tr, track_best=True)
        for k in ("sigma", "Is", "E_final", "E_best", "best_cycle"):
            np.testing.assert_array_equal(g[k][tr], o[k][0], err_msg=f"{k} trial {tr}")


@pytest.mark.parametrize("kind,start", [("large_gi_n50", 4799), ("sk_n8192", 1998)])
def test_late_anneal_against_oracle(kind, start):
    """The late regime of the large configurations: one trial resumed from the
    GPU's own state at cycle 4799 (config 3, 5000 cycles) or 1998 (config 4,
    2000 cycles), two more cycles on both sides.  Those cycles run at Table 2's
    top J_perp level (t mod tau (beta + 1) = 399 / 398 with tau = 100) and, for
    config 3, across the level's reset at t = 4800; counters are saturated and
    few spins flip."""
    c = W.CONFIGS[kind]
    if c["kind"] == "gi":
        I = gi(c["n"], c["p"], c["graph_seed"], c["perm_seed"])
    else:
        I = S.Ising.dense(W.sk_couplings(c["N"], c["j_seed"]), np.zeros(c["N"], np.int32))
    h, J, _ = I.export()
    tr = 3
    kw = dict(R=c["R"], trials=1, seed=c["seed"], tau=c["tau"], trial_offset=tr)
    first = S.anneal(I, cycles=start, want_hist=True, algo=S.ALGO_AUTO, **kw)
    nxt = S.anneal(I, cycles=2, want_hist=True, algo=S.ALGO_AUTO, init_mode=S.INIT_FROM_STATE, start_cycle=start,
                   state=first, track_best=True, **kw)
    st = dict(sigma=first["sigma"], Is=first["Is"], hist=first["hist"])
    o = O.anneal(h, J, cycles=2, init_mode=2, start_cycle=start, state=st, track_best=True, **kw)
    for k in ("sigma", "Is", "E_final", "E_best", "best_cycle", "hist"):
        np.testing.assert_array_equal(nxt[k], o[k], err_msg=k)
    # the state is the late regime: counters mostly saturated
    sat = np.isin(first["Is"], (-24, 23)).mean()
    assert sat > 0.5, sat
