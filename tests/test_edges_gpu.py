"""GPU edge cases: degenerate sizes, the size boundaries between the anneal
paths, couplings that the FP8 tensor paths cannot take exactly, and the
largest replica count.  Every comparison with the C oracle is bit-exact."""
import numpy as np
import pytest

import paper_2302_12454_gb300 as S
from paper_2302_12454_gb300 import build as B
from paper_2302_12454_gb300 import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu
ALL = [S.ALGO_AUTO, S.ALGO_TENSOR, S.ALGO_PLAIN, S.ALGO_DELTA]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def dense(N, seed, jmax=1, scale=12, hmax=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    J = rng.integers(-jmax, jmax + 1, size=(N, N)).astype(np.int64) * scale
    J = np.triu(J, 1)
    J = (J + J.T).astype(np.int8)
    h = (rng.integers(-hmax, hmax + 1, size=N) * scale).astype(np.int32)
    return S.Ising.dense(J, h), h, J


def check(I, h, J, algo, **kw):
    g = S.anneal(I, algo=algo, track_best=True, want_hist=True, **kw)
    okw = dict(kw)
    if "coupling" in okw:
        okw["coupling_both"] = okw.pop("coupling")
    o = O.anneal(h.astype(np.int64), J.astype(np.int64), track_best=True, **okw)
    for k in ("sigma", "Is", "E_final", "E_best", "best_cycle"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=f"{k} algo={algo}")
    if kw.get("delay", 1):
        np.testing.assert_array_equal(g["hist"], o["hist"])


@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("N", [1, 2, 17])
def test_tiny_instances(algo, N):
    # N = 1: no couplings at all (the field is h plus noise and replica terms)
    I, h, J = dense(N, 100 + N)
    check(I, h, J, algo, R=3, cycles=25, trials=2, seed=5, tau=3)


@pytest.mark.parametrize("algo", ALL)
def test_single_trial_single_replica(algo):
    I, h, J = dense(40, 7)
    check(I, h, J, algo, R=1, cycles=40, trials=1, seed=9, tau=4, delay=0)


@pytest.mark.parametrize("N,algos", [
    (256, ALL), (257, ALL + [S.ALGO_STREAMED]),               # one / two MMA chunks
    (512, [S.ALGO_AUTO, S.ALGO_PLAIN, S.ALGO_STREAMED]),       # resident maximum (R = 2 leaves room)
    (513, [S.ALGO_AUTO, S.ALGO_STREAMED, S.ALGO_DELTA]),       # streamed from here
])
def test_path_boundaries(N, algos):
    I, h, J = dense(N, N)
    for algo in algos:
        check(I, h, J, algo, R=2, cycles=12, trials=3, seed=N, tau=3)


def test_couplings_outside_fp8_fall_back():
    # J' = +-17 with odd fields: the common unit of J and h is 1 and 17 has no
    # exact E4M3 value, so the tensor paths refuse the instance, AUTO runs the
    # delta path, and results stay exact
    _, _, J = dense(300, 11, jmax=1, scale=17)
    h = (np.arange(300, dtype=np.int32) % 7) * 2 - 5
    I = S.Ising.dense(J, h)
    with pytest.raises(S.SSQAError):
        S.anneal(I, R=4, cycles=5, trials=2, seed=1, algo=S.ALGO_TENSOR)
    with pytest.raises(S.SSQAError):
        S.anneal(I, R=4, cycles=5, trials=2, seed=1, algo=S.ALGO_STREAMED)
    check(I, h, J, S.ALGO_AUTO, R=4, cycles=20, trials=2, seed=1, tau=3)


def test_accumulator_bound_falls_back():
    # J = +-64 on every pair of 300 spins (exact in E4M3, unit 1 because h is
    # odd): row sums of |J| reach 299 * 64 > 2^14, beyond the exact FP8/FP32
    # accumulation bound; both tensor paths refuse, AUTO runs the delta path
    N = 300
    rng = np.random.Generator(np.random.PCG64(12))
    Jf = np.triu(rng.integers(0, 2, size=(N, N)) * 128 - 64, 1)
    J = (Jf + Jf.T).astype(np.int8)
    h = (rng.integers(-3, 4, size=N) * 2 + 1).astype(np.int32)
    I = S.Ising.dense(J, h)
    for algo in (S.ALGO_TENSOR, S.ALGO_STREAMED):
        with pytest.raises(S.SSQAError):
            S.anneal(I, R=4, cycles=5, trials=2, seed=1, algo=algo)
    check(I, h, J, S.ALGO_AUTO, R=4, cycles=15, trials=2, seed=2, tau=3)


@pytest.mark.parametrize("algo", [S.ALGO_TENSOR, S.ALGO_STREAMED, S.ALGO_DELTA])
def test_max_replicas(algo):
    N = 300 if algo == S.ALGO_STREAMED else 60
    I, h, J = dense(N, 13)
    check(I, h, J, algo, R=128, cycles=10, trials=2, seed=3, tau=2, delay=3, coupling=S.COUPLING_BOTH)


def test_invalid_sizes_are_rejected():
    I, h, J = dense(10, 14)
    for bad in (dict(trials=0), dict(R=0), dict(R=129), dict(cycles=-1)):
        kw = dict(R=2, cycles=3, trials=1, seed=1)
        kw.update(bad)
        with pytest.raises(S.SSQAError):
            S.anneal(I, **kw)


@pytest.mark.parametrize("algo", ALL)
def test_counters_not_returned(algo):
    """A host anneal without the counter buffer (want_state=False) returns the
    same spins and energies as one with it, and the oracle's."""
    I, h, J = dense(40, 7)
    kw = dict(R=4, cycles=30, trials=3, seed=5, tau=4)
    g = S.anneal(I, algo=algo, want_state=False, **kw)
    assert "Is" not in g
    o = O.anneal(h.astype(np.int64), J.astype(np.int64), **kw)
    np.testing.assert_array_equal(g["sigma"], o["sigma"])
    np.testing.assert_array_equal(g["E_final"], o["E_final"])
