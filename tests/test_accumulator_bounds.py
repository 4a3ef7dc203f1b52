"""The tensor-core paths at the exact edges of their accumulator formats.

The FP8 field product of Eq. 6a is exact only while every partial sum of
(J sigma + h) / jm is an integer the accumulator holds exactly: the resident
kernel takes an FP16 accumulator when max_i (|h_i| + sum_j |J_ij|) / jm plus
max_i |h_i| / jm is at most 2048 (the energy term D + h / jm must also be
exact), and both tensor paths take FP32 accumulation up to row sums of 2^14.
These tests build instances whose row sums sit exactly at each bound (and one
unit past it), drive the partial sums to the bound at both signs with +-1
steps at the end of the K order and in the h-digit columns, and compare
sigma, Is and every energy with the C oracle bit for bit.  The CPU tests check
the host's choice of path and accumulator at each bound (ssqa_plan)."""
import numpy as np
import pytest

import paper_2302_12454_gb300 as S
from paper_2302_12454_gb300 import build as B
from oracle import oracle as O
from bound_instances import bound_instance, crafted_states

# name: (N, F = sum_j |J_ij| / jm, H = |h_i| / jm, jm)
CASES = {
    "f16_edge": (400, 2048, 0, 1),          # FP16: row sum + max |h| = 2048, D reaches +-2048
    "f16_edge_h": (400, 2000, 24, 1),       # FP16: 2024 + 24 = 2048, h digits 8 + 1 * 16 last
    "f16_past": (400, 2049, 0, 1),          # one past: the FP32 accumulator
    "f32_edge": (400, 16384 - 1329, 1329, 1),  # FP32: row sums exactly 2^14, h digits 1, 3, 5
    "f32_past": (400, 16385 - 1329, 1329, 1),  # one past: no tensor path (delta)
    "s_edge": (1000, 16384 - 300, 300, 6),  # streamed, 2^14 with jm = 6 (J' = 6 f)
    "s_past": (1000, 16385 - 300, 300, 6),
}
TABLE2 = dict(I0=24, alpha=1, n_rnd=12, jperp_min=0, jperp_max=6, beta=3, delay=1)


def instance(name):
    N, F, H, jm = CASES[name]
    J, h, u = bound_instance(N, F, H, seed=N + F, jm=jm)
    return S.Ising.dense(J, h), J, h, u


# ------------------------------------------------------------------ host (CPU)
def test_instances_sit_on_the_bounds():
    for name, (N, F, H, jm) in CASES.items():
        J, h, u = bound_instance(N, F, H, seed=N + F, jm=jm)
        assert (J == J.T).all() and (np.diag(J) == 0).all()
        rows = (np.abs(J.astype(np.int64)).sum(axis=1) + np.abs(h.astype(np.int64))) // jm
        assert (rows == F + H).all(), name
        # sigma = u: every partial sum of row i along K has the sign of u_i and
        # grows monotonically to u_i (F + H), the bound
        P = np.cumsum(J.astype(np.int64) * u[None, :].astype(np.int64), axis=1) // jm
        assert (np.diff(P * u[:, None], axis=1) >= 0).all()
        assert (P[:, -1] + h // jm == u.astype(np.int64) * (F + H)).all()
        # +-1 steps at the end of the K order for the last rows
        assert (np.abs(J[N - 16:, N - 16:].astype(np.int64)) // jm <= 1).all()


def _plan(I, **kw):
    kw.setdefault("R", 16)
    kw.setdefault("cycles", 5)
    kw.setdefault("trials", 8)
    return S.plan(I, **kw)


def test_plan_fp16_accumulator_up_to_2048():
    for name in ("f16_edge", "f16_edge_h"):
        I = instance(name)[0]
        algo, desc = _plan(I)
        assert algo == S.ALGO_TENSOR and "FP16 accumulator" in desc, (name, desc)
    algo, desc = _plan(instance("f16_past")[0])
    assert algo == S.ALGO_TENSOR and "FP32 accumulator" in desc, desc


def test_plan_fp32_accumulator_up_to_2_14():
    I = instance("f32_edge")[0]
    algo, desc = _plan(I)
    assert algo == S.ALGO_TENSOR and "FP32 accumulator" in desc, desc
    assert _plan(I, algo=S.ALGO_STREAMED)[0] == S.ALGO_STREAMED
    assert _plan(instance("s_edge")[0])[0] == S.ALGO_STREAMED
    for name in ("f32_past", "s_past"):
        I = instance(name)[0]
        algo, desc = _plan(I)
        assert algo == S.ALGO_DELTA and "2^14" in desc, (name, desc)
        for forced in (S.ALGO_TENSOR, S.ALGO_STREAMED):
            with pytest.raises(S.SSQAError) as e:
                _plan(I, algo=forced)
            assert e.value.code == S.ERR_UNSUPPORTED


# --------------------------------------------------------------- GPU parity
@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def _compare(I, J, h, algo, *, R, trials, cycles, seed, state=None, start_cycle=0, init_mode=S.INIT_RANDOM,
             trace=True):
    kw = dict(R=R, cycles=cycles, trials=trials, seed=seed, tau=5, **TABLE2)
    if state is not None:
        init_mode = S.INIT_FROM_STATE
    g = S.anneal(I, algo=algo, track_best=True, want_trace=trace and cycles > 0, want_hist=True, state=state,
                 init_mode=init_mode, start_cycle=start_cycle, **kw)
    o = O.anneal(h, J, track_best=True, trace=trace and cycles > 0, state=state, init_mode=init_mode,
                 start_cycle=start_cycle, **kw)
    keys = ["sigma", "Is", "E_final", "E_best", "best_cycle", "hist"]
    if trace and cycles > 0:
        keys.append("E_trace")
    for k in keys:
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    return g


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["f16_edge", "f16_edge_h", "f16_past", "f32_edge", "f32_past"])
@pytest.mark.parametrize("init_mode", [S.INIT_RANDOM, S.INIT_ALL_MINUS])
def test_resident_fresh_start_at_bounds(gpu, name, init_mode):
    """Fresh starts take the byte-counter variants (FP16 accumulator below
    2048).  The Mattis structure aligns the replicas with +-u within a few
    cycles, after which |D| sits at the bound every cycle."""
    I, J, h, u = instance(name)
    algo = S.ALGO_AUTO if name.endswith("past") and name.startswith("f32") else S.ALGO_TENSOR
    g = _compare(I, J, h, algo, R=16, trials=16, cycles=30, seed=11, init_mode=init_mode)
    # the run reached the aligned states (|field| at the bound) it was built for
    assert (np.abs(g["sigma"].astype(np.int64) @ u.astype(np.int64)) == u.shape[0]).any()


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["f16_edge", "f16_edge_h", "f32_edge", "f32_past"])
@pytest.mark.parametrize("cycles", [0, 3])
def test_resident_crafted_states_at_bounds(gpu, name, cycles):
    """Resumed states (half2 counters, FP32 accumulator): per column sigma = u,
    -u, u with spins of the last K-block flipped (sums climb to the top and
    step back by the flipped magnitudes, +-1 in the unit band), half u / half
    -u (up to half the bound and back near 0), and random; cycles = 0 checks
    the final-energy pass on exactly these states."""
    I, J, h, u = instance(name)
    st = crafted_states(u, trials=16, R=16, I0=24, seed=5)
    algo = S.ALGO_AUTO if name == "f32_past" else S.ALGO_TENSOR
    _compare(I, J, h, algo, R=16, trials=16, cycles=cycles, seed=12, state=st, start_cycle=37)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["s_edge", "f32_edge"])
@pytest.mark.parametrize("crafted", [False, True])
def test_streamed_at_fp32_bound(gpu, name, crafted):
    I, J, h, u = instance(name)
    R, trials = 8, 5
    st = crafted_states(u, trials=trials, R=R, I0=24, seed=9) if crafted else None
    _compare(I, J, h, S.ALGO_STREAMED, R=R, trials=trials, cycles=3 if crafted else 12, seed=13, state=st,
             start_cycle=101 if crafted else 0)


@pytest.mark.gpu
def test_streamed_past_fp32_bound_falls_back(gpu):
    I, J, h, u = instance("s_past")
    with pytest.raises(S.SSQAError) as e:
        S.anneal(I, R=8, cycles=2, trials=2, seed=1, algo=S.ALGO_STREAMED)
    assert e.value.code == S.ERR_UNSUPPORTED
    st = crafted_states(u, trials=3, R=8, I0=24, seed=10)
    _compare(I, J, h, S.ALGO_AUTO, R=8, trials=3, cycles=3, seed=14, state=st, start_cycle=5)
