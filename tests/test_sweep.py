"""The P_s / TTS sweep: its host logic (the success rule, the sizes and cases
taken from Tables 3 and 4) on CPU, and one sweep point against the oracle on
the GPU."""
import math

import pytest

from paper_2302_12454_gb300 import sweep as SW


def test_success_any_replica_final_and_ever():
    ground = -100
    e_final = [[-100, -90], [-80, -90], [-95, -100], [-99, -98]]
    e_best = [[-100, -90], [-100, -90], [-100, -100], [-99, -98]]
    ps, psb = SW.success(e_final, e_best, ground)
    assert ps == 0.5 and psb == 0.75


def test_table_constants():
    # Table 4 sizes are squares of graph sizes 5 .. 50
    assert all(int(round(math.sqrt(n))) ** 2 == n for n in SW.TABLE4_N)
    assert SW.TABLE4_N[-1] == 2500 and len(SW.TABLE4_N) == 7
    # Table 3 cases: iterations = EC / R / (tau (beta + 1)) with R = 25, beta = 3
    its = [(ec // 25) // (tau * 4) for ec, tau in SW.TABLE3_CASES]
    assert its == [2, 1, 4, 2, 4]


@pytest.mark.gpu
def test_sweep_point_on_gpu_matches_oracle():
    """One NEXT-1 sweep point on the GPU (ssqa_point's own anneal and success
    rule, small N) against the oracle on the same instance and parameters:
    every trial's final and best energies, and the resulting P_s."""
    import numpy as np

    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_12454_gb300 as S
    from paper_2302_12454_gb300 import build as B
    from paper_2302_12454_gb300 import workloads as W
    from oracle import oracle as O

    B.build()
    n, trials, cycles, tau = 6, 12, 240, 20
    I = SW._gi(S, W, n, 0)
    h, J, off = I.export()
    kw = dict(R=25, cycles=cycles, seed=7, tau=tau, **W.TABLE2)
    t, E, Eb = SW._timed_anneal(S, torch, I, trials, **kw)
    o = O.anneal(h, J, trials=trials, track_best=True, **kw)
    np.testing.assert_array_equal(E, o["E_final"])
    np.testing.assert_array_equal(Eb, o["E_best"])
    row = SW.ssqa_point(S, W, torch, n, trials=trials, cycles=cycles, tau=tau)
    ps, psb = SW.success(o["E_final"].tolist(), o["E_best"].tolist(), -off)
    assert (row["p_s"], row["p_s_best"]) == (ps, psb)
