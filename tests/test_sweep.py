"""Host logic of the P_s / TTS sweep (no GPU): the success rule and the sizes
and cases taken from Tables 3 and 4."""
import math

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
