"""CPU tests of the serving workload's request stream (config 5): each
request is drawn from its own generator keyed by (seed, j), so a stream is
the same whatever order or thread builds it, and its draws stay within the
stated ranges (n in [8, 50], p in [0.3, 0.7], cycles from the given set)."""
import numpy as np

from paper_2302_12454_gb300 import serving_bench as SB


def test_request_spec_is_keyed_by_seed_and_index():
    a = [SB.request_spec(j, 8, 50, (1000, 2000, 5000), 41) for j in range(200)]
    b = [SB.request_spec(j, 8, 50, (1000, 2000, 5000), 41) for j in reversed(range(200))][::-1]
    assert a == b
    c = [SB.request_spec(j, 8, 50, (1000, 2000, 5000), 42) for j in range(200)]
    assert a != c


def test_request_spec_ranges_and_spread():
    specs = [SB.request_spec(j, 8, 50, (1000, 2000, 5000), 41) for j in range(2000)]
    n = np.array([s[0] for s in specs])
    p = np.array([s[1] for s in specs])
    cyc = np.array([s[2] for s in specs])
    assert n.min() >= 8 and n.max() <= 50 and len(set(n.tolist())) == 43
    assert p.min() >= 0.3 and p.max() <= 0.7
    assert set(cyc.tolist()) == {1000, 2000, 5000}
    # the instance seed of request j is seed + j
    assert [s[3] for s in specs[:5]] == [41, 42, 43, 44, 45]
