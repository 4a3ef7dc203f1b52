"""CPU tests of the benchmark's host-side bookkeeping: the operand bytes per
cycle that the roofline record of a large workload reports, taken from the
streamed path's launch shape as `ssqa_plan` describes it."""
import pytest

import bench
import paper_2302_12454_gb300 as S
from paper_2302_12454_gb300 import build as B
from paper_2302_12454_gb300 import workloads as W
from paper_2302_12454_gb300.__main__ import _instance


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _plan(name):
    c = W.CONFIGS[name]
    I, _ = _instance(S, W, c)
    return S.plan(I, R=c["R"], cycles=c["cycles"], trials=c["trials"], seed=c["seed"], tau=c["tau"])


def test_operand_bytes_single_mode():
    algo, desc = _plan("large_gi_n50")
    assert algo == S.ALGO_STREAMED
    shape, per_cycle = bench.streamed_shape(desc)
    # N = 2500: 79 K-blocks, 10 chunks, 64 column groups of 128 columns, one per CTA
    assert (shape["KB"], shape["NCH"], shape["groups"], shape["dual"]) == (79, 10, 64, 0)
    # every (group, chunk) streams 79 A blocks of 4 KB and 79 B blocks of 8 KB
    assert per_cycle == 79 * 10 * 64 * (4096 + 8192)


def test_operand_bytes_dual_mode():
    algo, desc = _plan("sk_n8192")
    shape, per_cycle = bench.streamed_shape(desc)
    assert (shape["KB"], shape["NCH"], shape["groups"], shape["dual"]) == (256, 32, 16, 1)
    # two groups per CTA share each chunk's B blocks: 8 CTAs per chunk for 16 groups
    assert per_cycle == 256 * 32 * (16 * 4096 + 8 * 8192)
    assert shape["CTAs"] == 8 * shape["CS"]


def test_resident_plan_has_no_streamed_shape():
    algo, desc = _plan("batched_gi_n20")
    assert algo == S.ALGO_TENSOR
    assert bench.streamed_shape(desc) is None
