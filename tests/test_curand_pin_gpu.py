"""A second independent pin of the oracle's Philox4x32-10 (the generator of
the noise r in Eq. 6a): cuRAND's Philox4_32_10 device generator, compiled and
run on the GPU.  Draw n of a state initialised with (seed, subsequence s,
offset 0) is Philox4x32-10 of the counter (n, 0, s_lo, s_hi) under the key
(seed_lo, seed_hi)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_philox_matches_curand(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "curand_philox")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                           os.path.join(HERE, "curand_pin", "curand_philox.cu")])
    lines = subprocess.check_output([exe], text=True).strip().splitlines()
    assert len(lines) == 18
    for ln in lines:
        seed, sub, d, x, y, z, w = (int(v) for v in ln.split())
        ctr = [d, 0, sub & 0xFFFFFFFF, sub >> 32]
        got = O.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        np.testing.assert_array_equal(got, np.array([x, y, z, w], dtype=np.uint32), err_msg=ln)
