"""Kernels that need more than 48 KB of dynamic shared memory must be granted it on every
device a process uses (the attribute belongs to the device's context). Runs only where the
process sees two GPUs."""
import numpy as np
import pytest

from paper_1504_07028_gb300 import synth

pytestmark = pytest.mark.gpu


def test_second_device_gets_its_own_shared_memory_grants():
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    from paper_1504_07028_gb300 import binding as B
    from paper_1504_07028_gb300 import build
    build.build()
    # 2048-long rows: the row transforms take about 74 KB of shared memory per CTA
    sc = synth.scene(64, 2048, 16, S=8, gap=3.0, noise_std=1.0, wrong_frac=0.0, seed=61)
    p = sc.p.astype(np.float32)
    zs = []
    for dev in (0, 1):
        torch.cuda.set_device(dev)
        s = B.Solver(B.make_params(sc.H, sc.W, sc.K, M=1, sigma=0.5, lam=2.0))
        s.set_probs(p)
        s.solve(5)
        zs.append(s.get_z())
        s.close()
    torch.cuda.set_device(0)
    assert np.array_equal(zs[0], zs[1])
