"""Bounded device-side waits run out without faulting or hanging anything: with the wait
probe on, the first bulk-copy barrier of each sweep / MLR CTA expects 16 bytes that no copy
delivers, so its wait gives up after the (short) budget; the kernel sets the error flag,
gives its copies in flight a second bounded chance and returns. The call reports
SEGSALSA_ERR_TIMEOUT and the CUDA context and the handle stay usable."""
import numpy as np
import pytest

from paper_1504_07028_gb300 import synth

pytestmark = pytest.mark.gpu

SHORT = 200_000          # clock cycles, about 0.1 ms
DEFAULT = 2_000_000_000


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_07028_gb300 import binding
    return binding


def _params(B, sc, **kw):
    return B.make_params(sc.H, sc.W, sc.K, M=1, sigma=0.5, lam=1.5, mu=1.0, **kw)


def test_sweep_wait_runs_out_and_reports_timeout(B):
    sc = synth.scene(40, 37, 8, S=6, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=71)
    p = sc.p.astype(np.float32)
    s = B.Solver(_params(B, sc))
    s.set_probs(p)
    s.set_wait_budget(SHORT, probe=True)
    with pytest.raises(B.SegsalsaError) as e:
        s.solve(3)
    assert e.value.code == B.SEGSALSA_ERR_TIMEOUT
    # back to the default budget: the same handle solves again from set_probs, bit for bit
    # like a fresh handle
    s.set_wait_budget(DEFAULT, probe=False)
    s.set_probs(p)
    s.solve(20, trace_every=10)
    z = s.get_z()
    ref = B.Solver(_params(B, sc))
    ref.set_probs(p)
    ref.solve(20, trace_every=10)
    assert np.array_equal(z, ref.get_z())
    s.close()
    ref.close()


def test_mlr_wait_runs_out_and_keeps_p(B):
    import torch
    ms = synth.mlr_scene(24, 20, 5, 37, S=4, seed=72)
    bf = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(
        torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    x, w = bf(ms.x), bf(ms.Wc)
    s = B.Solver(B.make_params(ms.H, ms.W, ms.K, M=1, sigma=0.5, lam=1.5, mu=1.0))
    s.set_spectra(x, w)
    p0 = s.get_probs()
    s.set_wait_budget(SHORT, probe=True)
    x2 = bf(ms.x[::-1].copy())
    with pytest.raises(B.SegsalsaError) as e:
        s.set_spectra(x2, w)
    assert e.value.code == B.SEGSALSA_ERR_TIMEOUT
    assert np.array_equal(s.get_probs(), p0)         # p kept
    s.set_wait_budget(DEFAULT, probe=False)
    s.set_spectra(x2, w)
    s.solve(5)
    assert np.isfinite(s.get_z()).all()
    s.close()


def test_wait_budget_arguments(B):
    sc = synth.scene(16, 16, 4, S=3, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=73)
    s = B.Solver(_params(B, sc))
    for cyc, pr in ((0, 0), (-5, 0), (1000, 2)):
        with pytest.raises(B.SegsalsaError) as e:
            s.set_wait_budget(cyc, probe=pr)
        assert e.value.code == B.SEGSALSA_ERR_ARG
    s.close()
