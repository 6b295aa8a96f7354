"""MLR class model on the tensor cores (segsalsa_str_set_spectra) against the FP64 oracle.

The GPU multiplies BF16 spectra by BF16 weights with FP32 accumulation and takes the softmax in
FP32; the oracle takes the same BF16 values in FP64. A product of two BF16 numbers is exact in
FP32, so the logits differ only by the FP32 accumulation (about d * 2^-24 * sum |w x|, below
1e-5 here) and p by at most that times p (tolerance 3e-5)."""
import numpy as np
import pytest

from oracle import segsalsa_str_oracle as O
from paper_1504_07028_gb300 import synth
from tests.helpers import label_agreement, max_abs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_07028_gb300 import binding
    return binding


def _bf16(a, dev=True):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.cuda() if dev else t


def _f64(t):
    import torch
    return t.to(torch.float64).cpu().numpy()


def _solver(B, H, W, K, M=1, prec="fp32"):
    return B.Solver(B.make_params(H, W, K, M=M, sigma=0.5 if M == 1 else 1.0, lam=1.5, mu=1.0,
                                  schatten_p=1, precision=prec))


@pytest.mark.parametrize("H,W,K,d", [
    (37, 29, 9, 103),     # the 103-band, 9-class shape; 1073 pixels = 8 full tiles + a partial one
    (20, 13, 20, 7),      # K > 16 (N = 32 accumulator columns), d < 16
    (9, 15, 3, 256),      # the most bands
    (4, 32, 4, 16),       # exactly one tile, d one MMA step
    (5, 26, 2, 33),       # 130 pixels: a tile of 2
])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_mlr_probs_match_oracle(B, H, W, K, d, prec):
    import torch
    sc = synth.mlr_scene(H, W, K, d, S=4, seed=50 + K + d)
    bias = np.random.default_rng(d).normal(0, 0.3, size=K).astype(np.float32)
    x, w = _bf16(sc.x), _bf16(sc.Wc)
    bt = torch.from_numpy(bias).cuda()
    torch.cuda.synchronize()
    s = _solver(B, H, W, K, prec=prec)
    s.set_spectra(x, w, bt)
    p = s.get_probs()
    ref = O.mlr_probs(_f64(x).reshape(H, W, d), _f64(w), bias.astype(np.float64))
    assert max_abs(p, ref) < 3e-5
    assert np.abs(p.sum(axis=0) - 1).max() < 1e-5 and p.min() > 0
    lg = np.sort(ref, axis=0)
    clear = lg[-1] - lg[-2] > 1e-4
    assert np.array_equal(np.argmax(p, 0)[clear], np.argmax(ref, 0)[clear])
    assert s.get_iteration() == 0
    s.close()


def test_mlr_host_and_device_inputs_agree(B):
    import torch
    sc = synth.mlr_scene(23, 17, 6, 40, S=4, seed=60)
    s = _solver(B, 23, 17, 6)
    xh, wh = _bf16(sc.x, dev=False), _bf16(sc.Wc, dev=False)
    s.set_spectra(xh.view(torch.int16).numpy().view(np.uint16), wh.view(torch.int16).numpy().view(np.uint16))
    p_host = s.get_probs()
    xd, wd = xh.cuda(), wh.cuda()
    torch.cuda.synchronize()
    s.set_spectra(xd, wd)
    assert np.array_equal(s.get_probs(), p_host)
    # device spectra and weights that do not start on a 16-byte boundary (views one value in)
    big = torch.empty(xd.numel() + 1, dtype=torch.bfloat16, device="cuda")
    big[1:] = xd.reshape(-1)
    xm = big[1:].view(xd.shape)
    bigw = torch.empty(wd.numel() + 1, dtype=torch.bfloat16, device="cuda")
    bigw[1:] = wd.reshape(-1)
    wm = bigw[1:].view(wd.shape)
    assert xm.data_ptr() % 16 != 0 and wm.data_ptr() % 16 != 0
    torch.cuda.synchronize()
    s.set_spectra(xm, wm)
    assert np.array_equal(s.get_probs(), p_host)
    s.close()


def test_mlr_front_end_then_solve(B):
    """5x5 patch (M = 2), Schatten-1: the solve started from the tensor-core probabilities ends
    within 1e-4 of the oracle solve started from the oracle's probabilities."""
    import torch
    H, W, K, d = 33, 26, 9, 103
    sc = synth.mlr_scene(H, W, K, d, S=6, seed=61)
    x, w = _bf16(sc.x), _bf16(sc.Wc)
    torch.cuda.synchronize()
    s = _solver(B, H, W, K, M=2)
    s.set_spectra(x, w)
    s.solve(40)
    z = s.get_z()
    p_ref = O.mlr_probs(_f64(x).reshape(H, W, d), _f64(w))
    ref, _ = O.solve(p_ref, 2, 1.0, 1.5, 1.0, 1, 40)
    assert max_abs(z, ref.z) < 1e-4
    ok, _ = label_agreement(z, ref.z)
    assert ok
    s.close()


def test_mlr_rejects_bad_input(B):
    import torch
    H, W, K = 12, 10, 4
    s = _solver(B, H, W, K)
    sc = synth.mlr_scene(H, W, K, 257, S=3, seed=62)
    with pytest.raises(B.SegsalsaError) as e:
        s.set_spectra(_bf16(sc.x), _bf16(sc.Wc))
    assert e.value.code == B.SEGSALSA_ERR_ARG
    sc = synth.mlr_scene(H, W, K, 20, S=3, seed=63)
    s.set_spectra(_bf16(sc.x), _bf16(sc.Wc))
    s.solve(3)
    z0 = s.get_z()
    xb = sc.x.copy()
    xb[3, 4, 5] = np.nan
    xn = _bf16(xb)
    torch.cuda.synchronize()
    with pytest.raises(B.SegsalsaError) as e:
        s.set_spectra(xn, _bf16(sc.Wc))
    assert e.value.code == B.SEGSALSA_ERR_ARG
    assert s.get_iteration() == 3 and np.array_equal(s.get_z(), z0)
    s.close()


def test_mlr_staging_survives_traced_solves(B):
    """The handle's staging buffer for the weights outlives traced solves that grow the pinned
    trace buffer: front end, traced solve, front end again (same and new spectra) on one handle
    gives the probabilities of a fresh handle every time."""
    import torch
    H, W, K, d = 21, 19, 6, 40
    sc = synth.mlr_scene(H, W, K, d, S=4, seed=64)
    sc2 = synth.mlr_scene(H, W, K, d, S=4, seed=65)
    s = _solver(B, H, W, K)
    for i, (scn, iters, every) in enumerate([(sc, 20, 10), (sc, 200, 5), (sc2, 30, 1), (sc, 5, 1)]):
        x, w = _bf16(scn.x), _bf16(scn.Wc)
        torch.cuda.synchronize()
        s.set_spectra(x, w)
        p = s.get_probs()
        fresh = _solver(B, H, W, K)
        fresh.set_spectra(x, w)
        assert np.array_equal(p, fresh.get_probs()), i
        fresh.close()
        tr = s.solve(iters, trace_every=every)
        assert len(tr) >= iters // every
    s.close()
