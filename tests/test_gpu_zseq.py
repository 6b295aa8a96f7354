"""The z-update (eq. 12) as one launch of persistent CTAs that take the units of the three
passes (forward row transforms, column recursions, inverse row transforms) in ticket order
(tiling zfuse = 3). It runs the same unit bodies as the three launches, so its results must be
bit-identical to them, and both must match the oracle's DFT solve. Also checked: the ticket
counters return to zero after every launch (long graph-replayed solves, handles on concurrent
streams), and the dependency wait runs out cleanly under the wait probe."""
import numpy as np
import pytest
import torch

from oracle import segsalsa_str_oracle as O
from paper_1504_07028_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_07028_gb300 import binding
    return binding


def khw_to_hwk(a):
    return np.ascontiguousarray(np.transpose(a, (1, 2, 0)))


def hwk_to_khw(a):
    return np.ascontiguousarray(np.transpose(a, (2, 0, 1)))


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))))


SHAPES = [
    (64, 64, 4, 1, "fp64", 1.0), (145, 145, 16, 1, "fp32", 1.0), (37, 50, 5, 2, "fp32", 1.0),
    (33, 17, 32, 1, "fp32", 1.0), (96, 131, 4, 1, "fp32", 1.0), (40, 127, 8, 1, "fp32", 1.0),
    (40, 37, 8, 1, "fp64", 5.0), (71, 64, 6, 1, "fp32", 5.0), (35, 24, 3, 0, "fp64", 3.0),
    (300, 362, 16, 1, "fp32", 1.0), (9, 8, 2, 1, "fp32", 1.0)]


@pytest.mark.parametrize("H,W,K,M,prec,wscale", SHAPES)
def test_linear_solve_one_launch(B, H, W, K, M, prec, wscale):
    """linear_solve with zfuse = 3 against the three launches (bit for bit) and the oracle.
    The shapes include a Bluestein row length (127), a direct prime factor (37, 131), odd K,
    K = 32, weights whose column recursions span the whole period (wscale > 1), rows of 362
    (Bluestein, column segments lengthened to fit the one-launch CTA) and a 9 x 8 image."""
    om = wscale * O.gaussian_weights(M, 0.5 + 0.5 * M)
    dt = np.float64 if prec == "fp64" else np.float32
    rhs = synth.random_field((K, H, W), seed=H * 1000 + W + 11).astype(dt)
    ref = O.linear_solve(rhs.astype(np.float64), om, M)
    tol = 1e-11 if prec == "fp64" else 2e-5
    mk = lambda zf, cr=0: B.Solver(B.make_params(H, W, K, M=M, sigma=0.5 + 0.5 * M, precision=prec,
                                                 weights=om), tiling=B.make_tiling(col_rows=cr, zfuse=zf))
    s3 = mk(3)
    t3 = s3.tiling()
    assert t3[5] == 3
    s1 = mk(1, t3[4])          # the same column segments in three launches
    assert s1.tiling()[5] == 1 and s1.tiling()[:5] == t3[:5]
    z1 = s1.linear_solve(khw_to_hwk(rhs))
    s3.set_profiling(True)
    z3 = s3.linear_solve(khw_to_hwk(rhs))
    st = s3.kernel_stats()
    assert st["zupdate_fused"][0] == 1
    assert st["row_fft_forward"][0] == st["column_solve"][0] == st["row_fft_inverse"][0] == 0
    assert np.array_equal(z1, z3)
    assert max_abs(hwk_to_khw(z3), ref) <= tol * np.abs(ref).max()
    # a second launch on the same handle: the counters were returned to zero
    z3b = s3.linear_solve(khw_to_hwk(rhs))
    assert np.array_equal(z3, z3b)
    s1.close()
    s3.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_solve_one_launch_bitwise(B, prec):
    """Whole solves (CUDA-graph replay, a traced iteration every 10) with the one-launch
    z-update and with three launches: identical iterates and trace, and the oracle's iterate."""
    sc = synth.scene(145, 145, 16, S=40, gap=2.0, noise_std=1.5, wrong_frac=0.05, seed=2)
    dt = np.float64 if prec == "fp64" else np.float32
    out, tr = [], []
    for zf in (3, 1):
        s = B.Solver(B.make_params(145, 145, 16, M=1, sigma=0.5, lam=1.5, mu=1.0, schatten_p=1,
                                   precision=prec), tiling=B.make_tiling(zfuse=zf))
        assert s.tiling()[5] == zf
        s.set_probs(sc.p.astype(dt))
        tr.append(s.solve(60, trace_every=10))
        out.append(s.get_z())
        s.close()
    assert np.array_equal(out[0], out[1])
    assert np.array_equal(np.asarray(tr[0]), np.asarray(tr[1]))
    ref, _ = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 1, 60)
    assert max_abs(out[0], ref.z) < (1e-9 if prec == "fp64" else 1e-4)


def test_concurrent_handles_one_launch(B):
    """Four handles with the one-launch z-update solving at the same time on four streams (each
    handle has its own ticket counters): every result equals the same solve run alone."""
    scs = [synth.scene(96 + 8 * i, 80 + 4 * i, 8, S=12, gap=2.0, noise_std=1.0, wrong_frac=0.0,
                       seed=60 + i) for i in range(4)]
    alone = []
    for sc in scs:
        s = B.Solver(B.make_params(sc.H, sc.W, sc.K, M=1, sigma=0.5), tiling=B.make_tiling(zfuse=3))
        s.set_probs(sc.p.astype(np.float32))
        s.solve(200)
        alone.append(s.get_z())
        s.close()
    streams = [torch.cuda.Stream() for _ in scs]
    hs = []
    for sc, stm in zip(scs, streams):
        pr = B.make_params(sc.H, sc.W, sc.K, M=1, sigma=0.5)
        pr.stream = stm.cuda_stream
        s = B.Solver(pr, tiling=B.make_tiling(zfuse=3))
        s.set_probs(sc.p.astype(np.float32))
        hs.append(s)
    torch.cuda.synchronize()
    for s in hs:                      # solve() returns after its stream is done: run the
        s.solve(10)                   # graphs once first, then overlap the long solves
    import threading
    th = [threading.Thread(target=s.solve, args=(190,)) for s in hs]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for s, z in zip(hs, alone):
        assert np.array_equal(s.get_z(), z)
        s.close()


def test_one_launch_wait_runs_out(B):
    """With the wait probe on, the column units wait for one forward unit more than exists:
    the bounded wait gives up, linear_solve reports SEGSALSA_ERR_TIMEOUT, the counters are
    reset, and with the probe off the same handle solves correctly again."""
    H, W, K = 48, 40, 8
    rhs = synth.random_field((K, H, W), seed=5).astype(np.float32)
    s = B.Solver(B.make_params(H, W, K, M=1, sigma=0.5), tiling=B.make_tiling(zfuse=3))
    z0 = s.linear_solve(khw_to_hwk(rhs))
    s.set_wait_budget(200_000, probe=True)
    with pytest.raises(B.SegsalsaError) as e:
        s.linear_solve(khw_to_hwk(rhs))
    assert e.value.code == B.SEGSALSA_ERR_TIMEOUT
    s.set_wait_budget(2_000_000_000, probe=False)
    for _ in range(3):
        assert np.array_equal(s.linear_solve(khw_to_hwk(rhs)), z0)
    s.close()


def test_batch_one_launch_matches_single_handles(B):
    """A batch whose images use the one-launch z-update reproduces single handles bit for
    bit (lanes run images concurrently, each with its own counters)."""
    scs = [synth.scene(h, w, k, S=8, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=80 + i)
           for i, (h, w, k) in enumerate([(64, 64, 4), (100, 90, 8), (145, 145, 16), (33, 47, 5)])]
    prs = [B.make_params(sc.H, sc.W, sc.K, M=1, sigma=0.5) for sc in scs]
    bt = B.Batch(prs, tilings=[B.make_tiling(zfuse=3) for _ in scs])
    bt.set_lanes(3)
    for i, sc in enumerate(scs):
        bt.image(i).set_probs(sc.p.astype(np.float32))
    bt.solve(130)
    for i, sc in enumerate(scs):
        s = B.Solver(B.make_params(sc.H, sc.W, sc.K, M=1, sigma=0.5), tiling=B.make_tiling(zfuse=3))
        s.set_probs(sc.p.astype(np.float32))
        s.solve(130)
        assert np.array_equal(bt.image(i).get_z(), s.get_z()), i
        s.close()
    bt.close()
