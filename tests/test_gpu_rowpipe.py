"""The pipelined row passes (persistent CTAs that copy the next unit's input into shared memory
while transforming the current one) against the one-unit-per-CTA row passes and the oracle's
DFT solve of the z-update (eq. 12). Same kernels' arithmetic, same order of the partial sums:
the iterates must be identical; the solve of a dense rhs must match the oracle."""
import numpy as np
import pytest

from oracle import segsalsa_str_oracle as O
from paper_1504_07028_gb300 import synth
from tests.helpers import hwk_to_khw, khw_to_hwk, max_abs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_07028_gb300 import binding
    return binding


def _pair(B, H, W, K, M, prec, row_pairs=0, lam=1.5):
    mk = lambda pipe: B.Solver(B.make_params(H, W, K, M=M, sigma=0.5 + 0.5 * M, lam=lam, mu=1.0,
                                             precision=prec),
                               tiling=B.make_tiling(row_pipe=pipe, row_pairs=row_pairs))
    s1, s2 = mk(1), mk(2)
    assert s1.tiling()[6] == 1 and s2.tiling()[6] == 2
    return s1, s2


@pytest.mark.parametrize("H,W,K,M,prec,rp", [
    (40, 256, 8, 1, "fp32", 0),     # 256-point rows, the default pair count
    (37, 512, 16, 1, "fp32", 1),    # one pair per CTA: 8-byte loads and stores
    (29, 1024, 16, 1, "fp32", 2),   # radix 8, 8, 8, 2
    (45, 2048, 16, 1, "fp32", 2),   # radix 8, 8, 8, 4 (the 2048 x 2048 workload's rows)
    (21, 2048, 8, 2, "fp32", 4),    # four pairs per CTA, 5x5 patch: one buffer, stages in place
    (27, 2048, 16, 1, "fp32", 4),   # the 2048 x 2048 workload's row CTAs (one buffer)
    (19, 4096, 4, 1, "fp32", 1),    # 4096-point rows
    (13, 4096, 4, 1, "fp32", 2),    # 4096-point rows, two pairs: one buffer, stages in place
    (23, 512, 8, 1, "fp64", 2),     # FP64: 16-byte pairs
    (17, 1024, 4, 0, "fp64", 1),
    (9, 4096, 4, 1, "fp64", 1),     # FP64 4096-point rows (radix-8 last stage)
])
def test_power_of_two_row_passes_match(B, H, W, K, M, prec, rp):
    """Form 3 (compile-time plan, first stage fused into the load) against form 1: the
    iterates of a traced solve are identical."""
    sc = synth.scene(H, W, K, S=5, gap=2.0, noise_std=1.0, wrong_frac=0.05, seed=H + W + K + 7)
    dt = np.float64 if prec == "fp64" else np.float32
    p = sc.p.astype(dt)
    mk = lambda pipe: B.Solver(B.make_params(H, W, K, M=M, sigma=0.5 + 0.5 * M, lam=1.5, mu=1.0,
                                             precision=prec),
                               tiling=B.make_tiling(row_pipe=pipe, row_pairs=rp))
    s1, s3 = mk(1), mk(3)
    assert s1.tiling()[6] == 1 and s3.tiling()[6] == 3
    out = []
    for s in (s1, s3):
        s.set_probs(p)
        tr = s.solve(12, trace_every=4)
        out.append((s.get_z(), tr))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_power_of_two_linear_solve_against_oracle(B, prec):
    H, W, K = 33, 1024, 8
    dt = np.float64 if prec == "fp64" else np.float32
    rhs = synth.random_field((K, H, W), seed=77).astype(dt)
    s = B.Solver(B.make_params(H, W, K, M=1, sigma=0.5, precision=prec),
                 tiling=B.make_tiling(row_pipe=3))
    assert s.tiling()[6] == 3
    z = hwk_to_khw(s.linear_solve(khw_to_hwk(rhs)))
    s.close()
    ref = O.linear_solve(rhs.astype(np.float64), O.gaussian_weights(1, 0.5), 1)
    tol = 1e-11 if prec == "fp64" else 2e-5
    assert max_abs(z, ref) <= tol * np.abs(ref).max()


@pytest.mark.parametrize("H,W,K,M,prec,rp", [
    (40, 37, 8, 1, "fp32", 0),      # direct prime row (37), small image
    (33, 127, 5, 1, "fp32", 0),     # Bluestein row, odd K (element-wise copies, zero fill)
    (29, 509, 4, 1, "fp32", 0),     # Bluestein row, vector copies
    (61, 2048, 16, 1, "fp32", 2),   # long rows, two class pairs: one stage slot
    (45, 2048, 16, 1, "fp32", 1),   # long rows, one class pair: two stage slots
    (50, 96, 16, 2, "fp32", 4),     # 5x5 patch (wider halos), four class pairs per unit
    (31, 145, 16, 1, "fp64", 0),    # FP64
    (26, 64, 3, 0, "fp64", 0),      # 1x1 patch, odd K
])
def test_pipelined_row_passes_match(B, H, W, K, M, prec, rp):
    sc = synth.scene(H, W, K, S=5, gap=2.0, noise_std=1.0, wrong_frac=0.05, seed=H + W + K)
    dt = np.float64 if prec == "fp64" else np.float32
    p = sc.p.astype(dt)
    s1, s2 = _pair(B, H, W, K, M, prec, rp)
    zs = []
    for s in (s1, s2):
        s.set_probs(p)
        tr = s.solve(12, trace_every=4)
        zs.append((s.get_z(), tr))
        s.close()
    assert np.array_equal(zs[0][0], zs[1][0])
    assert np.array_equal(zs[0][1], zs[1][1])


@pytest.mark.parametrize("H,W,K,prec", [(48, 2048, 16, "fp32"), (37, 131, 6, "fp32"),
                                        (20, 206, 4, "fp64")])
def test_pipelined_linear_solve_dense_rhs(B, H, W, K, prec):
    dt = np.float64 if prec == "fp64" else np.float32
    rhs = synth.random_field((K, H, W), seed=H * 7 + W).astype(dt)
    s1, s2 = _pair(B, H, W, K, 1, prec)
    z1 = hwk_to_khw(s1.linear_solve(khw_to_hwk(rhs)))
    z2 = hwk_to_khw(s2.linear_solve(khw_to_hwk(rhs)))
    s1.close()
    s2.close()
    assert np.array_equal(z1, z2)
    ref = O.linear_solve(rhs.astype(np.float64), O.gaussian_weights(1, 1.0), 1)
    tol = 1e-11 if prec == "fp64" else 2e-5
    assert max_abs(z2, ref) <= tol * np.abs(ref).max()


def test_pipelined_full_solve_against_oracle(B):
    """A whole solve with the pipelined passes ends within 1e-4 of the oracle."""
    from tests.helpers import label_agreement
    sc = synth.scene(36, 150, 8, S=6, gap=2.0, noise_std=1.0, wrong_frac=0.05, seed=91)
    p = sc.p.astype(np.float32)
    s = B.Solver(B.make_params(sc.H, sc.W, sc.K, M=1, sigma=0.5, lam=1.5, mu=1.0),
                 tiling=B.make_tiling(row_pipe=2))
    s.set_probs(p)
    s.solve(60)
    z = s.get_z()
    s.close()
    ref, _ = O.solve(p.astype(np.float64), 1, 0.5, 1.5, 1.0, 1, 60)
    assert max_abs(z, ref.z) < 1e-4
    ok, _ = label_agreement(z, ref.z)
    assert ok
