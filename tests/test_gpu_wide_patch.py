"""Wide patches (M = 3, 4, 5: the 7x7, 9x9 and 11x11 patches of Sec. 5's patch-size study) run
the two-launch sweep (per-pixel Gram and prox coefficients, then the J^T gather over target
tiles). Parity with the FP64 oracle: one step from an oracle state (d and rhs of eqs. 12-14),
whole solves with traces, the simplex variant of g4, checkpoints and batches."""
import numpy as np
import pytest

from oracle import segsalsa_str_oracle as O
from paper_1504_07028_gb300 import synth
from tests.helpers import (d2_abi_to_oracle, hwk_to_khw, label_agreement, max_abs,
                           oracle_state_to_abi)

pytestmark = pytest.mark.gpu

SP = {1: 1, 2: 2, "inf": np.inf}


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_07028_gb300 import binding
    return binding


def _solver(B, H, W, K, M, sigma, lam, mu, sp, prec):
    return B.Solver(B.make_params(H, W, K, M=M, sigma=sigma, lam=lam, mu=mu, schatten_p=sp,
                                  precision=prec))


@pytest.mark.parametrize("H,W,K,M,sp,prec", [
    (21, 37, 5, 3, 1, "fp64"), (21, 37, 5, 3, 1, "fp32"), (24, 19, 4, 4, 2, "fp64"),
    (18, 26, 8, 5, "inf", "fp64"), (18, 26, 8, 5, 1, "fp32"), (12, 12, 3, 5, 1, "fp64"),
    (33, 40, 16, 3, "inf", "fp32"), (17, 13, 32, 3, 2, "fp32")])
def test_wide_sweep_step(B, H, W, K, M, sp, prec):
    """From an oracle state (z^k, d^k) one GPU sweep (set_state with k = 0 skips the z-update)
    gives the oracle's d^{k+1} and G^T(u^{k+1} + d^{k+1})."""
    sc = synth.scene(H, W, K, S=4, gap=2.0, noise_std=1.0, wrong_frac=0.05, seed=H * W + M)
    sigma, lam, mu = 0.5 * M, 1.5, 1.3
    om = O.gaussian_weights(M, sigma)
    dt = np.float64 if prec == "fp64" else np.float32
    p = sc.p.astype(dt).astype(np.float64)
    st, _ = O.solve(p, M, sigma, lam, mu, SP[sp], 5, omega=om)
    s = _solver(B, H, W, K, M, sigma, lam, mu, SP[sp], prec)
    s.set_probs(p.astype(dt))
    a = oracle_state_to_abi(st, om, M, dt)
    a["rhs"] = None
    s.set_state(a, 0)
    s.solve(1)
    g = s.get_state()
    z = a["z"].astype(np.float64).transpose(2, 0, 1)
    d = [np.asarray(x, np.float64) for x in (hwk_to_khw(a["d1"]), d2_abi_to_oracle(a["d2"]),
                                             hwk_to_khw(a["d3"]), hwk_to_khw(a["d4"]))]
    u, dn, _ = O.u_d_update(z, d, p, lam, mu, om, M, SP[sp])
    rhs = O.apply_GT([x + y for x, y in zip(u, dn)], om, M)
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert max_abs(hwk_to_khw(g["d1"]), dn[0]) <= tol
    assert max_abs(d2_abi_to_oracle(g["d2"]), dn[1]) <= tol
    assert max_abs(hwk_to_khw(g["d3"]), dn[2]) <= tol
    assert max_abs(hwk_to_khw(g["d4"]), dn[3]) <= tol
    assert max_abs(hwk_to_khw(g["rhs"]), rhs) <= 8 * tol * max(1.0, np.abs(rhs).max())
    s.close()


@pytest.mark.parametrize("M,K,sp,prec", [(3, 4, 1, "fp64"), (3, 8, 1, "fp32"), (5, 4, 2, "fp32"),
                                         (4, 6, "inf", "fp64")])
def test_wide_full_solve_against_oracle(B, M, K, sp, prec):
    H, W = 30, 34
    sc = synth.scene(H, W, K, S=5, gap=2.0, noise_std=1.0, wrong_frac=0.05, seed=100 + M + K)
    dt = np.float64 if prec == "fp64" else np.float32
    p = sc.p.astype(dt)
    sigma, lam = 0.5 * M, 1.5
    s = _solver(B, H, W, K, M, sigma, lam, 1.0, SP[sp], prec)
    s.set_probs(p)
    tr = s.solve(40, trace_every=10)
    z = s.get_z()
    s.close()
    ref, rtr = O.solve(p.astype(np.float64), M, sigma, lam, 1.0, SP[sp], 40, trace_every=10)
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert max_abs(z, ref.z) <= tol
    ok, _ = label_agreement(z, ref.z)
    assert ok
    rt = 1e-7 if prec == "fp64" else 2e-3
    assert np.allclose(tr[:, 1:4], rtr[:, 1:4], rtol=rt, atol=1e-6 if prec == "fp32" else 1e-10)


def test_wide_simplex_g4_against_oracle(B):
    H, W, K, M = 26, 22, 5, 3
    sc = synth.scene(H, W, K, S=4, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=131)
    s = _solver(B, H, W, K, M, 1.5, 1.2, 1.0, 1, "fp64")
    s.set_g4("simplex")
    s.set_probs(sc.p)
    s.solve(25)
    z = s.get_z()
    s.close()
    ref, _ = O.solve(sc.p, M, 1.5, 1.2, 1.0, 1, 25, g4="simplex")
    assert max_abs(z, ref.z) <= 1e-9


def test_wide_checkpoint_resume(B):
    """set_state with k > 0 (dense rhs given), then one full iteration."""
    H, W, K, M, sigma, lam, mu = 20, 27, 4, 4, 2.0, 1.5, 1.0
    sc = synth.scene(H, W, K, S=4, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=132)
    om = O.gaussian_weights(M, sigma)
    st, _ = O.solve(sc.p, M, sigma, lam, mu, 1, 4, omega=om)
    nxt, _, _ = O.salsa_step(st, sc.p, lam, mu, om, M, 1)
    s = _solver(B, H, W, K, M, sigma, lam, mu, 1, "fp64")
    s.set_probs(sc.p)
    s.set_state(oracle_state_to_abi(st, om, M, np.float64), st.k)
    s.solve(1)
    g = s.get_state()
    assert max_abs(hwk_to_khw(g["z"]), nxt.z) <= 1e-10
    assert max_abs(d2_abi_to_oracle(g["d2"]), nxt.d[1]) <= 1e-10
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_wide_state_round_trip_is_exact(B, prec):
    """The wide sweep keeps the prior's dual as (V, A) with d2 = V (A - I). get_state writes d2
    out, set_state loads it back as V = d2, A = 2I; a handle resumed from the checkpoint must
    continue bit for bit like the original (traced iterations included)."""
    H, W, K, M, sigma = 26, 23, 5, 3, 1.5
    sc = synth.scene(H, W, K, S=4, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=133)
    dt = np.float64 if prec == "fp64" else np.float32
    a = _solver(B, H, W, K, M, sigma, 1.5, 1.0, 2, prec)
    a.set_probs(sc.p.astype(dt))
    a.solve(7, trace_every=3)
    st = a.get_state()
    b = _solver(B, H, W, K, M, sigma, 1.5, 1.0, 2, prec)
    b.set_probs(sc.p.astype(dt))
    b.set_state(st, a.get_iteration())
    ta = a.solve(9, trace_every=3)
    tb = b.solve(9, trace_every=3)
    assert np.array_equal(a.get_z(), b.get_z())
    assert np.array_equal(a.get_state()["d2"], b.get_state()["d2"])
    assert np.array_equal(np.asarray(ta)[:, 1:], np.asarray(tb)[:, 1:])
    a.close()
    b.close()


def test_wide_and_narrow_patches_in_one_batch(B):
    cases = [(24, 30, 4, 1), (28, 21, 5, 3), (22, 25, 4, 5)]
    scenes = [synth.scene(H, W, K, S=4, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=140 + j)
              for j, (H, W, K, M) in enumerate(cases)]
    bt = B.Batch([B.make_params(H, W, K, M=M, sigma=0.5 * max(M, 1), lam=1.5)
                  for (H, W, K, M) in cases])
    for j, sc in enumerate(scenes):
        bt.image(j).set_probs(sc.p.astype(np.float32))
    bt.solve(30)
    for j, ((H, W, K, M), sc) in enumerate(zip(cases, scenes)):
        ref, _ = O.solve(sc.p.astype(np.float32).astype(np.float64), M, 0.5 * max(M, 1), 1.5,
                         1.0, 1, 30)
        assert max_abs(bt.image(j).get_z(), ref.z) < 1e-4, j
    bt.close()


def test_wide_rejects_the_reverse_pass(B):
    sc = synth.scene(14, 14, 3, S=3, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=150)
    s = _solver(B, 14, 14, 3, 3, 1.5, 1.5, 1.0, 1, "fp64")
    s.set_log_probs(np.log(sc.p))
    with pytest.raises(B.SegsalsaError) as e:
        s.backward(3, np.ones((3, 14, 14)), 1)
    assert e.value.code == B.SEGSALSA_ERR_ARG
    s.close()
