"""The differentiable solver (segsalsa_str_backward) against the oracle's reference gradient
(FP64 autograd through a transcription of the oracle iteration) and against FP64 central
finite differences of the GPU forward pass itself (step 1e-6).

Tolerances: the FP64 reverse pass agrees with the reference to rounding (1e-8 of the largest
gradient entry); the FP32 pass accumulates FP32 rounding over the unrolled iterations and is
held to 2e-3 of the largest entry."""
import numpy as np
import pytest

from oracle import segsalsa_str_oracle as O
from oracle import unrolled_grad as U
from paper_1504_07028_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_07028_gb300 import binding
    return binding


def _mk(B, H, W, K, M, sp, prec, lam=1.2, sigma=None):
    return B.Solver(B.make_params(H, W, K, M=M, sigma=sigma or (0.5 if M <= 1 else 1.0),
                                  lam=lam, mu=1.0, schatten_p=sp, precision=prec))


def _case(H, W, K, seed):
    sc = synth.scene(H, W, K, S=3, gap=1.5, noise_std=1.0, wrong_frac=0.1, seed=seed)
    return np.log(sc.p), np.random.default_rng(seed + 1).normal(size=(K, H, W))


@pytest.mark.parametrize("H,W,K,M,sp,T,C", [(12, 14, 3, 1, 1, 7, 3), (10, 9, 4, 0, 2, 6, 4),
                                            (11, 13, 5, 2, 1, 5, 2), (9, 16, 9, 1, 2, 8, 10),
                                            (10, 10, 2, 1, 1, 1, 1)])
def test_fp64_backward_matches_reference(B, H, W, K, M, sp, T, C):
    logp, zbar = _case(H, W, K, 70 + H + K)
    s = _mk(B, H, W, K, M, sp, "fp64")
    om = O.gaussian_weights(M, 0.5 if M <= 1 else 1.0)
    s.set_log_probs(logp)
    g, glam, gom = s.backward(T, zbar, checkpoint_every=C)
    r_lp, r_lam, r_om, r_z = U.reference_gradient(logp, 1.2, om, M, 1.0, sp, T, zbar)
    scale = max(np.abs(r_lp).max(), abs(r_lam), np.abs(r_om).max())
    assert np.abs(g - r_lp).max() < 1e-8 * scale
    assert abs(glam - r_lam) < 1e-8 * scale
    assert np.abs(gom - r_om).max() < 1e-8 * scale
    # the handle ends at iteration T with the forward state
    assert s.get_iteration() == T
    assert np.abs(s.get_z() - r_z).max() < 1e-10
    s.close()


def test_checkpoint_interval_does_not_change_the_gradient(B):
    logp, zbar = _case(13, 12, 4, 80)
    s = _mk(B, 13, 12, 4, 1, 1, "fp64")
    s.set_log_probs(logp)
    outs = [s.backward(9, zbar, checkpoint_every=c) for c in (1, 3, 4, 50)]
    for g, glam, gom in outs[1:]:
        # recomputation is deterministic: d/dlog p is bit for bit the same; the lambda and
        # omega sums gather FP64 block partials whose in-block order is not fixed
        assert np.array_equal(g, outs[0][0])
        assert abs(glam - outs[0][1]) <= 1e-12 * abs(outs[0][1])
        assert np.allclose(gom, outs[0][2], rtol=1e-12, atol=0)
    s.close()


def test_fp32_backward_close_to_fp64(B):
    logp, zbar = _case(24, 20, 6, 81)
    out = {}
    for prec, dt in (("fp64", np.float64), ("fp32", np.float32)):
        s = _mk(B, 24, 20, 6, 1, 1, prec)
        s.set_log_probs(logp.astype(dt))
        out[prec] = s.backward(12, zbar.astype(dt), checkpoint_every=5)
        s.close()
    g64, l64, o64 = out["fp64"]
    g32, l32, o32 = out["fp32"]
    scale = max(np.abs(g64).max(), abs(l64), np.abs(o64).max())
    assert np.abs(g32 - g64).max() < 2e-3 * scale
    assert abs(l32 - l64) < 2e-3 * scale and np.abs(o32 - o64).max() < 2e-3 * scale


@pytest.mark.parametrize("H,W,K,M,sp,g4,T,C", [
    (12, 14, 3, 1, "inf", "affine", 7, 3), (11, 13, 5, 2, "inf", "affine", 5, 2),
    (12, 14, 3, 1, 1, "simplex", 7, 3), (10, 9, 4, 0, 2, "simplex", 6, 4),
    (9, 16, 9, 1, "inf", "simplex", 8, 10)])
def test_fp64_backward_inf_and_simplex_match_reference(B, H, W, K, M, sp, g4, T, C):
    """Schatten p = infinity (the Moreau form of the prox) and g4 on the probability simplex
    (active set recomputed in the reverse pass) against the reference gradient; in the simplex
    cases classes leave the active set (the affine-set gradient differs)."""
    logp, zbar = _case(H, W, K, 90 + H + K)
    s = _mk(B, H, W, K, M, sp, "fp64")
    if g4 == "simplex":
        s.set_g4("simplex")
    om = O.gaussian_weights(M, 0.5 if M <= 1 else 1.0)
    s.set_log_probs(logp)
    g, glam, gom = s.backward(T, zbar, checkpoint_every=C)
    spo = np.inf if sp == "inf" else sp
    r_lp, r_lam, r_om, r_z = U.reference_gradient(logp, 1.2, om, M, 1.0, spo, T, zbar, g4)
    scale = max(np.abs(r_lp).max(), abs(r_lam), np.abs(r_om).max())
    assert np.abs(g - r_lp).max() < 1e-8 * scale
    assert abs(glam - r_lam) < 1e-8 * scale
    assert np.abs(gom - r_om).max() < 1e-8 * scale
    assert s.get_iteration() == T
    assert np.abs(s.get_z() - r_z).max() < 1e-10
    if g4 == "simplex":   # the active set matters: the affine-set gradient is another one
        a_lp = U.reference_gradient(logp, 1.2, om, M, 1.0, spo, T, zbar, "affine")[0]
        assert np.abs(a_lp - r_lp).max() > 1e-3 * scale
    s.close()


def test_fp32_backward_inf_simplex_close_to_fp64(B):
    logp, zbar = _case(24, 20, 6, 86)
    out = {}
    for prec, dt in (("fp64", np.float64), ("fp32", np.float32)):
        s = _mk(B, 24, 20, 6, 1, "inf", prec)
        s.set_g4("simplex")
        s.set_log_probs(logp.astype(dt))
        out[prec] = s.backward(12, zbar.astype(dt), checkpoint_every=5)
        s.close()
    g64, l64, o64 = out["fp64"]
    g32, l32, o32 = out["fp32"]
    scale = max(np.abs(g64).max(), abs(l64), np.abs(o64).max())
    assert np.abs(g32 - g64).max() < 2e-3 * scale
    assert abs(l32 - l64) < 2e-3 * scale and np.abs(o32 - o64).max() < 2e-3 * scale


def test_backward_rejects_unsupported(B):
    logp, zbar = _case(14, 14, 3, 82)
    s = _mk(B, 8, 8, 3, 1, 1, "fp64")
    s.set_log_probs(np.ascontiguousarray(logp[:, :8, :8]))
    with pytest.raises(B.SegsalsaError) as e:
        s.backward(0, np.ascontiguousarray(zbar[:, :8, :8]))
    assert e.value.code == B.SEGSALSA_ERR_ARG
    s.close()
    s = _mk(B, 14, 14, 3, 3, 1, "fp64", sigma=1.5)
    s.set_log_probs(logp)
    with pytest.raises(B.SegsalsaError) as e:
        s.backward(3, zbar)
    assert e.value.code == B.SEGSALSA_ERR_ARG
    s.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("fp32", 2e-3)])
def test_50_iterations_with_checkpoints_match_reference(B, prec, tol):
    """Schatten p = 1, K = 8, 50 iterations, a checkpoint every 10 (the differentiable-solver
    setting) on a 64x64 image, against the reference gradient."""
    H = W = 64
    K, T = 8, 50
    sc = synth.scene(H, W, K, S=6, gap=3.0, noise_std=1.0, wrong_frac=0.0, seed=5)
    logp = np.log(sc.p)
    zbar = np.random.default_rng(85).normal(size=(K, H, W))
    dt = np.float64 if prec == "fp64" else np.float32
    s = _mk(B, H, W, K, 1, 1, prec, lam=2.0)
    s.set_log_probs(logp.astype(dt))
    g, glam, gom = s.backward(T, zbar.astype(dt), checkpoint_every=10)
    r_lp, r_lam, r_om, _ = U.reference_gradient(logp.astype(dt).astype(np.float64), 2.0,
                                                O.gaussian_weights(1, 0.5), 1, 1.0, 1, T, zbar)
    scale = max(np.abs(r_lp).max(), abs(r_lam), np.abs(r_om).max())
    assert np.abs(g - r_lp).max() < tol * scale
    assert abs(glam - r_lam) < tol * scale and np.abs(gom - r_om).max() < tol * scale
    s.close()


def test_differentiable_solver_at_256x256_against_finite_differences(B):
    """The 256x256, K=8, 50-iteration unrolled solve with checkpoints every 10: the FP64
    reverse pass against central differences (step 1e-6) of the FP64 GPU forward pass for
    lambda, one shift weight and a random direction in log p; the FP32 reverse pass within
    2e-3 of the FP64 one; zero per-pixel sum of d/dlog p (scale invariance). The iteration is
    piecewise smooth (u3 = max(v3, 0) on half a million components near 0, the case switches of
    the Schatten prox), and a step of 1e-6 can cross a switch on one side: a check passes when
    the central difference or the one-sided difference on one side agrees (both one-sided
    differences and the central one agree wherever no switch lies within the step). Schatten
    p = 2 here; the p = 1 setting is checked against the reference gradient above."""
    import torch
    from paper_1504_07028_gb300.autograd import UnrolledSegSalsa
    H = W = 256
    K, T, h = 8, 50, 1e-6
    sc = synth.scene(H, W, K, S=16, gap=3.0, noise_std=1.0, wrong_frac=0.0, seed=4)
    logp = np.log(sc.p)
    zbar = np.random.default_rng(83).normal(size=(K, H, W))
    om = O.gaussian_weights(1, 0.5)
    s64 = _mk(B, H, W, K, 1, 2, "fp64", lam=2.0)
    s64.set_log_probs(logp)
    g, glam, gom = s64.backward(T, zbar, checkpoint_every=10)
    assert np.abs(g.sum(axis=0)).max() < 1e-9 * np.abs(g).max()

    def loss(lp=logp, lam=2.0, w=om):
        s64.set_lambda(lam)
        s64.set_weights(w)
        s64.set_log_probs(lp)
        s64.solve(T)
        return float(np.sum(zbar * s64.get_z()))
    f0 = loss()

    def agrees(fp, fm, grad):
        cands = ((fp - fm) / (2 * h), (fp - f0) / h, (f0 - fm) / h)
        return min(abs(c - grad) for c in cands) < 1e-5 * max(1.0, abs(grad)), cands

    ok, c = agrees(loss(lam=2.0 + h), loss(lam=2.0 - h), glam)
    assert ok, (c, glam)
    e = np.zeros_like(om)
    e[2] = h
    ok, c = agrees(loss(w=om + e), loss(w=om - e), gom[2])
    assert ok, (c, gom[2])
    dirn = np.random.default_rng(84).normal(size=logp.shape)
    ok, c = agrees(loss(lp=logp + h * dirn), loss(lp=logp - h * dirn), np.sum(g * dirn))
    assert ok, (c, np.sum(g * dirn))
    s64.close()
    # FP32 reverse pass through the autograd wrapper, on device tensors
    s32 = _mk(B, H, W, K, 1, 2, "fp32", lam=2.0)
    lp_t = torch.tensor(logp, dtype=torch.float32, device="cuda", requires_grad=True)
    lam_t = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
    om_t = torch.tensor(om, dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    z = UnrolledSegSalsa.apply(lp_t, lam_t, om_t, s32, T, 10)
    (z * torch.tensor(zbar, dtype=torch.float32, device="cuda")).sum().backward()
    scale = max(np.abs(g).max(), abs(glam), np.abs(gom).max())
    assert np.abs(lp_t.grad.double().cpu().numpy() - g).max() < 2e-3 * scale
    assert abs(float(lam_t.grad) - glam) < 2e-3 * scale
    assert np.abs(om_t.grad.numpy() - gom).max() < 2e-3 * scale
    s32.close()
