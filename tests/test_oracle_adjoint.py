"""Pins of the reference gradient of the unrolled SALSA iteration (oracle/unrolled_grad.py):
its forward pass is the numpy oracle's iteration, and its gradient of <zbar, z^T> with respect
to log p, lambda and the shift weights matches FP64 central finite differences (step 1e-6)."""
import numpy as np
import pytest
import torch

from oracle import segsalsa_str_oracle as O
from oracle import unrolled_grad as U
from paper_1504_07028_gb300 import synth


def _case(H, W, K, seed):
    sc = synth.scene(H, W, K, S=3, gap=1.5, noise_std=1.0, wrong_frac=0.1, seed=seed)
    return np.log(sc.p), np.random.default_rng(seed + 1).normal(size=(K, H, W))


@pytest.mark.parametrize("M,sp,g4", [(1, 1, "affine"), (0, 2, "affine"), (1, 2, "affine"),
                                     (1, np.inf, "affine"), (2, np.inf, "affine"),
                                     (1, 1, "simplex"), (1, np.inf, "simplex")])
def test_forward_is_the_numpy_oracle(M, sp, g4):
    logp, _ = _case(9, 11, 3, 60)
    om = O.gaussian_weights(M, 0.5)
    z = U.unrolled(torch.tensor(logp), torch.tensor(1.2, dtype=torch.float64),
                   torch.tensor(om), M, 1.0, sp, 7, g4).numpy()
    ref, _ = O.solve(np.exp(logp), M, 0.5, 1.2, 1.0, sp, 7, omega=om, g4=g4)
    assert np.abs(z - ref.z).max() < 1e-12


def test_torch_projections_match_the_oracle():
    """The l1-ball and simplex projections of the reference against the numpy oracle's
    (themselves pinned against brute force in test_oracle_pins.py), both branches included."""
    rng = np.random.default_rng(64)
    s = -np.sort(-np.abs(rng.normal(size=(200, 2))), axis=-1) * 2.0
    for r in (0.3, 1.0, 4.0):
        assert np.abs(U.proj_l1_ball(torch.tensor(s), r).numpy() - O.proj_l1_ball(s, r)).max() < 1e-14
    v = rng.normal(size=(5, 7, 6)) * 1.5
    assert np.abs(U.proj_simplex(torch.tensor(v)).numpy() - O.proj_simplex(v)).max() < 1e-14


def _loss(logp, lam, om, M, sp, T, zbar, g4="affine"):
    with torch.no_grad():
        z = U.unrolled(torch.tensor(logp), torch.tensor(lam, dtype=torch.float64),
                       torch.tensor(om), M, 1.0, sp, T, g4)
    return float(np.sum(zbar * z.numpy()))


@pytest.mark.parametrize("M,sp,g4", [(1, 1, "affine"), (1, 2, "affine"), (1, np.inf, "affine"),
                                     (1, 1, "simplex"), (1, np.inf, "simplex")])
def test_gradient_matches_central_differences(M, sp, g4):
    T, lam, h = 6, 0.9, 1e-6
    logp, zbar = _case(8, 9, 3, 61)
    om = O.gaussian_weights(M, 0.5) * np.linspace(0.8, 1.2, (2 * M + 1) ** 2)
    g_lp, g_lam, g_om, _ = U.reference_gradient(logp, lam, om, M, 1.0, sp, T, zbar, g4)
    f = lambda lp=logp, la=lam, o=om: _loss(lp, la, o, M, sp, T, zbar, g4)
    fd = (f(la=lam + h) - f(la=lam - h)) / (2 * h)
    assert abs(fd - g_lam) < 1e-6 * max(1.0, abs(g_lam))
    for j in (0, len(om) // 2, len(om) - 1):
        e = np.zeros_like(om)
        e[j] = h
        fd = (f(o=om + e) - f(o=om - e)) / (2 * h)
        assert abs(fd - g_om[j]) < 1e-6 * max(1.0, abs(g_om[j]))
    dirn = np.random.default_rng(62).normal(size=logp.shape)
    fd = (f(lp=logp + h * dirn) - f(lp=logp - h * dirn)) / (2 * h)
    assert abs(fd - np.sum(g_lp * dirn)) < 1e-6 * max(1.0, abs(fd))


def test_log_p_gradient_sums_to_zero_per_pixel():
    """The iterates do not change when a pixel's p is scaled, so the gradient with respect to
    log p has zero sum over the classes of every pixel."""
    logp, zbar = _case(7, 8, 4, 63)
    g_lp, _, _, _ = U.reference_gradient(logp, 1.1, O.gaussian_weights(1, 0.5), 1, 1.0, 1, 5,
                                         zbar)
    assert np.abs(g_lp.sum(axis=0)).max() < 1e-12
    assert np.abs(g_lp).max() > 1e-4


@pytest.mark.parametrize("name,bad", [
    ("D_v_T", lambda g: torch.roll(g, shifts=-1, dims=-2) - g),          # wrong direction
    ("prox_g1", lambda v, p, mu: v + p / (mu * 0.5 * (torch.sum(p * v, 0) - torch.sqrt(
        torch.sum(p * v, 0) ** 2 + 4.0 * torch.sum(p * p, 0) / mu)))),   # negative root
])
def test_planted_mistakes_are_caught(monkeypatch, name, bad):
    monkeypatch.setattr(U, name, bad)
    with pytest.raises(AssertionError):
        test_forward_is_the_numpy_oracle(1, 1, "affine")


def test_planted_l1_threshold_mistake_is_caught(monkeypatch):
    """A threshold search that drops the division by the active count (theta = css - r)."""
    def bad(u, radius):
        css = torch.cumsum(u, dim=-1)
        j = torch.arange(1, u.shape[-1] + 1, dtype=U.DT)
        rho = torch.sum(u - (css - radius) / j > 0, dim=-1, keepdim=True)
        return torch.gather(css, -1, rho - 1) - radius
    monkeypatch.setattr(U, "_threshold_sorted", bad)
    with pytest.raises(AssertionError):
        test_forward_is_the_numpy_oracle(1, np.inf, "affine")
