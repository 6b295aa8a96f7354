"""Reference gradient of the unrolled SALSA iteration, for the differentiable solver.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or execute this file:
only the tests and the CPU-baseline legs of ``bench.py`` do.

The SALSA iteration (12)-(14) of ``segsalsa_str_oracle`` is written out again with plain
PyTorch CPU operations in FP64, step for step in the same order (explicit J and J^T by
``torch.roll``, the z-update by the DFT of the impulse response of J^T J, the Schatten prox by
``torch.linalg.svd``), so that ``torch.autograd`` gives the exact derivative of z^T with
respect to log p, lambda and the shift weights omega. It shares no code with the CUDA path.

Scope: Schatten p in {1, 2, infinity} (for p = infinity the singular values are shrunk by
the Moreau decomposition s - proj_{tau B_1}(s), the l1-ball projection by its sort-based
threshold) and g4 on the affine set (eq. 10) or on the probability simplex (the sort-based
threshold again). The derivative is the one autograd takes through these piecewise-smooth
maps, defined wherever no threshold is hit exactly. Pinned in tests/test_oracle_adjoint.py
against the numpy oracle's iterates and against FP64 central finite differences.
"""
from __future__ import annotations

import numpy as np
import torch

from oracle import segsalsa_str_oracle as O

DT = torch.float64


def _roll(f, sy, sx):
    return torch.roll(f, shifts=(sy, sx), dims=(-2, -1))


def D_h(f):
    return _roll(f, 0, -1) - f


def D_v(f):
    return _roll(f, -1, 0) - f


def D_h_T(g):
    return _roll(g, 0, 1) - g


def D_v_T(g):
    return _roll(g, 1, 0) - g


def shift(f, s):
    return _roll(f, -s[0], -s[1])


def shift_T(g, s):
    return _roll(g, s[0], s[1])


def jacobian(z, omega, M):
    """(L, K, 2, H, W): [j, k, 0] = omega_j S_j D_h z_k, [j, k, 1] = omega_j S_j D_v z_k (eq. 4)."""
    dh, dv = D_h(z), D_v(z)
    return torch.stack([torch.stack([omega[j] * shift(dh, s), omega[j] * shift(dv, s)], dim=1)
                        for j, s in enumerate(O.patch_shifts(M))])


def jacobian_T(w, omega, M):
    out = torch.zeros(w.shape[1:2] + w.shape[3:], dtype=DT)
    for j, s in enumerate(O.patch_shifts(M)):
        out = out + omega[j] * (D_h_T(shift_T(w[j, :, 0], s)) + D_v_T(shift_T(w[j, :, 1], s)))
    return out


def apply_G(z, omega, M):
    return [z, jacobian(z, omega, M), z, z]


def apply_GT(x, omega, M):
    return x[0] + jacobian_T(x[1], omega, M) + x[2] + x[3]


def linear_solve(rhs, omega, M):
    """(3 I + J^T J)^{-1} rhs by the DFT of the impulse response of J^T J (eq. 12)."""
    K, H, W = rhs.shape
    delta = torch.zeros((1, H, W), dtype=DT)
    delta[0, 0, 0] = 1.0
    h = jacobian_T(jacobian(delta, omega, M), omega, M)[0]
    den = 3.0 + torch.fft.fft2(h).real
    return torch.fft.ifft2(torch.fft.fft2(rhs) / den).real


def prox_g1(v, p, mu):
    a = torch.sum(p * v, dim=0)
    b = torch.sum(p * p, dim=0)
    s = 0.5 * (a + torch.sqrt(a * a + 4.0 * b / mu))
    return v + p / (mu * s)


def _threshold_sorted(u, radius):
    """theta with sum_i max(u_i - theta, 0) = radius for rows u (last axis) sorted in
    descending order and sum u > radius: the sort-based threshold search (Held, Wolfe,
    Crowder 1974; Duchi et al. 2008)."""
    q = u.shape[-1]
    css = torch.cumsum(u, dim=-1)
    j = torch.arange(1, q + 1, dtype=DT)
    cond = u - (css - radius) / j > 0            # true on a prefix of the sorted row
    rho = torch.sum(cond, dim=-1, keepdim=True)
    return (torch.gather(css, -1, rho - 1) - radius) / rho


def proj_l1_ball(s, radius):
    """Projection of rows of non-negative values s (last axis, descending: singular values)
    onto {||y||_1 <= radius}."""
    y = torch.relu(s - _threshold_sorted(s, radius))
    return torch.where(torch.sum(s, dim=-1, keepdim=True) <= radius, s, y)


def proj_simplex(v):
    """Projection of every pixel vector (axis 0) onto the probability simplex."""
    x = torch.movedim(v, 0, -1)
    u = torch.sort(x, dim=-1, descending=True).values
    return torch.movedim(torch.relu(x - _threshold_sorted(u, 1.0)), -1, 0)


def prox_g2(J2, tau, sp):
    """Schatten-p prox of every pixel's (L K) x 2 matrix by its singular values."""
    L, K, _, H, W = J2.shape
    V = J2.reshape(L * K, 2, H * W).permute(2, 0, 1)            # (n, L K, 2)
    U, S, Vh = torch.linalg.svd(V, full_matrices=False)
    if sp == 1:
        St = torch.relu(S - tau)
    elif sp == 2:
        nrm = torch.sqrt(torch.sum(S * S, dim=-1, keepdim=True))
        St = S * torch.relu(1.0 - tau / nrm)
    elif sp == np.inf:
        St = S - proj_l1_ball(S, tau)                 # Moreau: s - proj_{tau B_1}(s)
    else:
        raise ValueError("Schatten p must be 1, 2 or inf")
    out = U @ torch.diag_embed(St) @ Vh
    return out.permute(1, 2, 0).reshape(L, K, 2, H, W)


def unrolled(log_p, lam, omega, M, mu, sp, iters, g4="affine"):
    """z^T of `iters` SALSA iterations from z^0 = p / 1^T p, u^0 = G z^0, d^0 = 0, with
    p = exp(log p); the same steps as segsalsa_str_oracle.solve (g4 on the affine set or on
    the probability simplex)."""
    p = torch.exp(log_p)
    z = p / torch.sum(p, dim=0, keepdim=True)
    u = apply_G(z, omega, M)
    d = [torch.zeros_like(b) for b in u]
    for _ in range(iters):
        z = linear_solve(apply_GT([a + b for a, b in zip(u, d)], omega, M), omega, M)
        Gz = apply_G(z, omega, M)
        v = [a - b for a, b in zip(Gz, d)]
        u4 = (v[3] - (torch.sum(v[3], dim=0, keepdim=True) - 1.0) / v[3].shape[0]
              if g4 == "affine" else proj_simplex(v[3]))
        u = [prox_g1(v[0], p, mu), prox_g2(v[1], lam / mu, sp), torch.relu(v[2]), u4]
        d = [dj - (gj - uj) for dj, gj, uj in zip(d, Gz, u)]
    return z


def reference_gradient(log_p, lam, omega, M, mu, sp, iters, zbar, g4="affine"):
    """Gradient of <zbar, z^T> with respect to (log p, lambda, omega), all FP64 numpy."""
    lp = torch.tensor(np.asarray(log_p, dtype=np.float64), requires_grad=True)
    la = torch.tensor(float(lam), dtype=DT, requires_grad=True)
    om = torch.tensor(np.asarray(omega, dtype=np.float64), requires_grad=True)
    z = unrolled(lp, la, om, M, mu, sp, iters, g4)
    loss = torch.sum(torch.tensor(np.asarray(zbar, dtype=np.float64)) * z)
    g = torch.autograd.grad(loss, (lp, la, om), allow_unused=True)   # z^1 does not see lambda
    g = [torch.zeros_like(x) if gi is None else gi for gi, x in zip(g, (lp, la, om))]
    return (g[0].numpy(), float(g[1]), g[2].numpy(), z.detach().numpy())
