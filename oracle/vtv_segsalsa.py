"""Independent FP64 SegSALSA iteration with the vectorial TV prior (1x1 patch).

TEST INFRASTRUCTURE ONLY (same rule as segsalsa_str_oracle.py). Sec. 3 and Sec. 5 state that
with 1x1 patches (L = 1) the structure-tensor prior reduces to VTV, i.e. SegSALSA. This file
writes that special case out on its own: forward differences by index arrays (not np.roll),
the z-update denominator from the closed-form eigenvalues of the periodic Laplacian, and the
Schatten prox of the K x 2 gradient matrix from the eigen-decomposition of its 2x2 Gram matrix
(not an SVD). It shares no code with segsalsa_str_oracle.py, so agreement between the two at
M = 0 pins the general oracle's patch machinery, linear solve and iteration assembly.
"""
from __future__ import annotations

import numpy as np


def _grad(z):
    K, H, W = z.shape
    xp = (np.arange(W) + 1) % W
    yp = (np.arange(H) + 1) % H
    return np.stack([z[:, :, xp] - z, z[:, yp, :] - z], axis=-1)      # (K, H, W, 2)


def _grad_T(g):
    K, H, W, _ = g.shape
    xm = (np.arange(W) - 1) % W
    ym = (np.arange(H) - 1) % H
    gh, gv = g[..., 0], g[..., 1]
    return (gh[:, :, xm] - gh) + (gv[:, ym, :] - gv)


def _solve(rhs):
    K, H, W = rhs.shape
    ky = np.arange(H)[:, None]
    kx = np.arange(W)[None, :]
    eig = 3.0 + 4.0 * np.sin(np.pi * ky / H) ** 2 + 4.0 * np.sin(np.pi * kx / W) ** 2
    return np.real(np.fft.ifft2(np.fft.fft2(rhs) / eig))


def _shrink(s1, s2, tau, sp):
    """Shrunk singular values (s1 >= s2 >= 0) for tau*||.||_{S_p}."""
    if sp == 1:
        return np.maximum(s1 - tau, 0.0), np.maximum(s2 - tau, 0.0)
    if sp == 2:
        n = np.hypot(s1, s2)
        f = np.maximum(0.0, 1.0 - tau / np.maximum(n, 1e-300))
        return s1 * f, s2 * f
    # p = inf: s - projection of s onto the l1 ball of radius tau, three cases for 2 entries
    zero = s1 + s2 <= tau
    top = (~zero) & (s1 - s2 >= tau)
    mid = ~(zero | top)
    t1 = np.where(top, s1 - tau, np.where(mid, 0.5 * (s1 + s2 - tau), 0.0))
    t2 = np.where(top, s2, np.where(mid, 0.5 * (s1 + s2 - tau), 0.0))
    return t1, t2


def _prox_vtv(V, tau, sp):
    """V: (n, K, 2) gradient matrices -> prox of tau*||.||_{S_p} via the 2x2 Gram matrix."""
    A = np.einsum("nkc,nkd->ncd", V, V)
    lam, Q = np.linalg.eigh(A)                      # ascending eigenvalues
    s2 = np.sqrt(np.maximum(lam[:, 0], 0.0))
    s1 = np.sqrt(np.maximum(lam[:, 1], 0.0))
    t1, t2 = _shrink(s1, s2, tau, sp)
    g1 = np.where(s1 > 0, t1 / np.where(s1 > 0, s1, 1.0), 0.0)
    g2 = np.where(s2 > 0, t2 / np.where(s2 > 0, s2, 1.0), 0.0)
    # V Q diag(g) Q^T with Q columns = (small, large) eigenvectors
    Dg = np.zeros_like(A)
    Dg[:, 0, 0] = g2
    Dg[:, 1, 1] = g1
    Mx = Q @ Dg @ np.swapaxes(Q, 1, 2)
    return np.einsum("nkc,ncd->nkd", V, Mx)


def vtv_solve(p, lam, mu, sp, iters):
    """SegSALSA with VTV prior: G = [I; D; I; I], same four MPOs, z^0 = normalised p."""
    p = np.asarray(p, dtype=np.float64)
    K, H, W = p.shape
    z = p / p.sum(axis=0, keepdims=True)
    u = [z.copy(), _grad(z), z.copy(), z.copy()]
    d = [np.zeros_like(b) for b in u]
    for _ in range(iters):
        r = [a + b for a, b in zip(u, d)]
        z = _solve(r[0] + _grad_T(r[1]) + r[2] + r[3])
        gz = _grad(z)
        v1, v2, v3, v4 = z - d[0], gz - d[1], z - d[2], z - d[3]
        a = np.sum(p * v1, axis=0)
        b = np.sum(p * p, axis=0)
        s = 0.5 * (a + np.sqrt(a * a + 4.0 * b / mu))
        u1 = v1 + p / (mu * s)
        Vn = np.transpose(v2, (1, 2, 0, 3)).reshape(H * W, K, 2)
        u2 = np.transpose(_prox_vtv(Vn, lam / mu, sp).reshape(H, W, K, 2), (2, 0, 1, 3))
        u3 = np.maximum(v3, 0.0)
        u4 = v4 - (v4.sum(axis=0, keepdims=True) - 1.0) / K
        u = [u1, u2, u3, u4]
        d = [d[0] - (z - u1), d[1] - (gz - u2), d[2] - (z - u3), d[3] - (z - u4)]
    return z
