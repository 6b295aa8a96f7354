"""FP64 CPU oracle of SegSALSA-STR (Condessa, Bioucas-Dias, Kovacevic, arXiv 1504.07028).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or execute this file:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of ``bench.py`` do.

It is the method written out plainly, step by step, in the paper's order and notation, with
numpy FP64 and library primitives (``np.roll`` for shifts, ``np.fft`` for the cyclic
convolution of the z-update, ``np.linalg.svd`` for the singular values, ``np.sort``).
It shares no code with the CUDA path; the only common module is the seeded input generator.

Notation (Sec. 2-4):
  z       hidden field, class-major array (K, H, W)  (z is K x n, n = H*W)
  p       class probabilities p_i, same shape as z   (eq. 7)
  J       patch-based Jacobian (eq. 4): (Jz)[j, k, c, y, x] with shift index j (row-major over
          (dy, dx) in [-M, M]^2), class k, column c (0 = horizontal difference D_h,
          1 = vertical difference D_v); [Jz]_i is the (L*K) x 2 matrix with rows (j, k)
  G       stacking [I; J; I; I] (eq. 9, 11); u = (u1, u2, u3, u4), d likewise
  g1..g4  -ln(p^T .), lambda*||.||_{S_p}, i_+, i_1(1^T .)  (eq. 10)

Readings where the paper is silent or ambiguous:
  * shift weights omega_j = sqrt(g_j), g_j a normalised Gaussian exp(-|s_j|^2 / (2 sigma^2))
    so that J^T J is a Gaussian-weighted structure tensor and sum omega_j^2 = 1 (Sec. 3);
  * periodic boundaries and forward differences (the "cyclic convolutions" of Sec. 4);
  * the u-update (13) uses the freshly computed z^{k+1};
  * g4 is the indicator of the affine set {1^T xi = 1} as defined in eq. (10), so its MPO is
    the affine projection (positivity is g3's job);
  * initial state z^0 = p normalised per pixel, u^0 = G z^0, d^0 = 0;
  * the dual residual is mu * ||G^T (u^k - u^{k-1})||, the primal one ||G z^k - u^k||.

Parity pins: every function is checked in tests/test_oracle_pins.py against closed forms,
invariants, brute force and an independently written VTV iteration. Nothing here is
"parity unpinned" except the paper's Fig. 1 accuracies, which need the missing dataset.
"""
from __future__ import annotations

import numpy as np

INF = np.inf


# ------------------------------------------------------------------------------------------
# Sec. 3: patch shifts, weights, difference and shift operators, patch-based Jacobian (eq. 4)
# ------------------------------------------------------------------------------------------

def patch_shifts(M: int):
    """The L = (2M+1)^2 shifts s_j = (dy, dx) of a (2M+1)x(2M+1) patch, row-major."""
    return [(dy, dx) for dy in range(-M, M + 1) for dx in range(-M, M + 1)]


def gaussian_weights(M: int, sigma: float) -> np.ndarray:
    """Shift weights omega_j (Sec. 3: each shift weighted by a Gaussian centred on the patch
    centre). Reading: omega_j = sqrt(g_j) with g normalised to sum 1."""
    g = np.array([np.exp(-(dy * dy + dx * dx) / (2.0 * sigma * sigma))
                  for dy, dx in patch_shifts(M)], dtype=np.float64)
    g = g / g.sum()
    return np.sqrt(g)


def D_h(f: np.ndarray) -> np.ndarray:
    """Horizontal forward difference, periodic: (D_h f)[y, x] = f[y, x+1] - f[y, x]."""
    return np.roll(f, -1, axis=-1) - f


def D_v(f: np.ndarray) -> np.ndarray:
    """Vertical forward difference, periodic: (D_v f)[y, x] = f[y+1, x] - f[y, x]."""
    return np.roll(f, -1, axis=-2) - f


def D_h_T(g: np.ndarray) -> np.ndarray:
    """Adjoint of D_h: (D_h^T g)[y, x] = g[y, x-1] - g[y, x]."""
    return np.roll(g, 1, axis=-1) - g


def D_v_T(g: np.ndarray) -> np.ndarray:
    return np.roll(g, 1, axis=-2) - g


def shift(f: np.ndarray, s) -> np.ndarray:
    """Unweighted shift: (S_s f)[i] = f[i + s], periodic."""
    return np.roll(f, (-s[0], -s[1]), axis=(-2, -1))


def shift_T(g: np.ndarray, s) -> np.ndarray:
    """Adjoint of shift(., s): (S_s^T g)[i] = g[i - s]."""
    return np.roll(g, (s[0], s[1]), axis=(-2, -1))


def jacobian(z: np.ndarray, omega: np.ndarray, M: int) -> np.ndarray:
    """Patch-based Jacobian of eq. (4), applied to every pixel at once.

    Returns an array of shape (L, K, 2, H, W): entry [j, k, 0] is omega_j (P_j D_h z)_k and
    [j, k, 1] is omega_j (P_j D_v z)_k, where P_j is the weighted shift by s_j.
    """
    dh, dv = D_h(z), D_v(z)
    out = np.empty((len(omega),) + (z.shape[0], 2) + z.shape[1:], dtype=np.float64)
    for j, s in enumerate(patch_shifts(M)):
        out[j, :, 0] = omega[j] * shift(dh, s)
        out[j, :, 1] = omega[j] * shift(dv, s)
    return out


def jacobian_T(w: np.ndarray, omega: np.ndarray, M: int) -> np.ndarray:
    """Adjoint J^T: (L, K, 2, H, W) -> (K, H, W)."""
    out = np.zeros((w.shape[1],) + w.shape[3:], dtype=np.float64)
    for j, s in enumerate(patch_shifts(M)):
        out += omega[j] * (D_h_T(shift_T(w[j, :, 0], s)) + D_v_T(shift_T(w[j, :, 1], s)))
    return out


def jacobian_matrices(Jz: np.ndarray) -> np.ndarray:
    """Per-pixel (L*K) x 2 matrices [Jz]_i (rows ordered (j, k)), shape (H*W, L*K, 2)."""
    L, K, _, H, W = Jz.shape
    return np.moveaxis(Jz.reshape(L * K, 2, H * W), -1, 0)


def from_jacobian_matrices(V: np.ndarray, L: int, K: int, H: int, W: int) -> np.ndarray:
    return np.moveaxis(V, 0, -1).reshape(L, K, 2, H, W)


# ------------------------------------------------------------------------------------------
# Sec. 4: z-update (12): (G^T G) z = G^T (u + d), G^T G = 3 I + J^T J, solved by cyclic
# convolution. J^T J is a circulant operator on each class image, so it is the cyclic
# convolution with its own impulse response h = J^T J delta, and the DFT diagonalises it.
# ------------------------------------------------------------------------------------------

def JTJ_symbol(H: int, W: int, omega: np.ndarray, M: int) -> np.ndarray:
    """DFT of the impulse response of J^T J (real: the operator is symmetric)."""
    delta = np.zeros((1, H, W))
    delta[0, 0, 0] = 1.0
    h = jacobian_T(jacobian(delta, omega, M), omega, M)[0]
    return np.fft.fft2(h).real


def apply_GTG(z: np.ndarray, omega: np.ndarray, M: int) -> np.ndarray:
    """G^T G z = 3 z + J^T J z, applied through the stencils (no DFT)."""
    return 3.0 * z + jacobian_T(jacobian(z, omega, M), omega, M)


def linear_solve(rhs: np.ndarray, omega: np.ndarray, M: int) -> np.ndarray:
    """z = (3 I + J^T J)^{-1} rhs, per class image, by the 2D DFT."""
    K, H, W = rhs.shape
    den = 3.0 + JTJ_symbol(H, W, omega, M)
    return np.fft.ifft2(np.fft.fft2(rhs, axes=(-2, -1)) / den, axes=(-2, -1)).real


# ------------------------------------------------------------------------------------------
# Sec. 4: Moreau proximity operators of g1..g4 with weight 1/mu (eq. 13 decoupled)
# ------------------------------------------------------------------------------------------

def prox_g1(v: np.ndarray, p: np.ndarray, mu: float) -> np.ndarray:
    """argmin_u -ln(p_i^T u_i) + (mu/2)||u_i - v_i||^2 for every pixel i.

    Stationarity gives u = v + p / (mu * s) with s = p^T u, hence the quadratic
    s^2 - (p^T v) s - ||p||^2 / mu = 0, whose positive root is the closed form of Sec. 4.
    """
    a = np.sum(p * v, axis=0)
    b = np.sum(p * p, axis=0)
    s = 0.5 * (a + np.sqrt(a * a + 4.0 * b / mu))
    return v + p / (mu * s)


def proj_l1_ball(x: np.ndarray, radius: float) -> np.ndarray:
    """Euclidean projection of each row of x (last axis) onto {||y||_1 <= radius}, by the
    sort-based threshold search (Duchi, Shalev-Shwartz, Singer, Chandra 2008)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    inside = a.sum(axis=-1) <= radius
    u = -np.sort(-a, axis=-1)
    css = np.cumsum(u, axis=-1)
    j = np.arange(1, x.shape[-1] + 1)
    cond = u - (css - radius) / j > 0
    rho = x.shape[-1] - np.argmax(cond[..., ::-1], axis=-1)     # last index where cond holds
    theta = (np.take_along_axis(css, (rho - 1)[..., None], axis=-1)[..., 0] - radius) / rho
    y = np.sign(x) * np.maximum(a - theta[..., None], 0.0)
    return np.where(inside[..., None], x, y)


def shrink_singular_values(sv: np.ndarray, tau: float, sp) -> np.ndarray:
    """prox of tau*||.||_p on the vector of singular values (unitarily invariant norm)."""
    if sp == 1:
        return np.maximum(sv - tau, 0.0)
    if sp == 2:
        nrm = np.sqrt(np.sum(sv * sv, axis=-1, keepdims=True))
        scale = np.where(nrm > tau, 1.0 - tau / np.where(nrm > 0, nrm, 1.0), 0.0)
        return sv * scale
    if sp == INF:
        # Moreau decomposition: prox_{tau ||.||_inf}(s) = s - proj_{tau B_1}(s)
        return sv - proj_l1_ball(sv, tau)
    raise ValueError("Schatten p must be 1, 2 or inf")


def prox_g2(V: np.ndarray, tau: float, sp) -> np.ndarray:
    """argmin_U tau*||U||_{S_p} + (1/2)||U - V||_F^2 for a stack of (L*K) x 2 matrices
    (Sec. 4, MPO of g2 with tau = lambda/mu): shrink the singular values of V."""
    U, s, Wt = np.linalg.svd(V, full_matrices=False)
    s2 = shrink_singular_values(s, tau, sp)
    return (U * s2[..., None, :]) @ Wt


def prox_g3(v: np.ndarray) -> np.ndarray:
    """Projection onto the positive orthant (indicator i_+)."""
    return np.maximum(v, 0.0)


def prox_g4(v: np.ndarray) -> np.ndarray:
    """Projection onto {xi : 1_K^T xi_i = 1 for every pixel} (indicator i_1(1^T .))."""
    K = v.shape[0]
    return v - (np.sum(v, axis=0, keepdims=True) - 1.0) / K


def proj_simplex(v: np.ndarray) -> np.ndarray:
    """Euclidean projection of every pixel vector (axis 0) onto the probability simplex, by
    the sort-based threshold (Held, Wolfe, Crowder 1974; Duchi et al. 2008)."""
    x = np.moveaxis(v, 0, -1)
    u = -np.sort(-x, axis=-1)
    css = np.cumsum(u, axis=-1)
    j = np.arange(1, x.shape[-1] + 1)
    cond = u - (css - 1.0) / j > 0
    rho = x.shape[-1] - np.argmax(cond[..., ::-1], axis=-1)
    theta = (np.take_along_axis(css, (rho - 1)[..., None], axis=-1)[..., 0] - 1.0) / rho
    return np.moveaxis(np.maximum(x - theta[..., None], 0.0), -1, 0)


# ------------------------------------------------------------------------------------------
# Problem (7), split form (8)-(11), SALSA iteration (12)-(14)
# ------------------------------------------------------------------------------------------

def schatten_norms(Jz: np.ndarray, sp) -> np.ndarray:
    """||[Jz]_i||_{S_p} for every pixel."""
    s = np.linalg.svd(jacobian_matrices(Jz), compute_uv=False)
    if sp == INF:
        return s.max(axis=-1)
    return np.sum(s ** sp, axis=-1) ** (1.0 / sp)


def objective(z: np.ndarray, p: np.ndarray, lam: float, omega, M: int, sp) -> float:
    """sum_i -ln(p_i^T z_i) + lambda sum_i ||[Jz]_i||_{S_p}  (eq. 7)."""
    data = -np.sum(np.log(np.sum(p * z, axis=0)))
    return float(data + lam * np.sum(schatten_norms(jacobian(z, omega, M), sp)))


def apply_G(z, omega, M):
    return [z, jacobian(z, omega, M), z, z]


def apply_GT(x, omega, M):
    return x[0] + jacobian_T(x[1], omega, M) + x[2] + x[3]


def _norm2(blocks) -> float:
    return float(np.sqrt(sum(np.sum(b * b) for b in blocks)))


class SalsaState:
    """ADMM state after k iterations: z^k, u^k, d^k (eqs. 12-14)."""

    def __init__(self, z, u, d, k=0):
        self.z, self.u, self.d, self.k = z, u, d, k

    def copy(self):
        return SalsaState(self.z.copy(), [b.copy() for b in self.u],
                          [b.copy() for b in self.d], self.k)

    def rhs(self, omega, M):
        """G^T (u^k + d^k): the right-hand side of the next z-update."""
        return apply_GT([a + b for a, b in zip(self.u, self.d)], omega, M)


def initial_state(p: np.ndarray, omega, M) -> SalsaState:
    z0 = p / np.sum(p, axis=0, keepdims=True)
    u0 = apply_G(z0, omega, M)
    d0 = [np.zeros_like(b) for b in u0]
    return SalsaState(z0, u0, d0, 0)


def u_d_update(z, d, p, lam, mu, omega, M, sp, g4="affine"):
    """Eqs. (13)-(14) given z^{k+1}: the four decoupled MPOs at v = G z^{k+1} - d^k, then
    d^{k+1} = d^k - (G z^{k+1} - u^{k+1}). Returns (u^{k+1}, d^{k+1}, G z^{k+1}).

    g4 = "affine": the MPO of g4 as eq. (10) defines it (projection onto 1^T xi = 1);
    g4 = "simplex": the projection onto the probability simplex, as Sec. 4's text describes the
    MPO of g4 (with g3 = i_+ also present, both variants constrain z to the same feasible set)."""
    L = len(omega)
    K, H, W = p.shape
    Gz = apply_G(z, omega, M)
    v = [a - b for a, b in zip(Gz, d)]
    u1 = prox_g1(v[0], p, mu)
    V2 = jacobian_matrices(v[1])
    u2 = from_jacobian_matrices(prox_g2(V2, lam / mu, sp), L, K, H, W)
    u3 = prox_g3(v[2])
    u4 = prox_g4(v[3]) if g4 == "affine" else proj_simplex(v[3])
    u = [u1, u2, u3, u4]
    dn = [dj - (gj - uj) for dj, gj, uj in zip(d, Gz, u)]
    return u, dn, Gz


def salsa_step(st: SalsaState, p, lam, mu, omega, M, sp, g4="affine"):
    """One SALSA iteration (12)-(14). Returns (new state, primal residual, dual residual)."""
    # (12) z^{k+1} = argmin ||G z - u^k - d^k||^2  <=>  G^T G z = G^T (u^k + d^k)
    z = linear_solve(st.rhs(omega, M), omega, M)
    # (13), (14)
    u, d, Gz = u_d_update(z, st.d, p, lam, mu, omega, M, sp, g4)
    primal = _norm2([gj - uj for gj, uj in zip(Gz, u)])
    dual = mu * _norm2([apply_GT([a - b for a, b in zip(u, st.u)], omega, M)])
    return SalsaState(z, u, d, st.k + 1), primal, dual


def diagnostics(st: SalsaState, p, lam, omega, M, sp) -> dict:
    """Objective (7) at the simplex projection of z, and the feasibility of z itself."""
    zp = proj_simplex(st.z)
    return {
        "objective": objective(zp, p, lam, omega, M, sp),
        "min_z": float(st.z.min()),
        "max_sum_dev": float(np.abs(np.sum(st.z, axis=0) - 1.0).max()),
    }


def solve(p, M, sigma, lam, mu, sp, iters, omega=None, trace_every=0, state=None, g4="affine"):
    """Run `iters` SALSA iterations from z^0 = p (normalised) or from `state`.

    Returns (state, trace) where trace rows are
    (k, primal residual, dual residual, objective at proj_simplex(z^k), min z^k,
    max |1^T z^k - 1|) for every k with k % trace_every == 0 and for the last k.
    """
    p = np.asarray(p, dtype=np.float64)
    if omega is None:
        omega = gaussian_weights(M, sigma)
    st = initial_state(p, omega, M) if state is None else state
    trace = []
    for it in range(iters):
        st, r, s = salsa_step(st, p, lam, mu, omega, M, sp, g4)
        if trace_every and (st.k % trace_every == 0 or it == iters - 1):
            dg = diagnostics(st, p, lam, omega, M, sp)
            trace.append((st.k, r, s, dg["objective"], dg["min_z"], dg["max_sum_dev"]))
    return st, np.array(trace, dtype=np.float64).reshape(-1, 6)


def labels_and_margin(z: np.ndarray):
    """Label readout argmax_k z_k (ties to the lowest k, link p(y_i=k|z_i) = [z_i]_k) and
    the top-two margin of every pixel."""
    lab = np.argmax(z, axis=0)
    srt = np.sort(z, axis=0)
    return lab, srt[-1] - srt[-2]


# ------------------------------------------------------------------------------------------
# Sec. 5: the class model that feeds problem (7). The experiments model the classes with a
# multinomial logistic regression (MLR); its posterior is the softmax of one affine function
# of the spectrum per class. The paper prints no formula; this is the standard definition,
# with an optional bias per class.
# ------------------------------------------------------------------------------------------

def mlr_probs(x: np.ndarray, Wc: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """p_i = softmax_k(w_k^T x_i + b_k) for spectra x of shape (H, W, d), weights Wc (K, d)
    and biases b (K,); returns p class-major (K, H, W) like z."""
    H, W, d = x.shape
    K = Wc.shape[0]
    logits = x.reshape(H * W, d) @ Wc.T                      # (n, K), a library matmul
    if b is not None:
        logits = logits + b[None, :]
    logits = logits - logits.max(axis=1, keepdims=True)      # exp of non-positive numbers
    e = np.exp(logits)
    p = e / e.sum(axis=1, keepdims=True)
    return np.ascontiguousarray(p.T.reshape(K, H, W))

