"""Degenerate Gram matrices in the FP32 sweep: the closed-form Schatten prox coefficients have
no division by the eigenvalue gap, so the FP32 path stays accurate when s1 = s2.

Class 0 rising along x and class 1 along y by exactly 1/64 per pixel make every pixel's Gram
matrix a multiple of the identity away from the wrap-around rows and columns (a = c exactly,
b = 0), i.e. the degenerate case s1 = s2 of Sec. 4's singular-value shrinkage. One sweep from
that state must match the FP64 oracle's u/d update."""
import numpy as np
import pytest

from oracle import segsalsa_str_oracle as O
from tests.helpers import d2_abi_to_oracle, hwk_to_khw, max_abs, oracle_state_to_abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_07028_gb300 import binding
    return binding


@pytest.mark.parametrize("sp,lam", [(1, 0.01), ("inf", 0.01), (1, 0.03), ("inf", 0.005)])
def test_degenerate_gram_sweep(B, sp, lam):
    H, W, K, M, sigma, mu = 24, 28, 2, 1, 0.5, 1.0
    spv = np.inf if sp == "inf" else sp
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    z = np.stack([xx / 64.0, yy / 64.0]).astype(np.float32)          # exact in FP32
    p = np.full((K, H, W), 0.5)
    om = O.gaussian_weights(M, sigma)
    st = O.initial_state(p, om, M)
    st.z = z.astype(np.float64)
    st.d = [np.zeros_like(x) for x in st.d]
    a = oracle_state_to_abi(st, om, M, np.float32)
    a["rhs"] = None
    s = B.Solver(B.make_params(H, W, K, M=M, sigma=sigma, lam=lam, mu=mu, schatten_p=sp))
    s.set_probs(p.astype(np.float32))
    s.set_state(a, 0)
    s.solve(1)
    g = s.get_state()
    u, dn, _ = O.u_d_update(st.z, st.d, p, lam, mu, om, M, spv)
    assert max_abs(d2_abi_to_oracle(g["d2"]), dn[1]) < 1e-6
    assert max_abs(hwk_to_khw(g["d1"]), dn[0]) < 1e-6
    s.close()


def _near_degenerate_state(H, W, K, M, tau, seed):
    """z constant (so J z = 0) and d2 = -V, so that v2 = J z - d2 = V: each pixel's (LK) x 2
    matrix V = Q diag(s1, s2) R(theta)^T with random orthonormal Q, a random rotation R
    (b != 0 in the Gram matrix) and eigenvalue gap (s1^2 - s2^2) = eps (s1^2 + s2^2), eps
    cycling through 1e-9, 1e-7, 1e-6, 1e-5. The pixels' largest singular value s1 is placed
    at 1.3 tau, tau (1 + eps/4), 0.7 tau or 0.4 tau in turn: both values above the threshold,
    the threshold between them, both below (p = 1 kills them; p = inf shrinks both to
    (s1 + s2 - tau)/2) and s1 + s2 below tau. Values are rounded to FP32 before either side
    sees them."""
    L = (2 * M + 1) ** 2
    rng = np.random.default_rng(seed)
    n = H * W
    eps = np.array([1e-9, 1e-7, 1e-6, 1e-5])[np.arange(n) % 4]
    place = np.array([1.3, 1.0, 0.7, 0.4])[(np.arange(n) // 4) % 4]
    s1 = np.where(place == 1.0, tau * (1.0 + eps / 4.0), place * tau)
    s2 = s1 * np.sqrt((1.0 - eps) / (1.0 + eps))
    V = np.empty((n, L * K, 2))
    for i in range(n):
        Q, _ = np.linalg.qr(rng.normal(size=(L * K, 2)))
        th = rng.uniform(0.0, np.pi)
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        V[i] = Q @ np.diag([s1[i], s2[i]]) @ R.T
    V = V.astype(np.float32).astype(np.float64)
    d2 = -O.from_jacobian_matrices(V, L, K, H, W)            # (L, K, 2, H, W)
    z = np.full((K, H, W), 1.0 / K)
    return z, d2


@pytest.mark.parametrize("sp", [1, "inf"])
def test_near_degenerate_gram_sweep(B, sp):
    """One FP32 sweep at Gram matrices with 0 < s1^2 - s2^2 << trace (Sec. 4, MPO of g2:
    the singular-value shrinkage of eq. (5)'s 2 x 2 eigenproblem) against the FP64 oracle,
    at the operator tolerance of the sweep-step parity tests (2e-5)."""
    from paper_1504_07028_gb300 import synth
    H, W, K, M, sigma, lam, mu = 16, 20, 4, 1, 0.5, 0.9, 1.0
    spv = np.inf if sp == "inf" else sp
    tau = lam / mu
    z, d2 = _near_degenerate_state(H, W, K, M, tau, seed=81)
    sc = synth.scene(H, W, K, S=4, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=82)
    p = sc.p.astype(np.float32).astype(np.float64)
    om = O.gaussian_weights(M, sigma)
    st = O.initial_state(p, om, M)
    st.z = z
    st.d = [np.zeros_like(st.d[0]), d2, np.zeros_like(st.d[2]), np.zeros_like(st.d[3])]
    a = oracle_state_to_abi(st, om, M, np.float32)
    a["rhs"] = None
    s = B.Solver(B.make_params(H, W, K, M=M, sigma=sigma, lam=lam, mu=mu, schatten_p=sp))
    s.set_probs(p.astype(np.float32))
    s.set_state(a, 0)
    s.solve(1)
    g = s.get_state()
    u, dn, _ = O.u_d_update(st.z, st.d, p, lam, mu, om, M, spv)
    rhs = O.apply_GT([x + y for x, y in zip(u, dn)], om, M)
    assert max_abs(d2_abi_to_oracle(g["d2"]), dn[1]) <= 2e-5
    assert max_abs(hwk_to_khw(g["d1"]), dn[0]) <= 2e-5
    assert max_abs(hwk_to_khw(g["rhs"]), rhs) <= 8e-5 * max(1.0, np.abs(rhs).max())
    s.close()
