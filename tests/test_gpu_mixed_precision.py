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
