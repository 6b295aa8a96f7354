"""Pins of the FP64 oracle against things other than itself: closed forms, invariants,
brute force on tiny inputs and an independently written VTV iteration (Sec. 3: a 1x1 patch
reduces SegSALSA-STR to SegSALSA with the VTV prior). CPU only."""
import itertools

import numpy as np
import pytest
from scipy import optimize

from oracle import segsalsa_str_oracle as O
from oracle import vtv_segsalsa as VTV
from paper_1504_07028_gb300 import synth


def _rand(shape, seed):
    return np.random.default_rng(seed).normal(size=shape)


# ---------------------------------------------------------------- weights and the Jacobian

def test_gaussian_weights_reading():
    assert np.allclose(O.gaussian_weights(0, 1.0), [1.0])
    for M, sigma in [(1, 0.5), (2, 1.0), (3, 2.0)]:
        w = O.gaussian_weights(M, sigma)
        assert w.shape == ((2 * M + 1) ** 2,)
        assert abs(np.sum(w * w) - 1.0) < 1e-14
        sh = O.patch_shifts(M)
        c = sh.index((0, 0))
        for j, (dy, dx) in enumerate(sh):
            # omega = sqrt(normalised Gaussian): ratio to the centre is exp(-|s|^2/(4 sigma^2))
            assert abs(w[j] / w[c] - np.exp(-(dy * dy + dx * dx) / (4 * sigma * sigma))) < 1e-14
            assert w[j] == pytest.approx(w[sh.index((-dy, -dx))], abs=0)


@pytest.mark.parametrize("M,H,W", [(1, 4, 5), (3, 8, 9), (5, 12, 13)])
def test_jacobian_brute_force_loops(M, H, W):
    K = 2
    z = _rand((K, H, W), 1)
    om = np.abs(_rand(((2 * M + 1) ** 2,), 2))
    J = O.jacobian(z, om, M)
    for j, (dy, dx) in enumerate(O.patch_shifts(M)):
        for k, y, x in itertools.product(range(K), range(H), range(W)):
            y0, x0 = (y + dy) % H, (x + dx) % W
            h = om[j] * (z[k, y0, (x0 + 1) % W] - z[k, y0, x0])
            v = om[j] * (z[k, (y0 + 1) % H, x0] - z[k, y0, x0])
            assert J[j, k, 0, y, x] == pytest.approx(h, abs=1e-14)
            assert J[j, k, 1, y, x] == pytest.approx(v, abs=1e-14)
    # per-pixel (L K) x 2 matrix: rows ordered (j, k) as in eq. (4)
    Vm = O.jacobian_matrices(J)
    i = 2 * W + 3
    assert np.allclose(Vm[i, 1 * K + 1], J[1, 1, :, 2, 3])


@pytest.mark.parametrize("M", [0, 1, 2, 3, 5])
def test_jacobian_adjoint(M):
    K, H, W = 3, 13, 12
    om = np.abs(_rand(((2 * M + 1) ** 2,), 3))
    x = _rand((K, H, W), 4)
    w = _rand(((2 * M + 1) ** 2, K, 2, H, W), 5)
    lhs = np.sum(O.jacobian(x, om, M) * w)
    rhs = np.sum(x * O.jacobian_T(w, om, M))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("M", [0, 1, 2, 3, 4, 5])
def test_JTJ_equals_weighted_laplacian(M):
    """Periodic shifts are isometries: ||Jz||^2 = (sum omega^2)(||D_h z||^2 + ||D_v z||^2)."""
    K, H, W = 2, 12, 14
    om = np.abs(_rand(((2 * M + 1) ** 2,), 6))
    z = _rand((K, H, W), 7)
    c = np.sum(om ** 2)
    a = np.sum(O.jacobian(z, om, M) ** 2)
    b = c * (np.sum(O.D_h(z) ** 2) + np.sum(O.D_v(z) ** 2))
    assert abs(a - b) <= 1e-12 * b


@pytest.mark.parametrize("H,W,M", [(6, 8, 1), (5, 7, 2), (9, 4, 0)])
def test_symbol_closed_form(H, W, M):
    om = np.abs(_rand(((2 * M + 1) ** 2,), 8))
    c = np.sum(om ** 2)
    ky = np.arange(H)[:, None]
    kx = np.arange(W)[None, :]
    ref = c * (4 * np.sin(np.pi * ky / H) ** 2 + 4 * np.sin(np.pi * kx / W) ** 2)
    assert np.allclose(O.JTJ_symbol(H, W, om, M), ref, atol=1e-12)


# ------------------------------------------------------------------------- linear step (12)

@pytest.mark.parametrize("H,W,K,M", [(16, 12, 3, 1), (15, 17, 2, 2), (8, 8, 4, 0)])
def test_linear_solve_residual_by_stencil(H, W, K, M):
    om = O.gaussian_weights(M, 0.5 + M)
    rhs = _rand((K, H, W), 9)
    z = O.linear_solve(rhs, om, M)
    res = O.apply_GTG(z, om, M) - rhs
    assert np.abs(res).max() <= 1e-12 * np.abs(rhs).max()


def test_linear_solve_dense_brute_force():
    H, W, K, M = 3, 4, 1, 1
    om = np.abs(_rand((9,), 10))
    n = H * W
    A = np.zeros((n, n))
    for c in range(n):
        e = np.zeros((1, H, W))
        e.reshape(-1)[c] = 1.0
        A[:, c] = O.apply_GTG(e, om, M).reshape(-1)
    assert np.allclose(A, A.T, atol=1e-13)
    rhs = _rand((1, H, W), 11)
    zd = np.linalg.solve(A, rhs.reshape(-1)).reshape(1, H, W)
    assert np.allclose(O.linear_solve(rhs, om, M), zd, atol=1e-12)


# ------------------------------------------------------------------------------- the MPOs

def test_prox_g1_stationarity():
    K, H, W = 5, 4, 6
    p = np.abs(_rand((K, H, W), 12)) + 0.01
    v = _rand((K, H, W), 13)
    for mu in (0.3, 1.0, 4.0):
        u = O.prox_g1(v, p, mu)
        s = np.sum(p * u, axis=0)
        assert (s > 0).all()
        assert np.allclose(mu * (u - v), p / s, atol=1e-12)


def test_prox_g1_brute_force():
    rng = np.random.default_rng(14)
    for _ in range(20):
        p = rng.uniform(0.05, 1.0, size=2)
        v = rng.normal(size=2)
        mu = rng.uniform(0.2, 3.0)
        u = O.prox_g1(v[:, None, None], p[:, None, None], mu)[:, 0, 0]

        def f(x):
            t = p @ x
            return np.inf if t <= 0 else -np.log(t) + 0.5 * mu * np.sum((x - v) ** 2)
        start = v + p / (mu * max(p @ v, 1e-3) if p @ v > 0 else v + 2.0 * p)
        best = min((optimize.minimize(f, x0, method="Nelder-Mead",
                                      options=dict(xatol=1e-12, fatol=1e-14, maxiter=20000))
                    for x0 in (start, v + p, np.abs(v) + 1.0)), key=lambda r: r.fun)
        assert np.allclose(u, best.x, atol=1e-6)


def _dual_norm(R, sp):
    s = np.linalg.svd(R, compute_uv=False)
    if sp == 1:
        return s.max(axis=-1)
    if sp == 2:
        return np.sqrt(np.sum(s * s, axis=-1))
    return s.sum(axis=-1)


def _schatten(U, sp):
    s = np.linalg.svd(U, compute_uv=False)
    if sp == np.inf:
        return s.max(axis=-1)
    return np.sum(s ** sp, axis=-1) ** (1.0 / sp)


@pytest.mark.parametrize("sp", [1, 2, np.inf])
def test_prox_g2_moreau_characterisation(sp):
    """U = prox_{tau||.||}(V) iff R = V - U has dual norm <= tau and <U, R> = tau ||U||."""
    V = _rand((400, 18, 2), 15) * np.linspace(0.05, 3.0, 400)[:, None, None]
    tau = 0.9
    U = O.prox_g2(V, tau, sp)
    R = V - U
    assert (_dual_norm(R, sp) <= tau * (1 + 1e-12) + 1e-14).all()
    inner = np.sum(U * R, axis=(1, 2))
    assert np.allclose(inner, tau * _schatten(U, sp), atol=1e-12)


@pytest.mark.parametrize("sp", [1, 2, np.inf])
def test_prox_g2_brute_force_2x2(sp):
    rng = np.random.default_rng(16)
    tau = 0.7
    for _ in range(8):
        V = rng.normal(size=(2, 2)) * 1.5
        U = O.prox_g2(V[None], tau, sp)[0]

        def f(x):
            X = x.reshape(2, 2)
            return tau * _schatten(X[None], sp)[0] + 0.5 * np.sum((X - V) ** 2)
        best = min((optimize.minimize(f, x0, method="Powell",
                                      options=dict(xtol=1e-12, ftol=1e-15, maxiter=200000))
                    for x0 in (V.ravel(), 0.5 * V.ravel(), np.zeros(4),
                               rng.normal(size=4))), key=lambda r: r.fun)
        fu = f(U.ravel())
        assert fu <= best.fun + 1e-9
        # 1-strong convexity: ||x - x*||^2 <= 2 (f(x) - f(x*)) for the search's point
        assert np.sum((best.x - U.ravel()) ** 2) <= 2.0 * (best.fun - fu) + 1e-9


def test_prox_g2_closed_forms():
    V = _rand((50, 12, 2), 17)
    tau = 1.3
    # p = 2 is the Frobenius block shrink
    nf = np.sqrt(np.sum(V * V, axis=(1, 2)))
    ref = V * np.maximum(0.0, 1.0 - tau / nf)[:, None, None]
    assert np.allclose(O.prox_g2(V, tau, 2), ref, atol=1e-13)
    # rank-one V: every Schatten norm is the Frobenius norm of a rank-one matrix
    a = _rand((50, 12, 1), 18)
    b = _rand((50, 1, 2), 19)
    R1 = a @ b
    n1 = np.sqrt(np.sum(R1 * R1, axis=(1, 2)))
    ref1 = R1 * np.maximum(0.0, 1.0 - tau / n1)[:, None, None]
    for sp in (1, 2, np.inf):
        assert np.allclose(O.prox_g2(R1, tau, sp), ref1, atol=1e-12)
    # tau = 0 is the identity
    assert np.allclose(O.prox_g2(V, 0.0, 1), V, atol=1e-13)


def test_proj_l1_ball_brute_force():
    """Compare with a generic solver on the smooth split form t = a - b, a, b >= 0,
    sum(a + b) <= r."""
    rng = np.random.default_rng(20)
    for _ in range(30):
        x = rng.normal(size=3) * 2
        r = rng.uniform(0.1, 3.0)
        y = O.proj_l1_ball(x[None], r)[0]
        assert np.sum(np.abs(y)) <= r + 1e-12
        obj = lambda ab: np.sum((ab[:3] - ab[3:] - x) ** 2)
        cons = [{"type": "ineq", "fun": lambda ab: r - np.sum(ab)}]
        best = optimize.minimize(obj, np.zeros(6), constraints=cons, method="SLSQP",
                                 bounds=[(0, None)] * 6,
                                 options=dict(ftol=1e-15, maxiter=2000))
        assert np.sum((y - x) ** 2) <= best.fun + 1e-9
        t = best.x[:3] - best.x[3:]
        assert np.allclose(t, y, atol=1e-5)


def test_projections_g3_g4_and_simplex():
    v = _rand((6, 5, 7), 21)
    u3 = O.prox_g3(v)
    assert (u3 >= 0).all() and np.all((u3 == v) | (u3 == 0))
    u4 = O.prox_g4(v)
    assert np.allclose(u4.sum(axis=0), 1.0, atol=1e-14)
    dlt = u4 - v
    assert np.allclose(dlt, dlt[:1], atol=1e-14)       # moved along 1_K only
    zp = O.proj_simplex(v)
    assert (zp >= 0).all() and np.allclose(zp.sum(axis=0), 1.0, atol=1e-13)
    # KKT: v - zp = theta*1 - nu, nu >= 0, nu_k zp_k = 0
    g = v - zp
    for y, x in itertools.product(range(5), range(7)):
        act = zp[:, y, x] > 0
        th = g[act, y, x]
        assert np.allclose(th, th[0], atol=1e-12)
        assert (g[~act, y, x] <= th[0] + 1e-12).all()


def test_proj_simplex_brute_force_k3():
    rng = np.random.default_rng(22)
    t = np.linspace(0, 1, 401)
    a, b = np.meshgrid(t, t, indexing="ij")
    ok = a + b <= 1
    pts = np.stack([a[ok], b[ok], 1 - a[ok] - b[ok]], axis=-1)
    for _ in range(10):
        v = rng.normal(size=3)
        zp = O.proj_simplex(v[:, None, None])[:, 0, 0]
        dbest = np.min(np.sum((pts - v) ** 2, axis=1))
        assert np.sum((zp - v) ** 2) <= dbest + 1e-12


# -------------------------------------------------------------------- whole-solver pins

@pytest.mark.parametrize("sp", [1, 2, np.inf])
def test_vtv_reduction_M0(sp):
    """Sec. 3 / Sec. 5: a 1x1 patch gives SegSALSA with the VTV prior."""
    sc = synth.scene(14, 11, 4, S=5, gap=2.0, noise_std=1.0, wrong_frac=0.1, seed=31)
    st, _ = O.solve(sc.p, 0, 1.0, 1.5, 1.3, sp, 40)
    zv = VTV.vtv_solve(sc.p, 1.5, 1.3, sp, 40)
    assert np.abs(st.z - zv).max() < 1e-11


def test_lambda_zero_gives_argmax_p():
    sc = synth.scene(12, 10, 3, S=4, gap=1.0, noise_std=1.0, wrong_frac=0.0, seed=32)
    st, _ = O.solve(sc.p, 1, 0.5, 0.0, 1.0, 1, 400)
    lab, _ = O.labels_and_margin(st.z)
    srt = np.sort(sc.p, axis=0)
    clear = srt[-1] - srt[-2] > 0.02
    assert clear.mean() > 0.9
    assert (lab[clear] == np.argmax(sc.p, axis=0)[clear]).all()


def test_constant_p_stays_constant():
    K, H, W = 4, 9, 8
    p1 = np.array([0.1, 0.5, 0.15, 0.25])
    p = np.broadcast_to(p1[:, None, None], (K, H, W)).copy()
    st, _ = O.solve(p, 1, 0.5, 2.0, 1.0, 1, 100)
    assert np.abs(st.z - st.z[:, :1, :1]).max() < 1e-12
    assert (O.labels_and_margin(st.z)[0] == 1).all()


def test_scale_invariance():
    sc = synth.scene(10, 9, 3, S=3, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=33)
    c = np.random.default_rng(34).uniform(0.1, 10.0, size=(1, 10, 9))
    a, _ = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 1, 30)
    b, _ = O.solve(sc.p * c, 1, 0.5, 1.5, 1.0, 1, 30)
    assert np.abs(a.z - b.z).max() < 1e-10


def test_dual_residual_identity():
    """For k >= 1, G^T d^k = G^T (u^k - u^{k-1}), because G^T G z^k = G^T (u^{k-1} + d^{k-1})."""
    sc = synth.scene(10, 12, 3, S=3, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=35)
    om = O.gaussian_weights(1, 0.5)
    st = O.initial_state(sc.p, om, 1)
    for _ in range(5):
        prev = st
        st, r, s = O.salsa_step(st, sc.p, 1.5, 1.0, om, 1, 1)
        a = O.apply_GT(st.d, om, 1)
        b = O.apply_GT([x - y for x, y in zip(st.u, prev.u)], om, 1)
        assert np.abs(a - b).max() < 1e-12
        assert abs(s - np.sqrt(np.sum(a * a))) < 1e-12
        assert abs(r - np.sqrt(sum(np.sum((x - y) ** 2) for x, y in zip(st.d, prev.d)))) < 1e-12


def test_residuals_decay_and_feasibility():
    sc = synth.scene(16, 16, 3, S=4, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=36)
    st, tr = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 1, 300, trace_every=10)
    k, r, s, obj, zmin, dev = tr.T
    assert r[-1] < 0.05 * r[0] and s[-1] < 0.05 * s[0]
    assert dev[-1] < 0.2 * dev[0]
    assert zmin[0] < zmin[-1] <= 0.0 + 1e-15 or zmin[-1] > 0
    # the objective at the projected iterate settles
    assert abs(obj[-1] - obj[-2]) < 1e-4 * abs(obj[-1])
    assert obj[-1] < obj[0]


@pytest.mark.parametrize("sp", [1, 2, np.inf])
def test_fixed_point_is_a_minimiser(sp):
    """After many iterations z minimises (7) over the simplex: random feasible
    perturbations never lower the objective (convexity makes this a global check)."""
    sc = synth.scene(8, 8, 3, S=3, gap=1.5, noise_std=1.0, wrong_frac=0.0, seed=37)
    om = O.gaussian_weights(1, 0.5)
    st, _ = O.solve(sc.p, 1, 0.5, 0.8, 1.0, sp, 3000)
    z = O.proj_simplex(st.z)
    f0 = O.objective(z, sc.p, 0.8, om, 1, sp)
    rng = np.random.default_rng(38)
    for eps in (1e-2, 1e-3):
        for _ in range(40):
            zq = O.proj_simplex(z + eps * rng.normal(size=z.shape))
            assert O.objective(zq, sc.p, 0.8, om, 1, sp) >= f0 - 1e-6


# ------------------------------------------- eq. (7): Schatten norms and the objective

def _corner_field():
    """4x5 image, K = 3: class 0 everywhere except pixel (0, 1) (class 1) and pixel (1, 0)
    (class 2). With M = 0 (one shift, omega = 1) the Jacobian of a pixel is the K x 2 matrix
    [D_h z, D_v z] (Sec. 3, eq. 4 reduces to the plain forward differences). By hand:
      (0, 0): [e1 - e0, e2 - e0], Gram [[2, 1], [1, 2]], eigenvalues 3 and 1, so singular
              values sqrt(3) and 1;
      (0, 1): [e0 - e1, e0 - e1] and (1, 0): [e0 - e2, e0 - e2], rank one, singular value 2;
      (3, 1): [0, e1 - e0] and (1, 4): [e2 - e0, 0] (periodic neighbours), singular value
              sqrt(2);
      every other pixel: zero."""
    z = np.zeros((3, 4, 5))
    z[0] = 1.0
    z[:, 0, 1] = (0.0, 1.0, 0.0)
    z[:, 1, 0] = (0.0, 0.0, 1.0)
    return z


def _corner_norms(sp):
    r3, r2 = np.sqrt(3.0), np.sqrt(2.0)
    n = np.zeros((4, 5))
    n[0, 0] = {1: 1.0 + r3, 2: 2.0, np.inf: r3}[sp]
    n[0, 1] = n[1, 0] = 2.0
    n[3, 1] = n[1, 4] = r2
    return n


@pytest.mark.parametrize("sp", [1, 2, np.inf])
def test_schatten_norms_closed_form(sp):
    """The Schatten-p norms (Sec. 3) of hand-computed Jacobians: S_1 = s1 + s2,
    S_2 = sqrt(s1^2 + s2^2), S_inf = s1; a rank-one matrix has every norm equal to its
    Frobenius norm."""
    z = _corner_field()
    n = O.schatten_norms(O.jacobian(z, np.ones(1), 0), sp).reshape(4, 5)
    assert np.abs(n - _corner_norms(sp)).max() < 1e-13


@pytest.mark.parametrize("sp", [1, 2, np.inf])
def test_objective_closed_form(sp):
    """Eq. (7) on the hand-computed field with uniform p = 1/3: every z_i is a vertex of the
    simplex, so p_i^T z_i = 1/3 and the data term is n ln 3; the prior is lambda times the
    sum of the norms above."""
    z = _corner_field()
    p = np.full_like(z, 1.0 / 3.0)
    lam = 0.7
    ref = 20 * np.log(3.0) + lam * _corner_norms(sp).sum()
    assert abs(O.objective(z, p, lam, np.ones(1), 0, sp) - ref) < 1e-12


@pytest.mark.parametrize("sp", [1, 2, np.inf])
def test_schatten_norms_from_gram_eigenvalues(sp):
    """Any patch size: the singular values of [Jz]_i are the square roots of the eigenvalues
    of its 2 x 2 Gram matrix (eq. 5), which have the closed form tr/2 +- sqrt((a-c)^2/4 + b^2)
    (no SVD); the norms built from them match."""
    sc = synth.scene(9, 7, 4, S=3, gap=1.0, noise_std=1.0, wrong_frac=0.0, seed=39)
    om = O.gaussian_weights(2, 1.0)
    Jz = O.jacobian(sc.p, om, 2)
    h, v = Jz[:, :, 0], Jz[:, :, 1]
    a = np.sum(h * h, axis=(0, 1)).ravel()
    b = np.sum(h * v, axis=(0, 1)).ravel()
    c = np.sum(v * v, axis=(0, 1)).ravel()
    r = np.sqrt(0.25 * (a - c) ** 2 + b * b)
    s1 = np.sqrt(0.5 * (a + c) + r)
    s2 = np.sqrt(np.maximum(0.5 * (a + c) - r, 0.0))
    ref = {1: s1 + s2, 2: np.sqrt(a + c), np.inf: s1}[sp]
    assert np.allclose(O.schatten_norms(Jz, sp), ref, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------- Sec. 5: MLR class model

def _mlr_brute(x, Wc, b):
    """p_k = 1 / sum_j exp(l_j - l_k), pixel by pixel with math.exp (a different formula from
    the oracle's shifted softmax)."""
    import math
    H, W, d = x.shape
    K = Wc.shape[0]
    p = np.zeros((K, H, W))
    for yy in range(H):
        for xx in range(W):
            lg = [sum(Wc[k, t] * x[yy, xx, t] for t in range(d)) + b[k] for k in range(K)]
            for k in range(K):
                p[k, yy, xx] = 1.0 / sum(math.exp(lj - lg[k]) for lj in lg)
    return p


def test_mlr_brute_force():
    sc = synth.mlr_scene(3, 4, 5, 7, S=3, seed=40)
    b = np.random.default_rng(41).normal(size=5)
    assert np.abs(O.mlr_probs(sc.x, sc.Wc, b) - _mlr_brute(sc.x, sc.Wc, b)).max() < 1e-14


def test_mlr_special_cases():
    sc = synth.mlr_scene(4, 5, 6, 9, S=3, seed=42)
    # zero weights: uniform posterior
    assert np.abs(O.mlr_probs(sc.x, np.zeros_like(sc.Wc), np.zeros(6)) - 1.0 / 6).max() < 1e-15
    # K = 2 is the logistic sigmoid of the logit difference
    W2, b2 = sc.Wc[:2], np.array([0.3, -0.2])
    l = sc.x @ W2.T + b2
    sig = 1.0 / (1.0 + np.exp(-(l[..., 1] - l[..., 0])))
    assert np.abs(O.mlr_probs(sc.x, W2, b2)[1] - sig).max() < 1e-14
    # a common shift of the biases changes nothing; sums are one; order follows the logits
    p = O.mlr_probs(sc.x, sc.Wc, sc.b)
    assert np.abs(O.mlr_probs(sc.x, sc.Wc, sc.b + 7.5) - p).max() < 1e-14
    assert np.abs(p.sum(axis=0) - 1.0).max() < 1e-14 and p.min() > 0
    lg = np.moveaxis(sc.x @ sc.Wc.T, -1, 0)
    assert np.array_equal(np.argmax(p, axis=0), np.argmax(lg, axis=0))
    # large weights: one-hot on the logit argmax (no overflow)
    ph = O.mlr_probs(sc.x, 1e4 * sc.Wc, sc.b)
    assert np.all(np.isfinite(ph)) and np.abs(ph.max(axis=0) - 1.0).max() < 1e-6


def test_mlr_scene_margin():
    """The synthetic weights give the true class a logit margin of about 2 (recipe check)."""
    sc = synth.mlr_scene(32, 32, 9, 103, S=12, seed=43)
    lg = sc.x @ sc.Wc.T
    y = sc.labels
    true = np.take_along_axis(lg, y[..., None], axis=-1)[..., 0]
    other = np.where(np.eye(9, dtype=bool)[y], -np.inf, lg).max(axis=-1)
    assert 0.5 < np.median(true - other) < 4.0
    assert np.mean(np.argmax(lg, axis=-1) == y) > 0.6


# ------------------------------------------- g4 read as the simplex indicator (variant)

def test_simplex_g4_variant_same_minimum():
    """Sec. 4 describes the MPO of g4 as the projection onto the probability simplex while
    eq. (10) defines g4 on the affine set; with g3 = i_+ present both splittings constrain z to
    the same simplex, so the convex problem (7) has the same minimum value either way."""
    sc = synth.scene(10, 10, 3, S=3, gap=1.5, noise_std=1.0, wrong_frac=0.0, seed=44)
    om = O.gaussian_weights(1, 0.5)
    sa, _ = O.solve(sc.p, 1, 0.5, 0.8, 1.0, 1, 2500)
    ss, _ = O.solve(sc.p, 1, 0.5, 0.8, 1.0, 1, 2500, g4="simplex")
    fa = O.objective(O.proj_simplex(sa.z), sc.p, 0.8, om, 1, 1)
    fs = O.objective(O.proj_simplex(ss.z), sc.p, 0.8, om, 1, 1)
    assert abs(fa - fs) < 1e-6 * abs(fa)
    assert np.abs(sa.z - ss.z).max() > 1e-12          # the iterates themselves differ


def test_simplex_g4_variant_u4_on_simplex():
    sc = synth.scene(8, 9, 4, S=3, gap=1.0, noise_std=2.0, wrong_frac=0.2, seed=45)
    om = O.gaussian_weights(1, 0.5)
    st, _ = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 2, 2, g4="simplex")
    u4 = st.u[3]
    assert u4.min() >= 0.0 and np.abs(u4.sum(axis=0) - 1.0).max() < 1e-12
    sa, _ = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 2, 2)
    assert sa.u[3].min() < 0.0                        # the affine variant leaves the orthant
