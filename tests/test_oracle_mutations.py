"""Plant plausible mistakes in the oracle (on the CPU, by monkeypatching) and check that the
pins in test_oracle_pins.py catch every one of them."""
import numpy as np
import pytest

from oracle import segsalsa_str_oracle as O
import tests.test_oracle_pins as P

_orig = {name: getattr(O, name) for name in
         ("shift", "prox_g1", "prox_g2", "linear_solve", "prox_g4", "D_v_T", "jacobian",
          "mlr_probs", "proj_simplex", "schatten_norms")}


def _wrong_shift(f, s):                     # shift sign flipped
    return np.roll(f, (s[0], s[1]), axis=(-2, -1))


def _wrong_root(v, p, mu):                  # negative root of the quadratic
    a = np.sum(p * v, axis=0)
    b = np.sum(p * p, axis=0)
    s = 0.5 * (a - np.sqrt(a * a + 4.0 * b / mu))
    return v + p / (mu * s)


def _wrong_tau(V, tau, sp):                 # lambda*mu in place of lambda/mu at mu = 1.3
    return _orig["prox_g2"](V, tau * 1.69, sp)


def _wrong_shrink(V, tau, sp):              # shrinks by tau twice
    return _orig["prox_g2"](V, 2 * tau, sp)


def _wrong_identity_weight(rhs, omega, M):  # 2 I in place of 3 I in G^T G
    K, H, W = rhs.shape
    den = 2.0 + O.JTJ_symbol(H, W, omega, M)
    return np.fft.ifft2(np.fft.fft2(rhs, axes=(-2, -1)) / den, axes=(-2, -1)).real


def _wrong_affine(v):                       # divides by K+1
    return v - (np.sum(v, axis=0, keepdims=True) - 1.0) / (v.shape[0] + 1)


def _wrong_adjoint(g):                      # transposed difference, wrong direction
    return np.roll(g, -1, axis=-2) - g


def _dropped_weight(z, omega, M):           # weights dropped from the Jacobian
    return _orig["jacobian"](z, np.ones_like(omega), M)


def _dropped_bias(x, Wc, b=None):           # MLR bias ignored
    return _orig["mlr_probs"](x, Wc, None)


def _wrong_softmax_axis(x, Wc, b=None):     # normalised over pixels instead of classes
    H, W, d = x.shape
    lg = x.reshape(H * W, d) @ Wc.T + (0 if b is None else b[None, :])
    e = np.exp(lg - lg.max(axis=0, keepdims=True))
    return np.ascontiguousarray((e / e.sum(axis=0, keepdims=True)).T.reshape(-1, H, W))


def _wrong_affine_for_simplex(v):           # the affine projection where the simplex one belongs
    return v - (np.sum(v, axis=0, keepdims=True) - 1.0) / v.shape[0]


def _dropped_root(Jz, sp):                   # sum of s^p without the 1/p root
    s = np.linalg.svd(O.jacobian_matrices(Jz), compute_uv=False)
    return s.max(axis=-1) if sp == np.inf else np.sum(s ** sp, axis=-1)


def _sum_for_max(Jz, sp):                   # S_inf as the sum of the singular values
    s = np.linalg.svd(O.jacobian_matrices(Jz), compute_uv=False)
    return s.sum(axis=-1) if sp == np.inf else _orig["schatten_norms"](Jz, sp)


MUTATIONS = [
    ("shift", _wrong_shift, [lambda: P.test_jacobian_brute_force_loops(1, 4, 5)]),
    ("prox_g1", _wrong_root, [P.test_prox_g1_stationarity]),
    ("prox_g2", _wrong_tau, [lambda: P.test_vtv_reduction_M0(1)]),
    ("prox_g2", _wrong_shrink, [lambda: P.test_prox_g2_moreau_characterisation(1)]),
    ("linear_solve", _wrong_identity_weight,
     [lambda: P.test_linear_solve_residual_by_stencil(16, 12, 3, 1)]),
    ("prox_g4", _wrong_affine, [P.test_projections_g3_g4_and_simplex]),
    ("D_v_T", _wrong_adjoint, [lambda: P.test_jacobian_adjoint(1)]),
    ("jacobian", _dropped_weight, [lambda: P.test_JTJ_equals_weighted_laplacian(1),
                                   lambda: P.test_symbol_closed_form(6, 8, 1)]),
    ("mlr_probs", _dropped_bias, [P.test_mlr_brute_force]),
    ("proj_simplex", _wrong_affine_for_simplex, [P.test_simplex_g4_variant_u4_on_simplex]),
    ("mlr_probs", _wrong_softmax_axis, [P.test_mlr_brute_force, P.test_mlr_special_cases]),
    ("schatten_norms", _dropped_root, [lambda: P.test_schatten_norms_closed_form(2),
                                       lambda: P.test_objective_closed_form(2),
                                       lambda: P.test_schatten_norms_from_gram_eigenvalues(2)]),
    ("schatten_norms", _sum_for_max, [lambda: P.test_schatten_norms_closed_form(np.inf),
                                      lambda: P.test_objective_closed_form(np.inf)]),
]


@pytest.mark.parametrize("idx", range(len(MUTATIONS)))
def test_planted_mistake_is_caught(idx, monkeypatch):
    name, bad, pins = MUTATIONS[idx]
    monkeypatch.setattr(O, name, bad)
    caught = 0
    for pin in pins:
        try:
            with np.errstate(all="ignore"):
                pin()
        except (AssertionError, FloatingPointError, ValueError, np.linalg.LinAlgError):
            caught += 1
    assert caught == len(pins), f"mutation of {name} slipped through"
