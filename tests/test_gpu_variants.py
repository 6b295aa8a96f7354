"""Method variants: g4 read as the probability simplex indicator (segsalsa_str_set_g4) and the
residual-based stopping rule of Sec. 4 (segsalsa_str_solve_until), against the FP64 oracle."""
import numpy as np
import pytest

from oracle import segsalsa_str_oracle as O
from paper_1504_07028_gb300 import synth
from tests.helpers import label_agreement, max_abs

pytestmark = pytest.mark.gpu
SP = {1: 1, 2: 2, "inf": np.inf}


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_07028_gb300 import binding
    return binding


def _solver(B, sc, M, sp, prec, lam=1.5, mu=1.0):
    return B.Solver(B.make_params(sc.H, sc.W, sc.K, M=M, sigma=0.5 if M == 1 else 1.0, lam=lam,
                                  mu=mu, schatten_p=sp, precision=prec))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("H,W,K,M,sp", [(31, 29, 5, 1, 1), (24, 37, 16, 1, "inf"), (20, 22, 3, 2, 2),
                                        (17, 19, 32, 0, 1)])
def test_g4_simplex_matches_oracle(B, prec, H, W, K, M, sp):
    sc = synth.scene(H, W, K, S=4, gap=1.5, noise_std=1.5, wrong_frac=0.1, seed=80 + K)
    dt = np.float64 if prec == "fp64" else np.float32
    p = sc.p.astype(dt)
    s = _solver(B, sc, M, sp, prec)
    s.set_g4("simplex")
    s.set_probs(p)
    tr = s.solve(40, trace_every=10)
    ref, rtr = O.solve(p.astype(np.float64), M, 0.5 if M == 1 else 1.0, 1.5, 1.0, SP[sp], 40,
                       trace_every=10, g4="simplex")
    z = s.get_z()
    assert max_abs(z, ref.z) < (1e-9 if prec == "fp64" else 1e-4)
    ok, _ = label_agreement(z, ref.z)
    assert ok
    if prec == "fp64":
        assert np.allclose(tr, rtr, rtol=1e-7, atol=1e-9)
    s.close()


def test_g4_switch_midway_and_back(B):
    sc = synth.scene(26, 30, 6, S=5, gap=1.5, noise_std=1.0, wrong_frac=0.05, seed=90)
    s = _solver(B, sc, 1, 1, "fp64")
    s.set_probs(sc.p)
    s.solve(10)
    s.set_g4("simplex")
    s.solve(10)
    s.set_g4("affine")
    s.solve(5)
    st, _ = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 1, 10)
    st, _ = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 1, 10, state=st, g4="simplex")
    st, _ = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 1, 5, state=st)
    assert s.get_iteration() == 25
    assert max_abs(s.get_z(), st.z) < 1e-9
    with pytest.raises(B.SegsalsaError) as e:
        s.set_g4(7)
    assert e.value.code == B.SEGSALSA_ERR_ARG
    s.close()


def test_g4_switch_reaches_batch_graphs(B):
    """A batch captured its graphs with the affine sweep; switching an image to the simplex
    variant must re-capture them (the image then equals a single simplex handle bit for bit)."""
    sc0 = synth.scene(28, 33, 4, S=4, gap=1.5, noise_std=1.0, wrong_frac=0.0, seed=91)
    sc1 = synth.scene(30, 21, 8, S=4, gap=1.5, noise_std=1.0, wrong_frac=0.0, seed=92)
    mk = lambda sc: B.make_params(sc.H, sc.W, sc.K, M=1, sigma=0.5, lam=1.5, mu=1.0, schatten_p=1)
    b = B.Batch([mk(sc0), mk(sc1)])
    b.image(0).set_probs(sc0.p.astype(np.float32))
    b.image(1).set_probs(sc1.p.astype(np.float32))
    b.solve(6)
    b.image(1).set_g4("simplex")
    b.solve(12)
    s = B.Solver(mk(sc1), tiling=B.make_tiling(*b.image(1).tiling()))
    s.set_probs(sc1.p.astype(np.float32))
    s.solve(6)
    s.set_g4("simplex")
    s.solve(12)
    assert np.array_equal(b.image(1).get_z(), s.get_z())
    s.close()
    b.close()


def test_solve_until_stops_where_the_oracle_does(B):
    sc = synth.scene(30, 28, 5, S=5, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=93)
    _, rtr = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 1, 300, trace_every=10)
    # thresholds set from the oracle's record at k = 120; the stop is the first record at or
    # under both of them
    row = rtr[np.searchsorted(rtr[:, 0], 120)]
    tp, td = 1.03 * row[1], 1.03 * row[2]
    hit = np.nonzero((rtr[:, 1] <= tp) & (rtr[:, 2] <= td))[0][0]
    k_star = int(rtr[hit, 0])
    s = _solver(B, sc, 1, 1, "fp64")
    s.set_probs(sc.p)
    n, rec = s.solve_until(300, tp, td, check_every=10)
    assert n == k_star
    assert np.allclose(rec, rtr[hit], rtol=1e-7, atol=1e-9)
    ref, _ = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 1, k_star)
    assert max_abs(s.get_z(), ref.z) < 1e-9
    # FP32 stops within one check period of the FP64 count
    s32 = _solver(B, sc, 1, 1, "fp32")
    s32.set_probs(sc.p.astype(np.float32))
    n32, _ = s32.solve_until(300, tp, td, check_every=10)
    assert abs(n32 - k_star) <= 10
    # zero tolerances run to max_iters; a short last block is allowed
    s.set_probs(sc.p)
    n0, rec0 = s.solve_until(37, 0.0, 0.0, check_every=10)
    assert n0 == 37 and rec0[0] == 37 and s.get_iteration() == 37
    with pytest.raises(B.SegsalsaError) as e:
        s.solve_until(10, 1e-3, 1e-3, check_every=0)
    assert e.value.code == B.SEGSALSA_ERR_ARG
    with pytest.raises(B.SegsalsaError) as e:
        s.solve_until(10, -1.0, 1e-3)
    assert e.value.code == B.SEGSALSA_ERR_ARG
    s.close()
    s32.close()
