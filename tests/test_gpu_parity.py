"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 GPU path 1e-9 max-abs on z (rounding only); FP32 path 1e-4 max-abs on z
(the stated bound), labels identical except where the oracle's top-two margin is < 1e-3.
Operator-level checks use tolerances derived from FP32 rounding (see each test)."""
import numpy as np
import pytest

from oracle import segsalsa_str_oracle as O
from paper_1504_07028_gb300 import synth
from tests.helpers import (d2_abi_to_oracle, hwk_to_khw, khw_to_hwk, label_agreement, max_abs,
                           oracle_state_to_abi)

pytestmark = pytest.mark.gpu

SP = {1: 1, 2: 2, "inf": np.inf}


def _solver(B, H, W, K, M, sigma, lam, mu, sp, prec):
    from paper_1504_07028_gb300 import binding as Bd
    return Bd.Solver(Bd.make_params(H, W, K, M=M, sigma=sigma, lam=lam, mu=mu,
                                    schatten_p=sp, precision=prec))


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_07028_gb300 import binding
    return binding


# ------------------------------------------------------------------ z-update (eq. 12) alone

@pytest.mark.parametrize("H,W,K,M,prec", [
    (64, 64, 4, 1, "fp64"), (64, 64, 4, 1, "fp32"), (145, 145, 16, 1, "fp32"),
    (37, 50, 5, 2, "fp32"), (12, 9, 3, 0, "fp64"), (4, 4, 2, 1, "fp64"), (97, 509, 4, 1, "fp32"),
    (256, 256, 8, 1, "fp32"), (61, 2048, 3, 1, "fp32"), (33, 17, 32, 1, "fp32"),
    # rows with two prime factors above 7 (the second direct stage twiddles its input) and
    # with a radix-7 / radix-3 tail after a direct stage
    (40, 143, 4, 1, "fp32"), (24, 121, 3, 1, "fp64"), (18, 2 * 3 * 7 * 13, 5, 1, "fp64"),
    # the largest direct prime (103) and the smallest row length sent to Bluestein (127)
    (20, 206, 4, 1, "fp64"), (30, 127, 3, 1, "fp32")])
def test_linear_solve(B, H, W, K, M, prec):
    s = _solver(B, H, W, K, M, 0.5 + 0.5 * M, 1.0, 1.0, 1, prec)
    dt = np.float64 if prec == "fp64" else np.float32
    rhs = synth.random_field((K, H, W), seed=H * 1000 + W).astype(dt)
    z = hwk_to_khw(s.linear_solve(khw_to_hwk(rhs)))
    ref = O.linear_solve(rhs.astype(np.float64), O.gaussian_weights(M, 0.5 + 0.5 * M), M)
    # the operator is well conditioned (eigenvalues in [3, 3 + 8c]); FP32 error ~ eps log N
    tol = 1e-11 if prec == "fp64" else 2e-5
    assert max_abs(z, ref) <= tol * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_linear_solve_element_aligned_device_buffers(B, prec):
    """Device rhs and z that are views one element into their buffers (aligned to the element,
    not to 16 bytes): the transforms fall back from 16-byte accesses and the result is the same
    as from aligned buffers."""
    import torch
    H, W, K = 40, 48, 16
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    rhs = synth.random_field((K, H, W), seed=31).astype(dt)
    ref = O.linear_solve(rhs.astype(np.float64), O.gaussian_weights(1, 0.5), 1)
    s = B.Solver(B.make_params(H, W, K, M=1, sigma=0.5, precision=prec))
    hwk = torch.from_numpy(np.ascontiguousarray(khw_to_hwk(rhs))).cuda()
    buf_r = torch.zeros(H * W * K + 1, dtype=tdt, device="cuda")
    buf_z = torch.zeros(H * W * K + 1, dtype=tdt, device="cuda")
    r1, z1 = buf_r[1:].view(H, W, K), buf_z[1:].view(H, W, K)
    r1.copy_(hwk)
    assert r1.data_ptr() % 16 != 0 and z1.data_ptr() % 16 != 0
    s.linear_solve(r1, z1)
    z0 = s.linear_solve(hwk.clone())
    torch.cuda.synchronize()
    assert torch.equal(z0, z1)
    tol = 1e-11 if prec == "fp64" else 2e-5
    assert max_abs(hwk_to_khw(z1.cpu().numpy()), ref) <= tol * np.abs(ref).max()
    s.close()


@pytest.mark.parametrize("H,W,K,M,prec,wscale", [
    (64, 64, 4, 1, "fp64", 1.0), (145, 145, 16, 1, "fp32", 1.0), (37, 50, 5, 2, "fp32", 1.0),
    (33, 17, 32, 1, "fp32", 1.0), (96, 131, 4, 1, "fp32", 1.0), (40, 37, 8, 1, "fp64", 5.0),
    (71, 64, 6, 1, "fp32", 5.0), (35, 24, 3, 0, "fp64", 3.0)])
def test_linear_solve_cluster_bands(B, H, W, K, M, prec, wscale):
    """The z-update fused over a thread-block cluster (every cluster size that the image admits)
    against the oracle's DFT solve and the three-launch path. wscale > 1 scales the shift
    weights: the column recursions then decay slowly and a band's start values come from
    several other bands, or from the whole period."""
    om = wscale * O.gaussian_weights(M, 0.5 + 0.5 * M)
    dt = np.float64 if prec == "fp64" else np.float32
    rhs = synth.random_field((K, H, W), seed=H * 1000 + W + 7).astype(dt)
    ref = O.linear_solve(rhs.astype(np.float64), om, M)
    tol = 1e-11 if prec == "fp64" else 2e-5
    mk = lambda zf: B.Solver(B.make_params(H, W, K, M=M, sigma=0.5 + 0.5 * M, precision=prec,
                                           weights=om), tiling=B.make_tiling(zfuse=zf))
    s1 = mk(1)
    assert s1.tiling()[5] == 1
    z1 = hwk_to_khw(s1.linear_solve(khw_to_hwk(rhs)))
    assert max_abs(z1, ref) <= tol * np.abs(ref).max()
    fused = 0
    for cs in (2, 4, 8, 16):
        if H < 2 * cs:
            continue
        s = mk(cs)
        if s.tiling()[5] != cs:          # the band does not fit: three launches
            assert s.tiling()[5] == 1
            continue
        fused += 1
        s.set_profiling(True)
        z = hwk_to_khw(s.linear_solve(khw_to_hwk(rhs)))
        assert s.kernel_stats()["zupdate_fused"][0] == 1
        assert max_abs(z, ref) <= tol * np.abs(ref).max(), cs
        assert max_abs(z, z1) <= 2 * tol * np.abs(ref).max(), cs
        s.close()
    assert fused >= 2
    s1.close()


def test_solve_fused_and_three_launch_agree(B):
    """Whole solves on a 145 x 145, K = 16 image with the z-update fused over 8-CTA clusters
    and with the default (three launches): both reach the oracle's iterate."""
    sc = synth.scene(145, 145, 16, S=40, gap=2.0, noise_std=1.5, wrong_frac=0.05, seed=2)
    out = []
    for zf in (8, 0):
        s = B.Solver(B.make_params(145, 145, 16, M=1, sigma=0.5, lam=1.5, mu=1.0, schatten_p=1,
                                   precision="fp32"), tiling=B.make_tiling(zfuse=zf))
        assert s.tiling()[5] == (8 if zf == 8 else 1)
        s.set_probs(sc.p.astype(np.float32))
        s.solve(60)
        out.append(s.get_z())
        s.close()
    ref, _ = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 1, 60)
    for z in out:
        assert max_abs(z, ref.z) < 1e-4
    assert max_abs(out[0], out[1]) < 1e-5


# ------------------------------------------------ sweep (eqs. 13-14 + next rhs) alone

@pytest.mark.parametrize("H,W,K,M,sp,prec", [
    (31, 29, 4, 1, 1, "fp64"), (31, 29, 4, 1, 1, "fp32"), (20, 40, 16, 1, "inf", "fp32"),
    (20, 40, 16, 1, 2, "fp32"), (23, 26, 9, 2, 1, "fp32"), (17, 19, 3, 0, 1, "fp64"),
    (10, 12, 32, 1, 1, "fp32"), (6, 6, 5, 2, "inf", "fp64")])
def test_sweep_step(B, H, W, K, M, sp, prec):
    """From an oracle state (z^k, d^k) the GPU sweep (iteration run with the z-update skipped,
    i.e. set_state with k = 0) must give the oracle's d^{k+1} and G^T(u^{k+1} + d^{k+1})."""
    sc = synth.scene(H, W, K, S=5, gap=2.0, noise_std=1.0, wrong_frac=0.05, seed=H + W + K)
    sigma, lam, mu = 0.5 + 0.5 * M, 1.5, 1.3
    om = O.gaussian_weights(M, sigma)
    dt = np.float64 if prec == "fp64" else np.float32
    p = sc.p.astype(dt).astype(np.float64)
    st, _ = O.solve(p, M, sigma, lam, mu, SP[sp], 7, omega=om)      # nonzero duals
    s = _solver(B, H, W, K, M, sigma, lam, mu, SP[sp], prec)
    s.set_probs(p.astype(dt))
    a = oracle_state_to_abi(st, om, M, dt)
    a["rhs"] = None
    s.set_state(a, 0)
    s.solve(1)
    g = s.get_state()
    u, dn, _ = O.u_d_update(a["z"].astype(np.float64).transpose(2, 0, 1),
                            [np.asarray(x, np.float64) for x in
                             (hwk_to_khw(a["d1"]), d2_abi_to_oracle(a["d2"]), hwk_to_khw(a["d3"]),
                              hwk_to_khw(a["d4"]))], p, lam, mu, om, M, SP[sp])
    rhs = O.apply_GT([x + y for x, y in zip(u, dn)], om, M)
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert max_abs(hwk_to_khw(g["d1"]), dn[0]) <= tol
    assert max_abs(d2_abi_to_oracle(g["d2"]), dn[1]) <= tol
    assert max_abs(hwk_to_khw(g["d3"]), dn[2]) <= tol
    assert max_abs(hwk_to_khw(g["d4"]), dn[3]) <= tol
    assert max_abs(hwk_to_khw(g["rhs"]), rhs) <= 4 * tol * max(1.0, np.abs(rhs).max())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_one_full_iteration_from_checkpoint(B, prec):
    """set_state(k > 0) then one iteration: z-update from rhs^k, then the sweep."""
    H, W, K, M, sigma, lam, mu = 26, 35, 6, 1, 0.5, 2.0, 1.0
    sc = synth.scene(H, W, K, S=4, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=5)
    om = O.gaussian_weights(M, sigma)
    dt = np.float64 if prec == "fp64" else np.float32
    p = sc.p.astype(dt).astype(np.float64)
    st, _ = O.solve(p, M, sigma, lam, mu, 1, 5, omega=om)
    nxt, _, _ = O.salsa_step(st, p, lam, mu, om, M, 1)
    s = _solver(B, H, W, K, M, sigma, lam, mu, 1, prec)
    s.set_probs(p.astype(dt))
    s.set_state(oracle_state_to_abi(st, om, M, dt), st.k)
    s.solve(1)
    assert s.get_iteration() == st.k + 1
    g = s.get_state()
    tol = 1e-10 if prec == "fp64" else 3e-5
    assert max_abs(hwk_to_khw(g["z"]), nxt.z) <= tol
    assert max_abs(d2_abi_to_oracle(g["d2"]), nxt.d[1]) <= tol
    assert max_abs(hwk_to_khw(g["rhs"]), nxt.rhs(om, M)) <= 4 * tol


# ---------------------------------------------------------------- full solves vs oracle

def _full(B, sc, M, sigma, lam, mu, sp, iters, prec, trace_every=10):
    dt = np.float64 if prec == "fp64" else np.float32
    p = sc.p.astype(dt)
    s = _solver(B, sc.H, sc.W, sc.K, M, sigma, lam, mu, sp, prec)
    s.set_probs(p)
    tr = s.solve(iters, trace_every=trace_every)
    z = s.get_z()
    lab = s.get_labels()
    ref, rtr = O.solve(p.astype(np.float64), M, sigma, lam, mu, sp, iters,
                       trace_every=trace_every)
    return z, lab, tr, ref, rtr


def test_scene_64x64_k4_fp64_and_fp32(B):
    """The 64x64, K=4, 3x3 patch, lambda=2 scene for 200 iterations: FP64 GPU path at rounding
    level, FP32 path within 1e-4 of the FP64 oracle, identical labels off the margin band."""
    sc = synth.scene_64x64_k4()
    cfg = synth.CFG_64
    z64, lab64, tr64, ref, rtr = _full(B, sc, cfg.M, cfg.sigma, cfg.lam, cfg.mu, cfg.schatten_p,
                                       cfg.iters, "fp64")
    assert max_abs(z64, ref.z) < 1e-9
    assert np.array_equal(lab64, np.argmax(ref.z, axis=0))
    assert np.allclose(tr64, rtr, rtol=1e-7, atol=1e-9)
    dt = np.float32
    s = _solver(B, sc.H, sc.W, sc.K, cfg.M, cfg.sigma, cfg.lam, cfg.mu, cfg.schatten_p, "fp32")
    s.set_probs(sc.p.astype(dt))
    tr32 = s.solve(cfg.iters, trace_every=10)
    z32 = s.get_z()
    ref32, _ = O.solve(sc.p.astype(dt).astype(np.float64), cfg.M, cfg.sigma, cfg.lam, cfg.mu,
                       cfg.schatten_p, cfg.iters)
    err = max_abs(z32, ref32.z)
    assert err < 1e-4, err
    ok, band = label_agreement(z32, ref32.z)
    assert ok
    assert np.allclose(tr32[:, 3], rtr[:, 3], rtol=1e-4)


@pytest.mark.parametrize("sp", [1, 2, "inf"])
def test_k16_scene_each_schatten_p(B, sp):
    """K=16 classes, 3x3 patch, lambda=1.5 as in the 145x145 workload, at a size the oracle
    runs in seconds; W = 37 is prime (Bluestein rows), H = 40 spans several tiles."""
    sc = synth.scene(40, 37, 16, S=12, gap=2.0, noise_std=1.5, wrong_frac=0.05, seed=21)
    z, lab, tr, ref, rtr = _full(B, sc, 1, 0.5, 1.5, 1.0, SP[sp], 60, "fp32")
    ref32, _ = O.solve(sc.p.astype(np.float32).astype(np.float64), 1, 0.5, 1.5, 1.0, SP[sp], 60)
    assert max_abs(z, ref32.z) < 1e-4
    ok, _ = label_agreement(z, ref32.z)
    assert ok
    assert np.allclose(tr[:, 1:4], rtr[:, 1:4], rtol=2e-3, atol=1e-5)


def test_5x5_patch_k9(B):
    """5x5 patch (M=2, sigma=1), K=9 (padded lanes), odd sizes."""
    sc = synth.scene(33, 47, 9, S=8, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=22)
    z, lab, tr, ref, rtr = _full(B, sc, 2, 1.0, 1.5, 1.0, 1, 40, "fp64")
    assert max_abs(z, ref.z) < 1e-9
    s = _solver(B, sc.H, sc.W, sc.K, 2, 1.0, 1.5, 1.0, 1, "fp32")
    s.set_probs(sc.p.astype(np.float32))
    s.solve(40)
    ref32, _ = O.solve(sc.p.astype(np.float32).astype(np.float64), 2, 1.0, 1.5, 1.0, 1, 40)
    assert max_abs(s.get_z(), ref32.z) < 1e-4


def test_vtv_one_pixel_patch(B):
    """M = 0: SegSALSA with the VTV prior (Sec. 3)."""
    sc = synth.scene(30, 24, 5, S=6, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=23)
    z, lab, tr, ref, rtr = _full(B, sc, 0, 1.0, 1.2, 0.8, 2, 50, "fp64")
    assert max_abs(z, ref.z) < 1e-9


# ------------------------------------------------------------------------- edge cases

@pytest.mark.parametrize("H,W,K,M", [(4, 4, 2, 1), (6, 6, 2, 2), (2, 2, 3, 0), (5, 131, 32, 1),
                                     (200, 5, 7, 1), (3, 3, 2, 0)])
def test_small_and_degenerate_shapes(B, H, W, K, M):
    sc = synth.scene(H, W, K, S=2, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=H * W + K)
    z, lab, tr, ref, rtr = _full(B, sc, M, 0.5 + 0.5 * M, 1.5, 1.0, 1, 15, "fp64", trace_every=5)
    assert max_abs(z, ref.z) < 1e-9
    assert np.allclose(tr, rtr, rtol=1e-6, atol=1e-9)


def test_lambda_zero_and_constant_p(B):
    sc = synth.scene(16, 16, 3, S=4, gap=1.0, noise_std=1.0, wrong_frac=0.0, seed=32)
    s = _solver(B, 16, 16, 3, 1, 0.5, 0.0, 1.0, 1, "fp32")
    s.set_probs(sc.p.astype(np.float32))
    s.solve(400)
    lab = s.get_labels()
    srt = np.sort(sc.p, axis=0)
    clear = srt[-1] - srt[-2] > 0.02
    assert np.array_equal(lab[clear], np.argmax(sc.p, axis=0)[clear])
    p1 = np.array([0.1, 0.5, 0.15, 0.25])
    pc = np.broadcast_to(p1[:, None, None], (4, 12, 10)).astype(np.float32).copy()
    s = _solver(B, 12, 10, 4, 1, 0.5, 2.0, 1.0, 1, "fp32")
    s.set_probs(pc)
    s.solve(100)
    zc = s.get_z()
    assert np.abs(zc - zc[:, :1, :1]).max() < 1e-6
    assert (s.get_labels() == 1).all()


def test_zero_iterations_and_continuation(B):
    sc = synth.scene(20, 22, 4, S=3, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=33)
    s = _solver(B, 20, 22, 4, 1, 0.5, 1.5, 1.0, 1, "fp64")
    s.set_probs(sc.p)
    s.solve(0)
    assert max_abs(s.get_z(), sc.p / sc.p.sum(0)) < 1e-15
    s.solve(7)
    s.solve(5)
    ref, _ = O.solve(sc.p, 1, 0.5, 1.5, 1.0, 1, 12)
    assert max_abs(s.get_z(), ref.z) < 1e-10
    # layouts of get_z agree
    zh = s.get_z(layout=1)
    assert np.array_equal(hwk_to_khw(zh), s.get_z())


def test_device_pointers_and_scale_invariance(B):
    import torch
    sc = synth.scene(32, 30, 8, S=5, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=34)
    s = _solver(B, 32, 30, 8, 1, 0.5, 1.5, 1.0, 1, "fp32")
    pt = torch.from_numpy(khw_to_hwk(sc.p.astype(np.float32))).cuda()
    torch.cuda.synchronize()       # the handle's stream does not wait for torch's stream
    s.set_probs(pt, layout=1)
    s.solve(20)
    zd = torch.empty((8, 32, 30), dtype=torch.float32, device="cuda")
    s.get_z(zd)
    ld = torch.empty((32, 30), dtype=torch.int32, device="cuda")
    s.get_labels(ld)
    c = np.random.default_rng(3).uniform(0.1, 10, size=(1, 32, 30)).astype(np.float32)
    s2 = _solver(B, 32, 30, 8, 1, 0.5, 1.5, 1.0, 1, "fp32")
    s2.set_probs((sc.p.astype(np.float32) * c).astype(np.float32))
    s2.solve(20)
    assert max_abs(zd.cpu().numpy(), s2.get_z()) < 2e-5
    assert np.array_equal(ld.cpu().numpy(), s.get_labels())


# ------------------------------------------------------------------------- error paths

def test_invalid_inputs_are_rejected(B):
    s = _solver(B, 8, 8, 3, 1, 0.5, 1.0, 1.0, 1, "fp32")
    with pytest.raises(B.SegsalsaError) as e:
        s.solve(3)
    assert e.value.code == B.SEGSALSA_ERR_STATE
    p = np.full((3, 8, 8), 1 / 3, dtype=np.float32)
    bad = p.copy(); bad[1, 2, 3] = -0.1
    with pytest.raises(B.SegsalsaError):
        s.set_probs(bad)
    bad = p.copy(); bad[0, 0, 0] = np.nan
    with pytest.raises(B.SegsalsaError):
        s.set_probs(bad)
    bad = p.copy(); bad[:, 4, 4] = 0.0
    with pytest.raises(B.SegsalsaError):
        s.set_probs(bad)
    with pytest.raises(B.SegsalsaError):   # still no state after the failed calls
        s.get_labels()
    s.set_probs(p)
    with pytest.raises(B.SegsalsaError):
        s.solve(-1)
    with pytest.raises(TypeError):
        s.set_probs(p.astype(np.float64))


def test_graph_replay_matches_eager_launches(B):
    """solve() replays captured CUDA graphs of whole trace periods; with profiling on it
    launches every kernel eagerly. Both must give bit-identical iterates and traces."""
    sc = synth.scene(37, 41, 6, S=5, gap=2.0, noise_std=1.0, wrong_frac=0.05, seed=40)
    out = []
    for prof in (False, True):
        s = _solver(B, 37, 41, 6, 1, 0.5, 1.5, 1.0, 1, "fp32")
        s.set_profiling(prof)
        s.set_probs(sc.p.astype(np.float32))
        tr = s.solve(47, trace_every=10)
        s.solve(35)                       # untraced: 16-iteration graphs plus a tail
        out.append((tr, s.get_z(), s.get_iteration()))
    (t0, z0, k0), (t1, z1, k1) = out
    assert k0 == k1 == 82
    assert np.array_equal(t0, t1)
    assert np.array_equal(z0, z1)
    assert list(t0[:, 0]) == [10, 20, 30, 40, 47]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_compact_local_duals_are_transparent(B, prec):
    """The affine sweep keeps d1 = c1 p and d4 = c4 1 as two scalars per pixel (the forms the
    MPOs of g1 and g4 leave); get_state expands them. Reading the state in the middle of a solve
    (which switches the handle to the full form for one sweep) must not change the iterates by a
    bit, and the expanded duals must be the oracle's."""
    H, W, K, M = 33, 41, 6, 1
    sc = synth.scene(H, W, K, S=5, gap=2.0, noise_std=1.0, wrong_frac=0.05, seed=97)
    dt = np.float64 if prec == "fp64" else np.float32
    p = sc.p.astype(dt)
    a = _solver(B, H, W, K, M, 0.5, 1.5, 1.0, 1, prec)
    b = _solver(B, H, W, K, M, 0.5, 1.5, 1.0, 1, prec)
    a.set_probs(p)
    b.set_probs(p)
    a.solve(40, trace_every=10)
    b.solve(17, trace_every=10)
    g = b.get_state()                       # mid-solve: the duals leave the compact form
    b.solve(23, trace_every=10)
    assert np.array_equal(a.get_z(), b.get_z())
    assert np.array_equal(a.get_state()["d1"], b.get_state()["d1"])
    st, _ = O.solve(p.astype(np.float64), M, 0.5, 1.5, 1.0, 1, 17)
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert max_abs(hwk_to_khw(g["d1"]), st.d[0]) <= tol
    assert max_abs(hwk_to_khw(g["d3"]), st.d[2]) <= tol
    assert max_abs(hwk_to_khw(g["d4"]), st.d[3]) <= tol
    # d4 is the same for every class of a pixel, d1 is parallel to p
    assert np.array_equal(g["d4"], np.repeat(g["d4"][..., :1], K, axis=-1))
    a.close()
    b.close()
