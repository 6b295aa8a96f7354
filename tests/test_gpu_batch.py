"""Batches of uneven images (segsalsa_str_batch_*) and explicit tilings.

Each image of a batch runs the same kernels on the same data as a single handle with the same
tiling, and the kernels are deterministic, so a batch must reproduce the single-handle iterates
bit for bit; parity with the FP64 oracle then follows from the single-handle parity, and is
also checked directly on small images. A tiling changes only the summation grouping of the
rhs partials, so any tiling stays within the FP32 tolerance (1e-4 max-abs on z) of the oracle."""
import numpy as np
import pytest

from oracle import segsalsa_str_oracle as O
from paper_1504_07028_gb300 import synth
from tests.helpers import label_agreement, max_abs

pytestmark = pytest.mark.gpu

# (H, W, K, M, schatten p, precision): uneven sizes, K, patch sizes, norms and precisions,
# including prime row lengths (Bluestein) and padded lanes
CASES = [
    (33, 47, 4, 1, 1, "fp32"),
    (40, 40, 8, 1, 2, "fp32"),
    (29, 61, 16, 1, np.inf, "fp32"),
    (50, 35, 5, 2, 1, "fp32"),
    (37, 37, 3, 0, 2, "fp64"),
    (24, 53, 12, 1, 1, "fp64"),
]


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_07028_gb300 import binding
    return binding


def _params(B, case, lam=1.5, mu=1.0):
    H, W, K, M, sp, prec = case
    return B.make_params(H, W, K, M=M, sigma=0.5 if M == 1 else 1.0, lam=lam, mu=mu,
                         schatten_p=sp, precision=prec)


def _scene(case, j):
    H, W, K = case[:3]
    return synth.scene(H, W, K, S=2 * K, gap=2.0, noise_std=1.0, wrong_frac=0.0, seed=700 + j)


def _dt(case):
    return np.float64 if case[5] == "fp64" else np.float32


def _single(B, case, tiling, p, iters, lam=1.5):
    s = B.Solver(_params(B, case, lam=lam), tiling=B.make_tiling(*tiling))
    s.set_probs(p)
    s.solve(iters)
    z = s.get_z()
    s.close()
    return z


@pytest.mark.parametrize("lanes", [1, 2, 6])
def test_batch_reproduces_single_handles_bitwise(B, lanes):
    scenes = [_scene(c, j) for j, c in enumerate(CASES)]
    b = B.Batch([_params(B, c) for c in CASES])
    b.set_lanes(lanes)
    assert b.lanes() == lanes
    for j, c in enumerate(CASES):
        b.image(j).set_probs(scenes[j].p.astype(_dt(c)))
    b.solve(7)
    b.solve(18)          # continues: 25 iterations in all
    for j, c in enumerate(CASES):
        img = b.image(j)
        assert img.get_iteration() == 25
        z = img.get_z()
        ref = _single(B, c, img.tiling(), scenes[j].p.astype(_dt(c)), 25)
        assert np.array_equal(z, ref), (j, max_abs(z, ref))
    b.close()


def test_batch_matches_oracle(B):
    """Every image of a mixed-precision batch against the FP64 oracle: FP64 images at rounding
    level, FP32 images within 1e-4 with labels identical off the 1e-3 margin band."""
    iters = 30
    scenes = [_scene(c, j) for j, c in enumerate(CASES)]
    b = B.Batch([_params(B, c) for c in CASES])
    for j, c in enumerate(CASES):
        b.image(j).set_probs(scenes[j].p.astype(_dt(c)))
    b.solve(iters)
    for j, c in enumerate(CASES):
        H, W, K, M, sp, prec = c
        p = scenes[j].p.astype(_dt(c)).astype(np.float64)
        ref, _ = O.solve(p, M, 0.5 if M == 1 else 1.0, 1.5, 1.0, sp, iters)
        z = b.image(j).get_z()
        err = max_abs(z, ref.z)
        assert err < (1e-9 if prec == "fp64" else 1e-4), (j, err)
        ok, _ = label_agreement(z, ref.z)
        assert ok, j
    b.close()


def test_batch_resumes_from_checkpoint_and_fresh_probs(B):
    """An image restored by set_state (dense rhs) and an image at iteration 0 in the same batch
    solve: each ends where its single handle would."""
    c0, c1 = CASES[0], CASES[1]
    s0, s1 = _scene(c0, 0), _scene(c1, 1)
    b = B.Batch([_params(B, c0), _params(B, c1)])
    b.image(0).set_probs(s0.p.astype(np.float32))
    b.image(1).set_probs(s1.p.astype(np.float32))
    b.solve(9)
    st = b.image(0).get_state()
    b.image(0).set_state(st, 9)          # next z-update reads the dense rhs
    b.image(1).set_probs(s1.p.astype(np.float32))   # back to iteration 0
    b.solve(11)
    assert b.image(0).get_iteration() == 20 and b.image(1).get_iteration() == 11
    z0 = _single(B, c0, b.image(0).tiling(), s0.p.astype(np.float32), 20)
    z1 = _single(B, c1, b.image(1).tiling(), s1.p.astype(np.float32), 11)
    assert max_abs(b.image(0).get_z(), z0) < 1e-6
    assert np.array_equal(b.image(1).get_z(), z1)
    b.close()


@pytest.mark.parametrize("tiling", [(4, 0, 0), (32, 0, 0), (6, 1, 1), (12, 8, 2), (0, 2, 8),
                                    (0, 0, 0, 128, 8), (0, 4, 0, 256, 2), (8, 1, 4, 1024, 64),
                                    (0, 8, 1, 64, 3)])
def test_explicit_tilings_match_oracle(B, tiling):
    """K=16 scene over several tiles with a prime row length: every tiling within 1e-4."""
    sc = synth.scene(72, 41, 16, S=12, gap=2.0, noise_std=1.5, wrong_frac=0.05, seed=31)
    s = B.Solver(B.make_params(72, 41, 16, M=1, sigma=0.5, lam=1.5, mu=1.0, schatten_p=1),
                 tiling=B.make_tiling(*tiling))
    t = s.tiling()
    if tiling[0]:
        assert t[0] == tiling[0]
    s.set_probs(sc.p.astype(np.float32))
    s.solve(40)
    ref, _ = O.solve(sc.p.astype(np.float32).astype(np.float64), 1, 0.5, 1.5, 1.0, 1, 40)
    assert max_abs(s.get_z(), ref.z) < 1e-4
    s.close()


def test_batch_rejects_bad_use(B):
    c = CASES[0]
    b = B.Batch([_params(B, c), _params(B, CASES[1])])
    b.image(0).set_probs(_scene(c, 0).p.astype(np.float32))
    with pytest.raises(B.SegsalsaError) as e:
        b.solve(3)                        # image 1 has no probabilities
    assert e.value.code == B.SEGSALSA_ERR_STATE
    with pytest.raises(B.SegsalsaError) as e:
        b.solve(-1)
    assert e.value.code == B.SEGSALSA_ERR_ARG
    with pytest.raises(B.SegsalsaError) as e:
        b.set_lanes(0)
    assert e.value.code == B.SEGSALSA_ERR_ARG
    b.close()
    import torch
    st = torch.cuda.Stream()
    bad = _params(B, c)
    bad.stream = st.cuda_stream
    with pytest.raises(B.SegsalsaError) as e:
        B.Batch([bad])
    assert e.value.code == B.SEGSALSA_ERR_ARG
    with pytest.raises(B.SegsalsaError) as e:
        B.Batch([_params(B, c)], tilings=[B.make_tiling(3, 0, 0)])
    assert e.value.code == B.SEGSALSA_ERR_ARG


def test_autotune_choices_are_cached_and_correct(B):
    """The autotuner returns a tiling per image, resets the images, and its per-class choice is
    used by a later batch created without tilings; results stay within 1e-4 of the oracle."""
    cases = [(64, 72, 8, 1, 1, "fp32"), (70, 64, 8, 1, 1, "fp32"), (48, 45, 4, 1, 1, "fp32")]
    b = B.Batch([_params(B, c) for c in cases])
    chosen = b.autotune(2)
    assert len(chosen) == 3 and all(t[0] >= 4 for t in chosen)
    with pytest.raises(B.SegsalsaError) as e:
        b.solve(1)                        # autotune left the images without probabilities
    assert e.value.code == B.SEGSALSA_ERR_STATE
    b.close()
    b2 = B.Batch([_params(B, c) for c in cases])
    assert [b2.image(j).tiling() for j in range(3)] == chosen
    scenes = [_scene(c, j) for j, c in enumerate(cases)]
    for j, c in enumerate(cases):
        b2.image(j).set_probs(scenes[j].p.astype(np.float32))
    b2.solve(30)
    for j, c in enumerate(cases):
        ref, _ = O.solve(scenes[j].p.astype(np.float32).astype(np.float64), 1, 0.5, 1.5, 1.0,
                         1, 30)
        assert max_abs(b2.image(j).get_z(), ref.z) < 1e-4
    b2.close()


def test_uneven_64_image_batch_full_size(B):
    """The serving-style workload at full size: 64 images, H, W uniform in [96, 512], K in
    {4, 8, 16}, 3x3 patch, p = 1, 200 iterations. Sampled images (the smallest, the largest,
    the Bluestein-length one) must equal their single-handle solves bit for bit, z must stay
    finite, and every image's labels must agree with argmax of its own z."""
    import torch
    scenes = synth.batch_scenes()
    cfg = synth.CFG_BATCH
    params = [B.make_params(s.H, s.W, s.K, M=cfg.M, sigma=cfg.sigma, lam=cfg.lam, mu=cfg.mu,
                            schatten_p=cfg.schatten_p) for s in scenes]
    b = B.Batch(params)
    p_dev = [torch.from_numpy(s.p.astype(np.float32)).cuda() for s in scenes]
    torch.cuda.synchronize()       # the library's streams do not wait for torch's stream
    for j, s in enumerate(scenes):
        b.image(j).set_probs(p_dev[j])
    b.solve(cfg.iters)
    sizes = [s.H * s.W * s.K for s in scenes]
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 0})
    for j in sample:
        s = scenes[j]
        z = b.image(j).get_z()
        assert np.all(np.isfinite(z))
        ref = _single(B, (s.H, s.W, s.K, cfg.M, cfg.schatten_p, "fp32"), b.image(j).tiling(),
                      s.p.astype(np.float32), cfg.iters, lam=cfg.lam)
        assert np.array_equal(z, ref), j
    for j, s in enumerate(scenes):
        lab = b.image(j).get_labels()
        z = b.image(j).get_z()
        assert np.array_equal(lab, np.argmax(z, axis=0)), j
    b.close()
