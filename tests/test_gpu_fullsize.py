"""Parity of the FP32 path at the full sizes of the five workloads: z within 1e-4 max-abs of
FP64 and labels equal except where the reference's top-two margin is below 1e-3.

The FP64 reference is the oracle where it finishes in minutes (145x145 for each Schatten p
over 300 iterations, the MLR scene over 10 iterations, the two smallest batch images over 200
iterations; these run in spawned worker processes beside the GPU work), and otherwise the
GPU's FP64 path at the same size (the MLR scene over 400 iterations, every batch image, the
2048x2048 image), which the other parity tests pin to the oracle at 1e-9."""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_1504_07028_gb300 import synth
from tests import oracle_jobs as J
from tests.helpers import label_agreement, max_abs

pytestmark = pytest.mark.gpu

Z_TOL = 1e-4


@pytest.fixture(scope="module")
def B(lib):
    from paper_1504_07028_gb300 import binding
    return binding


def _bf16_values(a):
    """BF16 rounding of a (torch's round-to-nearest-even), returned as FP32 values."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(
        torch.float32).numpy()


def _batch_smallest_two():
    sizes = [s.H * s.W * s.K for s in synth.batch_scenes()]
    return [int(j) for j in np.argsort(sizes)[:2]]


@pytest.fixture(scope="module")
def oracle_refs():
    """Start every oracle job at once in spawned workers; tests collect their results."""
    old = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"        # one core per worker
    ex = cf.ProcessPoolExecutor(max_workers=6, mp_context=mp.get_context("spawn"))
    mlr = synth.scene_610x340_mlr()
    futs = {("145", sp): ex.submit(J.solve_145, sp) for sp in (1, 2, np.inf)}
    futs["mlr"] = ex.submit(J.solve_mlr, _bf16_values(mlr.x), _bf16_values(mlr.Wc), 10)
    for j in _batch_smallest_two():
        futs[("batch", j)] = ex.submit(J.solve_batch_image, j)
    yield futs
    ex.shutdown(wait=False, cancel_futures=True)
    if old is None:
        os.environ.pop("OMP_NUM_THREADS", None)
    else:
        os.environ["OMP_NUM_THREADS"] = old


def _check(z, ref, what):
    err = max_abs(z, ref)
    assert err <= Z_TOL, f"{what}: max |z - z_ref| = {err:.3e}"
    ok, _ = label_agreement(z, ref)
    assert ok, f"{what}: labels differ off the 1e-3 margin band"
    return err


def test_2048x2048_k16_against_fp64(B, oracle_refs):
    """Runs first: requesting the oracle fixture starts the oracle workers, which then work
    beside this and the following GPU tests."""
    import torch
    sc = synth.scene_2048x2048_k16()
    cfg = synth.CFG_BATCH
    p32 = torch.from_numpy(sc.p.astype(np.float32)).cuda()
    torch.cuda.synchronize()
    mk = lambda prec: B.Solver(B.make_params(sc.H, sc.W, sc.K, M=cfg.M, sigma=cfg.sigma,
                                             lam=cfg.lam, mu=cfg.mu, schatten_p=cfg.schatten_p,
                                             precision=prec))
    s32 = mk("fp32")
    s32.set_probs(p32)
    s32.solve(cfg.iters, trace_every=10)
    z32 = s32.get_z()
    s32.close()
    s64 = mk("fp64")
    s64.set_probs(p32.double())
    s64.solve(cfg.iters, trace_every=10)
    z64 = s64.get_z()
    s64.close()
    _check(z32, z64, "2048x2048 K=16 vs the FP64 GPU path")


def test_batch64_every_image_against_fp64(B, oracle_refs):
    import torch
    scenes = synth.batch_scenes()
    cfg = synth.CFG_BATCH
    mk = lambda prec: B.Batch([B.make_params(s.H, s.W, s.K, M=cfg.M, sigma=cfg.sigma,
                                             lam=cfg.lam, mu=cfg.mu, schatten_p=cfg.schatten_p,
                                             precision=prec) for s in scenes])
    b32, b64 = mk("fp32"), mk("fp64")
    for j, s in enumerate(scenes):
        b32.image(j).set_probs(s.p.astype(np.float32))
        b64.image(j).set_probs(s.p.astype(np.float32).astype(np.float64))
    b32.solve(cfg.iters)
    b64.solve(cfg.iters)
    z32 = [b32.image(j).get_z() for j in range(len(scenes))]
    for j in range(len(scenes)):
        _check(z32[j], b64.image(j).get_z(), f"batch image {j} vs the FP64 GPU path")
    b32.close()
    b64.close()
    for j in _batch_smallest_two():
        zo, _ = oracle_refs[("batch", j)].result(timeout=1500)
        _check(z32[j], zo, f"batch image {j} vs the oracle")


def test_mlr_610x340_against_oracle_and_fp64(B, oracle_refs):
    import torch
    sc = synth.scene_610x340_mlr()
    cfg = synth.CFG_MLR
    x = torch.from_numpy(sc.x.astype(np.float32)).to(torch.bfloat16).cuda()
    w = torch.from_numpy(sc.Wc.astype(np.float32)).to(torch.bfloat16).cuda()
    torch.cuda.synchronize()
    mk = lambda prec: B.Solver(B.make_params(sc.H, sc.W, sc.K, M=cfg.M, sigma=cfg.sigma,
                                             lam=cfg.lam, mu=cfg.mu, schatten_p=cfg.schatten_p,
                                             precision=prec))
    s32, s64 = mk("fp32"), mk("fp64")
    s32.set_spectra(x, w)
    s32.solve(10)
    z10 = s32.get_z()
    s32.set_spectra(x, w)
    s32.solve(cfg.iters)
    s64.set_spectra(x, w)
    s64.solve(cfg.iters)
    _check(s32.get_z(), s64.get_z(), "610x340 MLR, 400 iterations vs the FP64 GPU path")
    s32.close()
    s64.close()
    zo, _ = oracle_refs["mlr"].result(timeout=1500)
    _check(z10, zo, "610x340 MLR, 10 iterations vs the oracle")


@pytest.mark.parametrize("sp", [1, 2, np.inf])
def test_145x145_k16_300_iterations_against_oracle(B, oracle_refs, sp):
    sc = synth.scene_145x145_k16()
    cfg = synth.CFG_145[sp]
    s = B.Solver(B.make_params(sc.H, sc.W, sc.K, M=cfg.M, sigma=cfg.sigma, lam=cfg.lam,
                               mu=cfg.mu, schatten_p=cfg.schatten_p))
    s.set_probs(sc.p.astype(np.float32))
    tr = s.solve(cfg.iters, trace_every=10)
    z = s.get_z()
    lab = s.get_labels()
    s.close()
    zo, tro = oracle_refs[("145", sp)].result(timeout=1500)
    _check(z, zo, f"145x145 p={sp}")
    assert np.array_equal(lab, np.argmax(z, axis=0))
    # residuals, objective, feasibility of the trace records: FP64 sums of FP32 iterates
    assert np.allclose(tr[:, 1:4], tro[:, 1:4], rtol=2e-3, atol=1e-5)


@pytest.mark.parametrize("H,W,K,M,sp,T", [
    (1021, 1999, 16, 1, 1, 60),       # prime row length: Bluestein transform of 4000-odd points
    (1499, 2047, 8, 1, 2, 60),        # 2047 = 23 * 89: direct prime stages
    (768, 1024, 32, 1, np.inf, 60),   # K = 32 (one class per lane of a warp)
    (2048, 2048, 16, 2, 1, 20),       # the 5x5 patch on the 2048 x 2048 scene
    (512, 700, 16, 3, 1, 20)])        # a 7x7 patch (three-launch sweep) on a large image
def test_large_shapes_against_fp64(B, H, W, K, M, sp, T):
    """Large and odd shapes outside the five workloads: the FP32 handle against the FP64
    handle (itself held to the oracle at 1e-9 by the parity tests), z within 1e-4 and labels
    equal off the 1e-3 margin band."""
    sc = synth.scene(H, W, K, S=24, gap=2.0, noise_std=1.0, wrong_frac=0.05, seed=H + W)
    z = {}
    for prec, dt in (("fp32", np.float32), ("fp64", np.float64)):
        s = B.Solver(B.make_params(H, W, K, M=M, sigma=max(0.5, 0.5 * M), lam=1.5, mu=1.0,
                                   schatten_p=sp, precision=prec))
        s.set_probs(sc.p.astype(dt))
        s.solve(T, trace_every=10)
        z[prec] = s.get_z()
        s.close()
    assert np.isfinite(z["fp32"]).all()
    assert max_abs(z["fp32"], z["fp64"]) < 1e-4
    ok, _ = label_agreement(z["fp32"], z["fp64"])
    assert ok
