"""Seeded synthetic scenes shaped like the paper's workloads (Sec. 5: a labelled scene whose
per-pixel class probabilities p_i feed problem (7)).

This module only draws inputs. It holds none of the method's arithmetic: no Jacobian, no
prox, no solve. Both the CUDA path and the FP64 oracle are fed from here, and nothing else is
shared between them.

Recipe (all draws from ``numpy.random.default_rng(seed)`` in this order):

1. Voronoi label map: ``S`` seed points uniform in ``[0,H) x [0,W)``; every pixel centre
   ``(y+0.5, x+0.5)`` takes the nearest seed (Euclidean, non-periodic, ties to the lower seed
   index); seed ``j`` carries label ``j mod K``.
2. Logits ``gap * onehot(y_i) + N(0, noise_std^2)`` i.i.d. per pixel and class.
3. Optionally a fraction ``wrong_frac`` of pixels (drawn without replacement) moves its gap to a
   class drawn uniformly among the K-1 wrong ones.
4. ``p_i = softmax(logits_i)`` in FP64.

Arrays are class-major ``(K, H, W)`` like the hidden field z in Sec. 2 (z is K x n).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class SolverConfig:
    """Solver settings of one workload (problem (7) and the SALSA loop (12)-(14))."""

    M: int                 # patch (2M+1)x(2M+1), L = (2M+1)^2 shifts (eq. 4)
    sigma: float           # Gaussian bandwidth of the shift weights
    lam: float             # prior weight lambda of eq. (7)
    mu: float              # ADMM penalty mu of eq. (13)
    schatten_p: float      # 1, 2 or np.inf
    iters: int             # fixed iteration count (Sec. 4 stopping remark)


@dataclasses.dataclass(frozen=True)
class Scene:
    H: int
    W: int
    K: int
    labels: np.ndarray     # (H, W) int64 ground truth
    p: np.ndarray          # (K, H, W) float64 class probabilities


def voronoi_labels(rng: np.random.Generator, H: int, W: int, S: int, K: int) -> np.ndarray:
    seeds = rng.uniform(low=(0.0, 0.0), high=(float(H), float(W)), size=(S, 2))
    ys = np.arange(H, dtype=np.float64) + 0.5
    xs = np.arange(W, dtype=np.float64) + 0.5
    best = np.full((H, W), np.inf)
    arg = np.zeros((H, W), dtype=np.int64)
    for j in range(S):  # strict '<' keeps the lower index on ties
        d2 = (ys[:, None] - seeds[j, 0]) ** 2 + (xs[None, :] - seeds[j, 1]) ** 2
        take = d2 < best
        best = np.where(take, d2, best)
        arg = np.where(take, j, arg)
    return arg % K


def _softmax0(logits: np.ndarray) -> np.ndarray:
    m = logits.max(axis=0, keepdims=True)
    e = np.exp(logits - m)
    return e / e.sum(axis=0, keepdims=True)


def scene(H: int, W: int, K: int, S: int, gap: float, noise_std: float,
          wrong_frac: float, seed: int) -> Scene:
    rng = np.random.default_rng(seed)
    y = voronoi_labels(rng, H, W, S, K)
    noise = rng.normal(0.0, noise_std, size=(K, H, W))
    cls = y.copy()
    if wrong_frac > 0.0:
        n = H * W
        nw = int(round(wrong_frac * n))
        idx = rng.choice(n, size=nw, replace=False)
        shift = rng.integers(1, K, size=nw)          # uniform over the K-1 wrong classes
        flat = cls.reshape(-1)
        flat[idx] = (flat[idx] + shift) % K
    logits = noise
    logits[cls, np.arange(H)[:, None], np.arange(W)[None, :]] += gap
    return Scene(H=H, W=W, K=K, labels=y, p=_softmax0(logits))


# ---------------------------------------------------------------------------------------------
# Named workloads. Sizes follow the paper's scene (145x145, 16 classes, Sec. 5) and the
# synthetic stand-ins for the other scenes; none of the paper's data is used.
# ---------------------------------------------------------------------------------------------

def scene_64x64_k4() -> Scene:
    """64x64, K=4, 6 Voronoi seeds, logits 3*onehot + N(0,1) (seed 1)."""
    return scene(64, 64, 4, S=6, gap=3.0, noise_std=1.0, wrong_frac=0.0, seed=1)


def scene_145x145_k16() -> Scene:
    """145x145, K=16 (the shape of the paper's Indian Pines subscene), 40 seeds,
    logits 2*onehot + N(0,1.5^2), 5% of pixels with a wrong-class gap (seed 2)."""
    return scene(145, 145, 16, S=40, gap=2.0, noise_std=1.5, wrong_frac=0.05, seed=2)


def scene_256x256_k8() -> Scene:
    """256x256, K=8, 16 seeds, logits as the 64x64 scene (seed 4)."""
    return scene(256, 256, 8, S=16, gap=3.0, noise_std=1.0, wrong_frac=0.0, seed=4)


def scene_2048x2048_k16() -> Scene:
    """2048x2048, K=16, 64 seeds, logits 3*onehot + N(0,1) (seed 55)."""
    return scene(2048, 2048, 16, S=64, gap=3.0, noise_std=1.0, wrong_frac=0.0, seed=55)


def batch_scenes(count: int = 64, seed_base: int = 5000):
    """Uneven batch: H, W uniform in [96, 512]; image 0 forced to 97x509, image 1 to 512x512;
    K uniform in {4, 8, 16}; 2K Voronoi seeds; logits as the 64x64 scene."""
    out = []
    for j in range(count):
        rng = np.random.default_rng(seed_base + j)
        H, W = (int(v) for v in rng.integers(96, 513, size=2))
        K = int(rng.choice([4, 8, 16]))
        if j == 0:
            H, W = 97, 509
        elif j == 1:
            H, W = 512, 512
        out.append(scene(H, W, K, S=2 * K, gap=3.0, noise_std=1.0, wrong_frac=0.0,
                         seed=seed_base + 1000 + j))
    return out


@dataclasses.dataclass(frozen=True)
class MlrScene:
    """Spectra, MLR weights and labels of a scene whose class probabilities come from a
    multinomial logistic regression (the class model of the paper's experiments, Sec. 5)."""

    H: int
    W: int
    K: int
    d: int
    labels: np.ndarray     # (H, W) int64 ground truth
    x: np.ndarray          # (H, W, d) float64 spectra, pixel-major
    Wc: np.ndarray         # (K, d) float64 MLR weights
    b: np.ndarray          # (K,) float64 MLR biases


def mlr_scene(H: int, W: int, K: int, d: int, S: int, seed: int) -> MlrScene:
    """Voronoi labels (as in ``scene``); class means mu_k ~ U(0,1)^d; spectra
    x_i = mu_{y_i} + N(0, 0.05^2) per band; weights Wc_k = (24/d)(mu_k - mean_j mu_j) +
    N(0, 1/d) (the first term gives the true class an expected logit margin of about 2, since
    E|mu_y - mu_k|^2 / 2 = d/12 for uniform means); biases 0. Draw order: labels, means,
    noise, weight noise."""
    rng = np.random.default_rng(seed)
    y = voronoi_labels(rng, H, W, S, K)
    mu = rng.uniform(0.0, 1.0, size=(K, d))
    x = mu[y] + rng.normal(0.0, 0.05, size=(H, W, d))
    Wc = (24.0 / d) * (mu - mu.mean(axis=0, keepdims=True)) + rng.normal(
        0.0, 1.0 / np.sqrt(d), size=(K, d))
    return MlrScene(H=H, W=W, K=K, d=d, labels=y, x=x, Wc=Wc, b=np.zeros(K))


def scene_610x340_mlr() -> MlrScene:
    """610x340, K=9 classes, d=103 bands (the shape of a university hyperspectral scene),
    30 Voronoi seeds (seed 3)."""
    return mlr_scene(610, 340, 9, 103, S=30, seed=3)


CFG_64 = SolverConfig(M=1, sigma=0.5, lam=2.0, mu=1.0, schatten_p=1, iters=200)
CFG_145 = {sp: SolverConfig(M=1, sigma=0.5, lam=1.5, mu=1.0, schatten_p=sp, iters=300)
           for sp in (1, 2, np.inf)}
CFG_256 = SolverConfig(M=1, sigma=0.5, lam=2.0, mu=1.0, schatten_p=1, iters=50)
CFG_BATCH = SolverConfig(M=1, sigma=0.5, lam=2.0, mu=1.0, schatten_p=1, iters=200)
CFG_MLR = SolverConfig(M=2, sigma=1.0, lam=1.5, mu=1.0, schatten_p=1, iters=400)


def random_field(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Plain N(0, scale^2) FP64 array for operator-level checks (rhs of the linear step,
    dual variables)."""
    return np.random.default_rng(seed).normal(0.0, scale, size=shape)
