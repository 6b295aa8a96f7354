"""Oracle solves of the full-size workloads, run in worker processes (spawned, so that no
worker inherits a CUDA context) while the GPU tests of the same module run. Each job returns
the oracle's z (class-major, FP64) and its trace."""
import numpy as np

from oracle import segsalsa_str_oracle as O
from paper_1504_07028_gb300 import synth


def solve_145(sp):
    """145x145, K = 16, 3x3 patch, lambda = 1.5, mu = 1, 300 iterations at Schatten p."""
    sc = synth.scene_145x145_k16()
    cfg = synth.CFG_145[sp]
    p = sc.p.astype(np.float32).astype(np.float64)
    st, tr = O.solve(p, cfg.M, cfg.sigma, cfg.lam, cfg.mu, cfg.schatten_p, cfg.iters,
                     trace_every=10)
    return st.z, tr


def solve_mlr(x32, w32, iters):
    """The 610x340, K = 9 MLR workload from the BF16-rounded spectra and weights (given as
    FP32 arrays holding BF16 values): oracle probabilities, then `iters` iterations."""
    cfg = synth.CFG_MLR
    p = O.mlr_probs(x32.astype(np.float64), w32.astype(np.float64))
    st, tr = O.solve(p, cfg.M, cfg.sigma, cfg.lam, cfg.mu, cfg.schatten_p, iters)
    return st.z, tr


def solve_batch_image(j):
    """Image j of the 64-image uneven batch, 200 iterations."""
    sc = synth.batch_scenes()[j]
    cfg = synth.CFG_BATCH
    p = sc.p.astype(np.float32).astype(np.float64)
    st, tr = O.solve(p, cfg.M, cfg.sigma, cfg.lam, cfg.mu, cfg.schatten_p, cfg.iters)
    return st.z, tr
