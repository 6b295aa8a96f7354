"""segsalsa_str_linear_solve_static: the z-update for callers that cannot allocate device
memory (a fixed memory budget, an outside allocator, no handle to keep). It must give the
same result as the handle's segsalsa_str_linear_solve and as the oracle's DFT solve, call after
call, while its scratch lives in the library's static device array. Collected last on purpose
(file name)."""
import numpy as np
import pytest

from oracle import segsalsa_str_oracle as O
from paper_1504_07028_gb300 import synth

pytestmark = pytest.mark.gpu

# Against the handle's FP32 z-update (the same kernels, possibly another work split)
REL_TOL = 1e-6
# Against the oracle's FP64 DFT solve: the operator is well conditioned (eigenvalues in
# [3, 3 + 8c]), so the FP32 error is of the order of eps log N; the tolerance of the
# handle's own z-update parity tests
ORACLE_TOL = 2e-5


@pytest.fixture(scope="module")
def B():
    from paper_1504_07028_gb300 import binding
    from paper_1504_07028_gb300 import build
    build.build()
    binding.load()
    return binding


def _rhs_np(H, W, K, seed):
    return synth.random_field((H, W, K), seed).astype(np.float32)


def _oracle(rhs_hwk, omega, M):
    """The oracle's z-update of the same FP32 rhs, pixel-major."""
    z = O.linear_solve(np.moveaxis(rhs_hwk.astype(np.float64), -1, 0), omega, M)
    return np.moveaxis(z, 0, -1)


@pytest.mark.parametrize("H,W,K,weights", [
    (145, 145, 16, None),          # Bluestein row length
    (64, 96, 8, None),             # 7-smooth row length
    (33, 50, 5, np.ones(9)),       # explicit weights, c = 9
])
def test_static_matches_handle_two_calls(B, H, W, K, weights):
    import torch
    s = B.Solver(B.make_params(H, W, K, M=1, sigma=0.5, weights=weights))
    c = 1.0 if weights is None else float(np.sum(np.asarray(weights) ** 2))
    om = O.gaussian_weights(1, 0.5) if weights is None else np.asarray(weights, np.float64)
    for call in range(2):
        rhs_np = _rhs_np(H, W, K, seed=100 * call + H)
        rhs = torch.from_numpy(rhs_np).cuda()
        ref = torch.empty_like(rhs)
        s.linear_solve(rhs, ref)
        out = torch.full_like(rhs, float("nan"))
        rc = B.segsalsa_str_linear_solve_static(rhs, out, c_omega=c)
        torch.cuda.synchronize()
        assert rc == B.SEGSALSA_OK
        err = (out - ref).abs().max().item()
        assert err <= REL_TOL * ref.abs().max().item(), (call, err)
        zo = _oracle(rhs_np, om, 1)
        erro = float(np.abs(out.cpu().numpy() - zo).max())
        assert erro <= ORACLE_TOL * np.abs(zo).max(), (call, erro)
    s.close()


def test_static_zero_weights_is_a_scaling(B):
    """c_omega = 0: the operator is 3 I, so z = rhs / 3 (the oracle with all shift weights 0)."""
    import torch
    H, W, K = 40, 27, 6
    rhs_np = _rhs_np(H, W, K, seed=7)
    rhs = torch.from_numpy(rhs_np).cuda()
    for call in range(2):
        out = torch.full_like(rhs, float("nan"))
        assert B.segsalsa_str_linear_solve_static(rhs, out, c_omega=0.0) == B.SEGSALSA_OK
        torch.cuda.synchronize()
        z = out.cpu().numpy()
        zo = _oracle(rhs_np, np.zeros(9), 1)
        assert np.abs(zo - rhs_np.astype(np.float64) / 3.0).max() < 1e-12
        assert np.abs(z - zo).max() <= ORACLE_TOL * np.abs(zo).max(), call


def test_static_geometries_chained_on_a_caller_stream(B):
    """Shapes A, B, A on one non-default stream, no synchronisation between the calls: each
    call that changes the geometry rebuilds the tables in the array, and the row pass that
    follows must see them. Every result matches the handle and the oracle."""
    import torch
    shapes = [(96, 80, 8), (61, 127, 4), (96, 80, 8)]       # 127: Bluestein row length
    rhs_np = [_rhs_np(H, W, K, seed=300 + j) for j, (H, W, K) in enumerate(shapes)]
    rhs = [torch.from_numpy(r).cuda() for r in rhs_np]
    outs = [torch.full_like(r, float("nan")) for r in rhs]
    torch.cuda.synchronize()
    refs = []
    for (H, W, K), r in zip(shapes, rhs):
        s = B.Solver(B.make_params(H, W, K, M=1, sigma=0.5))
        ref = torch.empty_like(r)
        s.linear_solve(r, ref)
        torch.cuda.synchronize()
        refs.append(ref.cpu().numpy())
        s.close()
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    for r, o in zip(rhs, outs):
        assert B.segsalsa_str_linear_solve_static(r, o, c_omega=1.0,
                                                  stream=st.cuda_stream) == B.SEGSALSA_OK
    st.synchronize()
    om = O.gaussian_weights(1, 0.5)
    for j, (o, ref) in enumerate(zip(outs, refs)):
        z = o.cpu().numpy()
        assert np.abs(z - ref).max() <= REL_TOL * np.abs(ref).max(), j
        zo = _oracle(rhs_np[j], om, 1)
        assert np.abs(z - zo).max() <= ORACLE_TOL * np.abs(zo).max(), j


def test_static_rejects_sizes_beyond_its_array(B):
    import torch
    H, W, K = 1024, 1024, 8      # 1024 * 513 * 8 complex > 2 Mi
    x = torch.zeros((1, 1, 1), dtype=torch.float32, device="cuda")
    lib = B.load()
    rc = lib.segsalsa_str_linear_solve_static(x.data_ptr(), x.data_ptr(), H, W, K, 1.0, None)
    assert rc == B.SEGSALSA_ERR_OOM
    rc = lib.segsalsa_str_linear_solve_static(x.data_ptr(), x.data_ptr(), 8, 8, 0, 1.0, None)
    assert rc == B.SEGSALSA_ERR_ARG
