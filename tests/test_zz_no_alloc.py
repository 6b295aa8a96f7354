"""segsalsa_str_linear_solve_static: the z-update for callers that cannot allocate device
memory (a fixed memory budget, an outside allocator, no handle to keep). It must give the
same result as the handle's segsalsa_str_linear_solve, call after call, while its scratch
lives in the library's static device array. Collected last on purpose (file name)."""
import numpy as np
import pytest

from paper_1504_07028_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1504_07028_gb300 import binding
    from paper_1504_07028_gb300 import build
    build.build()
    binding.load()
    return binding


def _rhs(H, W, K, seed):
    import torch
    return torch.from_numpy(synth.random_field((H, W, K), seed).astype(np.float32)).cuda()


@pytest.mark.parametrize("H,W,K,weights", [
    (145, 145, 16, None),          # Bluestein row length
    (64, 96, 8, None),             # 7-smooth row length
    (33, 50, 5, np.ones(9)),       # explicit weights, c = 9
])
def test_static_matches_handle_two_calls(B, H, W, K, weights):
    import torch
    s = B.Solver(B.make_params(H, W, K, M=1, sigma=0.5, weights=weights))
    c = 1.0 if weights is None else float(np.sum(np.asarray(weights) ** 2))
    for call in range(2):
        rhs = _rhs(H, W, K, seed=100 * call + H)
        ref = torch.empty_like(rhs)
        s.linear_solve(rhs, ref)
        out = torch.full_like(rhs, float("nan"))
        rc = B.segsalsa_str_linear_solve_static(rhs, out, c_omega=c)
        torch.cuda.synchronize()
        assert rc == B.SEGSALSA_OK
        err = (out - ref).abs().max().item()
        assert err <= 1e-6 * ref.abs().max().item(), (call, err)
    s.close()


def test_static_rejects_sizes_beyond_its_array(B):
    import torch
    H, W, K = 1024, 1024, 8      # 1024 * 513 * 8 complex > 2 Mi
    x = torch.zeros((1, 1, 1), dtype=torch.float32, device="cuda")
    lib = B.load()
    rc = lib.segsalsa_str_linear_solve_static(x.data_ptr(), x.data_ptr(), H, W, K, 1.0, None)
    assert rc == B.SEGSALSA_ERR_OOM
    rc = lib.segsalsa_str_linear_solve_static(x.data_ptr(), x.data_ptr(), 8, 8, 0, 1.0, None)
    assert rc == B.SEGSALSA_ERR_ARG
