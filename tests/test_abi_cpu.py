"""CPU-side checks of the C ABI: the shared library builds for sm_103a, loads without a GPU,
exports every function declared in include/segsalsa_str.h, and its host-side parameter checks
and planning (workspace sizing) behave. No compute call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1504_07028_gb300 import binding as B
from paper_1504_07028_gb300 import build as Bu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    Bu.build()
    return B.load()


def _declared():
    hdr = open(os.path.join(ROOT, "include", "segsalsa_str.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(segsalsa_str_[a-z_0-9]+)\s*\(", hdr)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 16
    raw = ctypes.CDLL(B.library_path())
    for n in names:
        assert hasattr(raw, n), n
    assert set(names) == set(B.SYMBOLS)


def test_params_struct_matches_header():
    # int32 x4, pointer, 3 doubles, int32 x2, pointer: 64 bytes on LP64
    assert ctypes.sizeof(B.Params) == 64
    assert B.Params.weights.offset == 16 and B.Params.stream.offset == 56


@pytest.mark.parametrize("kw,ok", [
    (dict(H=145, W=145, K=16), True), (dict(H=3, W=3, K=4), False), (dict(H=8, W=8, K=1), False),
    (dict(H=8, W=8, K=33), False), (dict(H=8, W=8, K=4, M=3), True),
    (dict(H=12, W=12, K=4, M=5), True), (dict(H=11, W=12, K=4, M=5), False),
    (dict(H=16, W=16, K=4, M=6), False),
    (dict(H=8, W=8, K=4, lam=-1.0), False), (dict(H=8, W=8, K=4, mu=0.0), False),
    (dict(H=8, W=8, K=4, schatten_p=3), False), (dict(H=8, W=8, K=4, sigma=0.0), False),
    (dict(H=2, W=2, K=4, M=0), True), (dict(H=2048, W=2048, K=16), True),
    (dict(H=30000, W=8, K=4), False), (dict(H=8, W=9000, K=4), False),
    # the documented row-transform and column-solve limits
    (dict(H=8, W=8192, K=4), True), (dict(H=8, W=8137, K=4), True), (dict(H=8, W=8191, K=4), False),
    (dict(H=8, W=4093, K=4), True), (dict(H=8, W=4099, K=4), False),
    (dict(H=25600, W=8, K=4), True), (dict(H=25601, W=8, K=4), False),
    (dict(H=12800, W=8, K=4, precision="fp64"), True),
    (dict(H=12801, W=8, K=4, precision="fp64"), False)])
def test_parameter_checks(lib, kw, ok):
    pr = B.make_params(**kw)
    if ok:
        assert B.segsalsa_str_workspace_bytes(pr) > 0
    else:
        with pytest.raises(B.SegsalsaError) as e:
            B.segsalsa_str_workspace_bytes(pr)
        assert e.value.code == B.SEGSALSA_ERR_ARG
        assert B.segsalsa_str_last_error()


def test_workspace_grows_with_state(lib):
    a = B.segsalsa_str_workspace_bytes(B.make_params(256, 256, 8))
    b = B.segsalsa_str_workspace_bytes(B.make_params(256, 256, 8, M=2, sigma=1.0))
    c = B.segsalsa_str_workspace_bytes(B.make_params(256, 256, 8, precision="fp64"))
    n, K = 256 * 256, 8
    # d2 alone is 2 L K n elements
    assert a > 4 * 2 * 9 * K * n and b - a >= 4 * 2 * 16 * K * n and c > 1.9 * a


def test_weights_validation(lib):
    w = np.ones(9)
    assert B.segsalsa_str_workspace_bytes(B.make_params(16, 16, 4, weights=w)) > 0
    w[3] = np.nan
    with pytest.raises(B.SegsalsaError):
        B.segsalsa_str_workspace_bytes(B.make_params(16, 16, 4, weights=w))


def test_tiling_struct_matches_header():
    assert ctypes.sizeof(B.Tiling) == 28
    assert B.Tiling.row_pairs.offset == 4 and B.Tiling.col_rows.offset == 16
    assert B.Tiling.zfuse.offset == 20 and B.Tiling.row_pipe.offset == 24


@pytest.mark.parametrize("tiling,ok", [
    ((0, 0, 0), True), ((4, 1, 1), True), ((32, 16, 8), True), ((3, 0, 0), False),
    ((33, 0, 0), False), ((8, -1, 0), False), ((8, 0, 9), False), ((8, 65, 0), False),
    ((0, 0, 0, 256, 16), True), ((0, 0, 0, 32, 0), False), ((0, 0, 0, 2048, 0), False),
    ((0, 0, 0, 0, 1), False), ((0, 0, 0, 0, 0, 1), True), ((0, 0, 0, 0, 0, 16), True),
    ((0, 0, 0, 0, 0, 3), True), ((0, 0, 0, 0, 0, 5), False), ((0, 0, 0, 0, 0, 32), False), ((0, 0, 0, 0, 0, -1), False),
    ((0, 0, 0, 0, 0, 0, 1), True), ((0, 0, 0, 0, 0, 0, 2), True), ((0, 0, 0, 0, 0, 0, 3), True),
    ((0, 0, 0, 0, 0, 0, 4), False), ((0, 0, 0, 0, 0, 0, -1), False)])
def test_tiling_checks(lib, tiling, ok):
    pr = B.make_params(145, 145, 16)
    t = B.make_tiling(*tiling)
    if ok:
        assert B.segsalsa_str_workspace_bytes_tiled(pr, t) > 0
    else:
        with pytest.raises(B.SegsalsaError) as e:
            B.segsalsa_str_workspace_bytes_tiled(pr, t)
        assert e.value.code == B.SEGSALSA_ERR_ARG


def test_taller_tiles_need_fewer_partials(lib):
    """The rhs tile partials hold every tile plus its halo rows: taller tiles, fewer halo rows,
    a smaller workspace; no tiling equals the defaults."""
    pr = B.make_params(512, 512, 16)
    sizes = [B.segsalsa_str_workspace_bytes_tiled(pr, B.make_tiling(th)) for th in (4, 8, 16, 32)]
    assert sizes == sorted(sizes, reverse=True) and sizes[0] > sizes[-1]
    assert B.segsalsa_str_workspace_bytes_tiled(pr, None) == B.segsalsa_str_workspace_bytes(pr)
