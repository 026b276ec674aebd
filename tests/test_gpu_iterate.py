"""Iterated products on the GPU (Section 2.2: min-plus W^k = shortest walks of
exactly k edges): W^k by repeated squaring against the oracle's sequential
products, and k-hop distances against dense Bellman-Ford relaxation."""
import numpy as np
import pytest

import oracle
from _util import assert_pattern_equal, assert_values
from paper_2504_06408_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2504_06408_gb300 import spgemm as api  # noqa: E402
from paper_2504_06408_gb300 import iterate  # noqa: E402

from test_gpu_spgemm import values_for  # noqa: E402


@pytest.mark.parametrize("k", [1, 2, 3, 5])
@pytest.mark.parametrize("sr", [api.MIN_PLUS_F32, api.BOOL_OR_AND, api.PLUS_TIMES_I64])
def test_power_matches_oracle(sr, k):
    W = values_for(sr, I.rmat(9, seed=4, dtype=None), 2)
    if sr == api.PLUS_TIMES_I64:   # small values keep the powers readable
        W = W.with_values(np.random.default_rng(1).integers(-3, 4, W.nnz).astype(np.int64))
    dW = api.DeviceCSR.from_host(W, val_dtype=api.IN_NP[sr])
    got = api.to_host(iterate.power(sr, dW, k), sr)
    # the same association as repeated squaring (float min-plus sums are not
    # associative, so the order of the products is part of the result)
    result, base, e = None, W, k
    while True:
        if e & 1:
            result = base if result is None else oracle.spgemm(sr, result, base)
        e >>= 1
        if not e:
            break
        base = oracle.spgemm(sr, base, base)
    exp = result
    assert_pattern_equal(got.rp, got.col, exp.rp, exp.col)
    if sr != api.BOOL_OR_AND:
        assert_values(sr, got.val, exp.val)


def _dense(M, fill):
    D = np.full((M.nrows, M.ncols), fill, dtype=np.float64)
    for i in range(M.nrows):
        a, b = int(M.rp[i]), int(M.rp[i + 1])
        D[i, M.col[a:b]] = M.val[a:b]
    return D


@pytest.mark.parametrize("k", [1, 2, 4])
def test_min_plus_hops_match_bellman_ford(k):
    sr = api.MIN_PLUS_F32
    W = I.rmat(8, seed=6, dtype=np.float32)
    dW = api.DeviceCSR.from_host(W, val_dtype=np.float32)
    got = api.to_host(iterate.hops(sr, dW, k), sr)
    Wd = _dense(W, np.inf)
    D = Wd.copy()
    for _ in range(k - 1):   # relax: walks of one more edge
        D = np.minimum(D, np.min(D[:, :, None] + Wd[None, :, :], axis=1))
    G = _dense(got, np.inf)
    assert np.array_equal(np.isfinite(G), np.isfinite(D))
    fin = np.isfinite(D)
    # float32 sums along different walk orders: exact here (integer-valued weights
    # would be exact; these are U[1,100) floats, so compare within float32 rounding
    # of a k-edge sum)
    assert np.allclose(G[fin], D[fin], rtol=k * 2**-23, atol=0)


def test_boolean_hops_are_reachability():
    sr = api.BOOL_OR_AND
    W = I.rmat(8, seed=7, dtype=None)
    dW = api.DeviceCSR.from_host(W)
    got = api.to_host(iterate.hops(sr, dW, 3), sr)
    R = _dense(W.with_values(np.ones(W.nnz)), 0) > 0
    reach = R.copy()
    step = R.copy()
    for _ in range(2):
        step = (step.astype(np.int64) @ R.astype(np.int64)) > 0
        reach |= step
    G = np.zeros_like(reach)
    for i in range(got.nrows):
        G[i, got.col[got.rp[i]:got.rp[i + 1]]] = True
    assert np.array_equal(G, reach)
