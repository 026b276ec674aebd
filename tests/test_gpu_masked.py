"""Masked product on the GPU against the oracle's definition (the full
product restricted to the mask), every semiring, plus triangle counting."""
import numpy as np
import pytest

import oracle
from _util import abs_csr, assert_pattern_equal, assert_values
from paper_2504_06408_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2504_06408_gb300 import spgemm as api  # noqa: E402

from test_gpu_spgemm import SR, values_for  # noqa: E402
from test_oracle_pins import _lower  # noqa: E402


def dev(sr, M):
    return api.DeviceCSR.from_host(M, val_dtype=api.IN_NP[sr])


@pytest.mark.parametrize("mask", ["random", "own_pattern", "empty"])
@pytest.mark.parametrize("sr", SR)
def test_masked_matches_oracle(sr, mask):
    pat = I.rmat(10, seed=2, dtype=None)
    A = values_for(sr, pat, 3)
    B = values_for(sr, pat, 4) if sr != api.OVERLAP_I32 else I.positions_csr(pat, 4)
    if mask == "random":
        M = I.random_csr(pat.nrows, pat.ncols, 0.08, 9, dtype=None, empty_row_frac=0.2)
    elif mask == "own_pattern":
        C = oracle.spgemm(oracle.SR_BOOL, pat, pat)
        M = I.CSR(C.nrows, C.ncols, C.rp, C.col, None)
    else:
        M = I.random_csr(pat.nrows, pat.ncols, 0.0, 1, dtype=None)
    got = api.to_host(api.masked_spgemm(sr, dev(sr, A), dev(sr, B), api.DeviceCSR.from_host(M)), sr)
    exp = oracle.masked(sr, A, B, M)
    assert_pattern_equal(got.rp, got.col, exp.rp, exp.col)
    if sr == api.PLUS_TIMES_F64:
        bound = oracle.masked(sr, abs_csr(A), abs_csr(B), M)
        assert_values(sr, got.val, exp.val, bound=bound.val)
    elif sr == api.PLUS_TIMES_F32:
        assert np.allclose(got.val, exp.val, rtol=1e-5, atol=1e-5)
    elif sr != api.BOOL_OR_AND:
        assert_values(sr, got.val, exp.val)


def test_masked_triangle_count():
    A = I.rmat(12, seed=4, dtype=None)
    L = _lower(A)
    dL = api.DeviceCSR.from_host(L, val_dtype=np.int64)
    C = api.masked_spgemm(api.PLUS_TIMES_I64, dL, dL, dL)
    got = int(C.val.sum().item())
    exp = oracle.masked(oracle.SR_PT_I64, L, L, L)
    assert got == int(exp.val.sum()) > 0
