"""Row-panel products (spgemm.panel_product, the route for products whose C
exceeds device memory) against the oracle, every semiring.

A's rows are shuffled and its heaviest row placed a quarter of the way down,
and the panel budget is the output of rows [0, hub] exactly, so the first
panel boundary falls right after the hub row and the product runs in at
least three panels.  Each panel's rows are compared with the oracle's rows,
element by element.
"""
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


def hub_shuffled_rmat(scale, seed):
    pat = I.rmat(scale, seed=seed, dtype=None)
    ub = oracle.row_upper_bounds(pat, pat)
    rng = np.random.default_rng(seed)
    order = rng.permutation(pat.nrows)
    hub = int(np.argmax(ub))
    at = pat.nrows // 4
    pos = int(np.nonzero(order == hub)[0][0])
    order[pos], order[at] = order[at], order[pos]
    deg = np.diff(pat.rp)[order]
    rp = np.zeros(pat.nrows + 1, np.int64)
    np.cumsum(deg, out=rp[1:])
    col = np.concatenate([pat.col[pat.rp[r]:pat.rp[r + 1]] for r in order])
    return I.CSR(pat.nrows, pat.ncols, rp, col.astype(np.int32), None), pat, at


@pytest.mark.parametrize("sr", SR)
def test_panel_product_matches_oracle(sr):
    A, B, at = hub_shuffled_rmat(12, 41)
    A = values_for(sr, A, 1)
    B = values_for(sr, B, 2)
    exp = oracle.spgemm(sr, A, B)
    per = 4 + api.OUT_BYTES[sr]
    budget = int(exp.rp[at + 1]) * per
    dA = api.DeviceCSR.from_host(A, val_dtype=api.IN_NP[sr])
    dB = api.DeviceCSR.from_host(B, val_dtype=api.IN_NP[sr])
    seen = []
    bound = oracle.spgemm(sr, abs_csr(A), abs_csr(B)) if sr == api.PLUS_TIMES_F64 else None
    terms = None
    if sr == api.PLUS_TIMES_F32:
        ones_a = A.with_values(np.ones(A.nnz, np.float64))
        ones_b = B.with_values(np.ones(B.nnz, np.float64))
        terms = oracle.spgemm(api.PLUS_TIMES_F64, ones_a, ones_b).val
        bound = oracle.spgemm(api.PLUS_TIMES_F64, abs_csr(A.with_values(A.val.astype(np.float64))),
                              abs_csr(B.with_values(B.val.astype(np.float64))))

    def on_panel(r0, r1, C):
        got = api.to_host(C, sr)
        a, b = int(exp.rp[r0]), int(exp.rp[r1])
        assert_pattern_equal(got.rp, got.col, exp.rp[r0:r1 + 1] - a, exp.col[a:b],
                             f"panel [{r0}, {r1})")
        if sr == api.PLUS_TIMES_F64:
            assert_values(sr, got.val, exp.val[a:b], bound=bound.val[a:b])
        elif sr == api.PLUS_TIMES_F32:
            assert_values(sr, got.val, exp.val[a:b], bound=bound.val[a:b], terms=terms[a:b])
        elif sr != api.BOOL_OR_AND:
            assert_values(sr, got.val, exp.val[a:b])
        seen.append((r0, r1))

    total, npanels = api.panel_product(sr, dA, dB, budget, on_panel)
    assert total == exp.nnz
    assert npanels >= 3 and len(seen) == npanels
    # the first boundary falls right after the hub row (or after the empty
    # rows that follow it)
    assert seen[0][0] == 0 and seen[0][1] > at and exp.rp[seen[0][1]] == exp.rp[at + 1]
    assert [s[0] for s in seen[1:]] == [s[1] for s in seen[:-1]] and seen[-1][1] == A.nrows
