"""The host-memory C ABI call (spgemm_host_symbolic / spgemm_host_numeric,
the call the end-to-end benchmark times) against the oracle: small outputs
in one piece, larger ones through the row-panel pipeline whose downloads
overlap the next panel's kernels (forced here with small panels)."""
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

from test_gpu_spgemm import values_for  # noqa: E402


def host_product(sr, A, B, panel_bytes=0):
    h = api.Handle(tuning={"host_panel_bytes": panel_bytes} if panel_bytes else None)
    rp, col, val, n = h.host_multiply(sr, A, B)
    if val is not None:
        val = val[:n * api.OUT_BYTES[sr]].view(oracle.OUT_DTYPE[sr])
    return rp, col[:n], val


@pytest.mark.parametrize("panel_bytes", [0, 64 << 10, 1 << 20])
@pytest.mark.parametrize("sr", [api.MIN_PLUS_F32, api.PLUS_TIMES_F64, api.BOOL_OR_AND,
                                api.OVERLAP_I32])
def test_host_api_matches_oracle(sr, panel_bytes):
    pat = I.rmat(12, seed=8, dtype=None)
    A = values_for(sr, pat, 3)
    B = values_for(sr, pat, 4) if sr != api.OVERLAP_I32 else I.positions_csr(pat, 4)
    rp, col, val = host_product(sr, A, B, panel_bytes)
    exp = oracle.spgemm(sr, A, B)
    assert_pattern_equal(rp, col, exp.rp, exp.col)
    if sr == api.PLUS_TIMES_F64:
        assert_values(sr, val, exp.val, bound=oracle.spgemm(sr, abs_csr(A), abs_csr(B)).val)
    elif sr != api.BOOL_OR_AND:
        assert_values(sr, val, exp.val)


def test_host_api_same_arrays_and_repeat():
    sr = api.MIN_PLUS_F32
    A = values_for(sr, I.rmat(11, seed=2, dtype=None), 5)
    h = api.Handle(tuning={"host_panel_bytes": 32 << 10})
    exp = oracle.spgemm(sr, A, A)
    for _ in range(2):
        rp, col, val, n = h.host_multiply(sr, A, A)
        assert np.array_equal(rp, exp.rp)
        assert np.array_equal(col[:n], exp.col)
        assert np.array_equal(val[:n * 4].view(np.float32).view(np.uint32),
                              exp.val.view(np.uint32))


def test_host_api_allocation_limit_gives_oom_and_recovers():
    """A handle whose device buffers would exceed spg_tuning.host_alloc_limit
    returns SPG_ERR_OOM (the allocation that would cross the limit is never
    made); with the limit raised the same handle computes the product."""
    sr = api.MIN_PLUS_F32
    A = values_for(sr, I.rmat(11, seed=4, dtype=None), 6)
    exp = oracle.spgemm(sr, A, A)
    h = api.Handle(tuning={"host_alloc_limit": 64 << 10})   # far below A's own copy
    with pytest.raises(api.SpgemmError) as e:
        h.host_multiply(sr, A, A)
    assert e.value.status == 3   # SPG_ERR_OOM
    assert "host_alloc_limit" in str(e.value)
    rp = np.empty(A.nrows + 1, np.int64)
    col = np.empty(exp.nnz, np.int32)
    val = np.empty(exp.nnz * 4, np.uint8)
    h.set_tuning(host_alloc_limit=1 << 40)
    rp2, col2, val2, n = h.host_multiply(sr, A, A, out={"rp": rp, "col": col, "val": val})
    assert np.array_equal(rp2, exp.rp) and np.array_equal(col2[:n], exp.col)
    assert np.array_equal(val2[:n * 4].view(np.uint32), exp.val.view(np.uint32))
