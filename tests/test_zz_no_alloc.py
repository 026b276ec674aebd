"""The allocation-free transpose (spgemm_transpose_noalloc) against the
regular spgemm_transpose, through the C ABI.

Some callers cannot allocate device memory where they need a transpose (an
allocation-free graph-building framework, a custom allocator's callback);
this entry point runs the same kernels with their scratch in a fixed
device array owned by the library.  The test allocates the inputs and
outputs itself, as such a caller would have them, and checks two calls in a
row (the second must not see the first call's leftovers in the shared
scratch) plus the size limit.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2504_06408_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2504_06408_gb300 import spgemm as api  # noqa: E402


def _noalloc_transpose(lib, dA, value_bytes):
    a = dA.c()
    t_rp = torch.empty(dA.ncols + 1, dtype=torch.int64, device="cuda")
    t_col = torch.empty(max(dA.nnz, 1), dtype=torch.int32, device="cuda")
    t_val = torch.empty(max(dA.nnz, 1) * value_bytes, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.spgemm_transpose_noalloc(ctypes.byref(a), value_bytes, t_rp.data_ptr(),
                                      t_col.data_ptr(), t_val.data_ptr(), stream)
    return st, t_rp, t_col, t_val


def _long_column_matrix():
    """20,000 rows x 64 columns with column 0 in every row: a column longer
    than the 16,384 keys one CTA sorts in shared memory, so its sort runs in
    the part of the static scratch array that the other cases leave unused."""
    M = I.random_csr(20000, 64, 0.05, 12)
    rows = np.repeat(np.arange(M.nrows), np.diff(M.rp))
    keep = M.col != 0
    rows = np.concatenate([rows[keep], np.arange(M.nrows)])
    cols = np.concatenate([M.col[keep], np.zeros(M.nrows, np.int32)])
    vals = np.concatenate([M.val[keep], np.arange(M.nrows, dtype=np.float64)])
    order = np.lexsort((cols, rows))
    rp = np.zeros(M.nrows + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=M.nrows), out=rp[1:])
    return I.CSR(M.nrows, M.ncols, rp, cols[order].astype(np.int32), vals[order])


def test_noalloc_transpose_matches_transpose_on_two_calls():
    lib = api.load_library()
    h = api.Handle()
    cases = [
        (I.kmer(3000, 1 << 14, len_lo=10, len_hi=80, col_cap=40, seed=3), np.int32, 4),
        (I.random_csr(900, 5000, 0.01, 8, empty_row_frac=0.2), np.float64, 8),
        (_long_column_matrix(), np.float64, 8),
    ]
    for A, dt, vb in cases:
        dA = api.DeviceCSR.from_host(A, val_dtype=dt)
        if A.nrows == 20000:
            assert int(np.sum(A.col == 0)) > 16384
        ref = h.transpose(dA, vb)
        st, t_rp, t_col, t_val = _noalloc_transpose(lib, dA, vb)
        torch.cuda.synchronize()
        assert st == 0
        assert torch.equal(t_rp, ref.rp)
        assert torch.equal(t_col[:dA.nnz], ref.col)
        assert torch.equal(t_val[:dA.nnz * vb], ref.val.view(torch.uint8).reshape(-1))


def test_noalloc_transpose_of_row_view():
    """A row view whose first entry is far into the arrays (entry numbers are
    kept relative to the view's first entry)."""
    lib = api.load_library()
    h = api.Handle()
    A = I.random_csr(3000, 700, 0.02, 14)
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float64).rows(1000, 2500)
    for _ in range(2):
        ref = h.transpose(dA, 8)
        st, t_rp, t_col, t_val = _noalloc_transpose(lib, dA, 8)
        torch.cuda.synchronize()
        assert st == 0
        assert torch.equal(t_rp, ref.rp)
        assert torch.equal(t_col[:dA.nnz], ref.col)
        assert torch.equal(t_val[:dA.nnz * 8], ref.val.view(torch.uint8).reshape(-1))
    # against the definition: column j of the view lists its rows in order
    sub = A.rp[1000:2501] - A.rp[1000]
    rows = np.repeat(np.arange(1500), np.diff(sub))
    cols = A.col[A.rp[1000]:A.rp[2500]]
    order = np.lexsort((rows, cols))
    assert np.array_equal(t_col[:dA.nnz].cpu().numpy(), rows[order])


def test_noalloc_transpose_rejects_oversize_before_any_work():
    lib = api.load_library()
    # 16M columns need 128 MiB of cursors and lists: beyond the 32 MiB scratch
    rp = torch.zeros(2, dtype=torch.int64, device="cuda")
    big = api.DeviceCSR(1, 1 << 24, rp, torch.zeros(0, dtype=torch.int32, device="cuda"))
    a = big.c()
    st = lib.spgemm_transpose_noalloc(ctypes.byref(a), 0, rp.data_ptr(), None, None, None)
    assert st == 5   # SPG_ERR_UNSUPPORTED
