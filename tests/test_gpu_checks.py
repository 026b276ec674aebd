"""The checked build (-DSPG_CHECKS, libspgemm_checks.so) through the C ABI.

The checked build validates every input matrix on the device before it queues
a product kernel, checks C's row pointers in a numeric call against the count
of the symbolic call that left the workspace, and range-checks each rank of
the rank-indexed accumulation.  These tests feed it malformed inputs and read
the SPG_ERR_* status back: the malformed matrices are refused by the
validation kernel (which reads only within the arrays' bounds) before any
product kernel runs, so no kernel ever indexes memory with their values.
Valid products must match the oracle exactly as the regular build does.
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

from test_gpu_spgemm import TIERS, values_for  # noqa: E402

INVALID_CSR, OVERFLOW = 2, 6


def checked_handle(**tuning):
    return api.Handle(tuning=tuning or None, lib_path=api.CHECKS_LIB_PATH)


@pytest.mark.parametrize("tier", ["default", "all_dense", "dense_rebuild", "all_block"])
@pytest.mark.parametrize("sr", [api.MIN_PLUS_F32, api.PLUS_TIMES_F64, api.BOOL_OR_AND,
                                api.OVERLAP_I32])
def test_checked_build_matches_oracle(sr, tier):
    pat = I.rmat(11, seed=21, dtype=None)
    A = values_for(sr, pat, 1)
    B = values_for(sr, pat, 2)
    h = checked_handle(**TIERS[tier])
    dA = api.DeviceCSR.from_host(A, val_dtype=api.IN_NP[sr])
    dB = api.DeviceCSR.from_host(B, val_dtype=api.IN_NP[sr])
    got = api.to_host(api.spgemm(sr, dA, dB, handle=h), sr)
    exp = oracle.spgemm(sr, A, B)
    assert_pattern_equal(got.rp, got.col, exp.rp, exp.col, tier)
    if sr == api.PLUS_TIMES_F64:
        assert_values(sr, got.val, exp.val,
                      bound=oracle.spgemm(sr, abs_csr(A), abs_csr(B)).val)
    elif sr != api.BOOL_OR_AND:
        assert_values(sr, got.val, exp.val)


def _malformed(kind):
    """(A, B) host CSRs of a product whose A is malformed in one way."""
    B = I.random_csr(60, 50, 0.2, 3, dtype=np.float32)
    A = I.random_csr(40, 60, 0.2, 4, dtype=np.float32)
    rp, col = A.rp.copy(), A.col.copy()
    r = int(np.argmax(np.diff(rp) >= 2))
    if kind == "column_out_of_range":
        col[rp[r]] = 60 + 1000                 # beyond B's rows
    elif kind == "negative_column":
        col[rp[r] + 1] = -7
    elif kind == "unsorted_row":
        col[rp[r]], col[rp[r] + 1] = col[rp[r] + 1], col[rp[r]]
    elif kind == "row_ptr_beyond_nnz":
        rp[r + 1:] += 1 << 40                   # rows reach far past the column array
        rp[-1] = A.nnz
    elif kind == "row_ptr_decreasing":
        rp[r + 1] = rp[r] - 1 if rp[r] > 0 else 0
        rp[r] = rp[r + 1] + 1
    return I.CSR(A.nrows, A.ncols, rp, col, A.val), B


@pytest.mark.parametrize("kind", ["column_out_of_range", "negative_column", "unsorted_row",
                                  "row_ptr_beyond_nnz", "row_ptr_decreasing"])
def test_malformed_input_refused_before_any_product_kernel(kind):
    sr = api.MIN_PLUS_F32
    A, B = _malformed(kind)
    h = checked_handle()
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float32)
    dB = api.DeviceCSR.from_host(B, val_dtype=np.float32)
    ws = torch.empty(h.workspace_size(sr, dA, dB), dtype=torch.uint8, device="cuda")
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(api.SpgemmError) as e:
        h.symbolic(sr, dA, dB, c_rp, ws)
    assert e.value.status == INVALID_CSR
    # the malformed matrix as the right operand: X (30 x 40) times A
    X = I.random_csr(30, A.nrows, 0.3, 6, dtype=np.float32)
    dX = api.DeviceCSR.from_host(X, val_dtype=np.float32)
    ws2 = torch.empty(h.workspace_size(sr, dX, dA), dtype=torch.uint8, device="cuda")
    x_rp = torch.empty(X.nrows + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(api.SpgemmError) as e:
        h.symbolic(sr, dX, dA, x_rp, ws2)
    assert e.value.status == INVALID_CSR
    torch.cuda.synchronize()
    # the handle and the device stay usable
    good = api.DeviceCSR.from_host(B, val_dtype=np.float32)
    C = api.to_host(api.spgemm(sr, good, api.DeviceCSR.from_host(
        I.random_csr(50, 30, 0.3, 5, dtype=np.float32), val_dtype=np.float32), handle=h), sr)
    assert C.rp[-1] == C.nnz


def test_numeric_row_pointers_checked_against_symbolic_count():
    sr = api.MIN_PLUS_F32
    pat = I.rmat(10, seed=23, dtype=None)
    A = values_for(sr, pat, 1)
    h = checked_handle()
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float32)
    ws = torch.empty(h.workspace_size(sr, dA, dA), dtype=torch.uint8, device="cuda")
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda")
    nnz = h.symbolic(sr, dA, dA, c_rp, ws)
    c_col = torch.empty(nnz, dtype=torch.int32, device="cuda")
    c_val = torch.empty(nnz, dtype=torch.float32, device="cuda")
    # (a) row pointers of a smaller product: refused before any numeric kernel
    short = c_rp.clone()
    short[-1] -= 1
    with pytest.raises(api.SpgemmError) as e:
        h.numeric(sr, dA, dA, short, c_col, c_val, ws)
    assert e.value.status == INVALID_CSR
    # (b) decreasing row pointers
    dec = c_rp.clone()
    r = int(torch.argmax((c_rp[1:] - c_rp[:-1] > 2).to(torch.int32)).item())
    dec[r + 1] = dec[r] - 1
    with pytest.raises(api.SpgemmError) as e:
        h.numeric(sr, dA, dA, dec, c_col, c_val, ws)
    assert e.value.status == INVALID_CSR
    # (c) same total, one entry moved from a row to the next: both rows stay
    # inside C, the kernels find counts that disagree and write neither row
    moved = c_rp.clone()
    moved[r + 1] -= 1
    h.numeric(sr, dA, dA, moved, c_col, c_val, ws)
    with pytest.raises(api.SpgemmError) as e:
        h.check(ws)
    assert e.value.status == OVERFLOW
    # (d) the true row pointers still give the oracle's C on the same workspace
    nnz = h.symbolic(sr, dA, dA, c_rp, ws)
    h.numeric(sr, dA, dA, c_rp, c_col, c_val, ws)
    h.check(ws)
    exp = oracle.spgemm(sr, A, A)
    assert np.array_equal(c_rp.cpu().numpy(), exp.rp)
    assert np.array_equal(c_col.cpu().numpy(), exp.col)
    assert np.array_equal(c_val.cpu().numpy().view(np.uint32), exp.val.view(np.uint32))


def test_checked_masked_and_learned_paths():
    sr = api.MIN_PLUS_F32
    pat = I.rmat(10, seed=24, dtype=None)
    A = values_for(sr, pat, 1)
    h = checked_handle()
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float32)
    exp = oracle.spgemm(sr, A, A)
    # learned path with the trained network and a capacity of one entry for
    # every row it sizes: those rows overflow into the exact path, C is unchanged
    from paper_2504_06408_gb300 import learned as L
    params, _ = L.load()
    got = api.to_host(api.learned_spgemm(sr, dA, dA, model=params, margin=1e-6, handle=h,
                                         exact_max_ub=1), sr)
    assert h.stats()["overflow_rows"] > 0
    assert np.array_equal(got.rp, exp.rp) and np.array_equal(got.col, exp.col)
    assert np.array_equal(got.val.view(np.uint32), exp.val.view(np.uint32))
    # masked product with a malformed mask is refused
    M = I.random_csr(A.nrows, A.ncols, 0.01, 6, dtype=None)
    col = M.col.copy()
    col[0] = A.ncols + 5
    dM = api.DeviceCSR.from_host(I.CSR(M.nrows, M.ncols, M.rp, col, None))
    with pytest.raises(api.SpgemmError) as e:
        api.masked_spgemm(sr, dA, dA, dM, handle=h)
    assert e.value.status == INVALID_CSR
