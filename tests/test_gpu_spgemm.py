"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element, on the same seeded inputs.

Bit-exact for boolean, min-plus, int64 and overlap semirings; plus-times FP64
within 1e-12 * sum_k |a_ik b_kj| per entry; identical patterns always.
Tiers are forced through the tuning struct so that every kernel tier
(warp / block / dense, single and multi-slab) runs on small inputs.
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

SR = [api.PLUS_TIMES_F64, api.BOOL_OR_AND, api.MIN_PLUS_F32, api.OVERLAP_I32,
      api.PLUS_TIMES_I64, api.PLUS_TIMES_F32]

# tuning presets that route rows to one tier
TIERS = {
    "default": {},
    "all_warp": dict(sym_warp_max_ub=1 << 20, sym_block_max_ub=1 << 20,
                     num_warp_max_nnz=2048, num_block_max_nnz=2048),
    "all_block": dict(sym_warp_max_ub=1, sym_block_max_ub=1 << 14,
                      num_warp_max_nnz=1, num_block_max_nnz=8192),
    "all_dense": dict(sym_warp_max_ub=1, sym_block_max_ub=1, num_warp_max_nnz=1,
                      num_block_max_nnz=1),
    "dense_small_slabs": dict(sym_warp_max_ub=1, sym_block_max_ub=1, num_warp_max_nnz=1,
                              num_block_max_nnz=1, dense_slab_cols=1024, sym_slab_cols=1024),
    # dense tiers without the symbolic phase's bitmap cache: the rank kernel
    # rebuilds every row's bitmap from its products
    "dense_rebuild": dict(sym_warp_max_ub=1, sym_block_max_ub=1, num_warp_max_nnz=1,
                          num_block_max_nnz=1, bitmap_cache_bytes=1),
    # the rank kernel with 1024-column slabs: many value passes per row, every
    # row on the 1024-thread kernel (no light rows on half-SM CTAs)
    "dense_small_slabs_rank": dict(sym_warp_max_ub=1, sym_block_max_ub=1, num_warp_max_nnz=1,
                                   num_block_max_nnz=1, dense_slab_cols=1024, rank_light_ub=-1),
}


def values_for(sr, M, seed):
    rng = np.random.default_rng(seed)
    if sr == api.BOOL_OR_AND:
        return M.with_values(None)
    if sr == api.OVERLAP_I32:
        return I.positions_csr(M, seed)
    if sr == api.PLUS_TIMES_I64:
        return M.with_values(rng.integers(-2**40, 2**40, M.nnz).astype(np.int64))
    if sr == api.MIN_PLUS_F32:
        return M.with_values((rng.random(M.nnz) * 200 - 100).astype(np.float32))
    if sr == api.PLUS_TIMES_F32:
        return M.with_values((rng.random(M.nnz) * 2 - 1).astype(np.float32))
    return M.with_values(rng.random(M.nnz) * 2 - 1)


def gpu_product(sr, A, B, tuning=None, handle=None):
    h = handle or api.Handle(tuning=tuning)
    dA = api.DeviceCSR.from_host(A, val_dtype=api.IN_NP[sr])
    dB = api.DeviceCSR.from_host(B, val_dtype=api.IN_NP[sr])
    C = api.spgemm(sr, dA, dB, handle=h)
    torch.cuda.synchronize()
    return api.to_host(C, sr), h


def check(sr, A, B, tuning=None, what=""):
    got, h = gpu_product(sr, A, B, tuning)
    exp = oracle.spgemm(sr, A, B)
    assert_pattern_equal(got.rp, got.col, exp.rp, exp.col, what)
    if sr == api.PLUS_TIMES_F64:
        bound = oracle.spgemm(sr, abs_csr(A), abs_csr(B))
        assert_values(sr, got.val, exp.val, bound=bound.val, what=what)
    elif sr == api.PLUS_TIMES_F32:
        a64 = A.with_values(np.abs(A.val).astype(np.float64))
        b64 = B.with_values(np.abs(B.val).astype(np.float64))
        bound = oracle.spgemm(oracle.SR_PT_F64, a64, b64)
        terms = oracle.spgemm(oracle.SR_OVERLAP, I.positions_csr(A, 1), I.positions_csr(B, 2))
        assert_values(sr, got.val, exp.val, bound=bound.val,
                      terms=terms.val["count"].astype(np.float64), what=what)
    else:
        assert_values(sr, got.val, exp.val, what=what)
    return got, h


@pytest.mark.parametrize("tier", list(TIERS))
@pytest.mark.parametrize("sr", SR)
def test_rmat_all_tiers(sr, tier):
    pat = I.rmat(11, seed=3, dtype=None)      # 2048 vertices: hubs, empty rows
    A = values_for(sr, pat, 5)
    B = values_for(sr, pat, 6) if sr != api.OVERLAP_I32 else I.positions_csr(pat, 6)
    check(sr, A, B, TIERS[tier], f"{tier}")


@pytest.mark.parametrize("sr", [api.PLUS_TIMES_F64, api.BOOL_OR_AND])
def test_er4096_full(sr):
    A = I.er(4096, 8, seed=1)
    if sr == api.BOOL_OR_AND:
        A = A.with_values(None)
    got, h = check(sr, A, A)
    st = h.stats()
    assert st["products"] == 4096 * 64


@pytest.mark.parametrize("tier", ["default", "all_block", "dense_small_slabs"])
def test_kmer_overlap_with_gpu_transpose(tier):
    A = I.kmer(3000, 1 << 16, len_lo=20, len_hi=80, col_cap=16, seed=4)
    h = api.Handle(tuning=TIERS[tier])
    dA = api.DeviceCSR.from_host(A, val_dtype=np.int32)
    dAt = h.transpose(dA, 4)
    torch.cuda.synchronize()
    At = oracle.transpose(A, np.int32)
    assert np.array_equal(dAt.rp.cpu().numpy(), At.rp)
    assert np.array_equal(dAt.col.cpu().numpy(), At.col)
    assert np.array_equal(dAt.val.cpu().numpy(), At.val)
    C = api.to_host(api.spgemm(api.OVERLAP_I32, dA, dAt, handle=h), api.OVERLAP_I32)
    O = oracle.spgemm(oracle.SR_OVERLAP, A, At)
    assert_pattern_equal(C.rp, C.col, O.rp, O.col)
    assert_values(oracle.SR_OVERLAP, C.val, O.val)


def test_transpose_long_columns():
    """Columns longer than the shared-memory sort (16384) use the global scratch sort."""
    rng = np.random.default_rng(3)
    n, m = 40000, 64
    dens = np.zeros((n, m), bool)
    dens[:, 0] = True                    # one column of 40000 entries
    dens[:, 1] = rng.random(n) < 0.5     # ~20000
    dens[:, 2:] = rng.random((n, m - 2)) < 0.01
    rows, cols = np.nonzero(dens)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    A = I.CSR(n, m, rp, cols.astype(np.int32), rng.random(rows.size))
    h = api.Handle()
    dAt = h.transpose(api.DeviceCSR.from_host(A, val_dtype=np.float64), 8)
    At = oracle.transpose(A, np.float64)
    assert np.array_equal(dAt.rp.cpu().numpy(), At.rp)
    assert np.array_equal(dAt.col.cpu().numpy(), At.col)
    assert np.array_equal(dAt.val.cpu().numpy(), At.val)


def test_laplacian_closed_form_g64():
    L = I.laplacian(64)
    got, _ = check(api.PLUS_TIMES_F64, L, L)
    assert got.nnz == 64 * 64 + 4 * 64 * 63 + 4 * 64 * 62 + 4 * 63 ** 2


@pytest.mark.parametrize("sr", SR)
def test_edge_cases(sr):
    h = api.Handle()
    # empty A
    Z = I.random_csr(7, 5, 0.0, 1)
    B = values_for(sr, I.random_csr(5, 9, 0.5, 2, dtype=None), 3)
    Zv = values_for(sr, Z.with_values(None), 1) if sr != api.OVERLAP_I32 else I.positions_csr(Z, 1)
    got, _ = gpu_product(sr, Zv, B, handle=h)
    assert got.nnz == 0 and np.all(got.rp == 0)
    # zero rows
    Z0 = I.CSR(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32), None)
    Z0 = values_for(sr, Z0, 1) if sr != api.OVERLAP_I32 else Z0.with_values(np.zeros(0, np.int32))
    got, _ = gpu_product(sr, Z0, B, handle=h)
    assert got.nnz == 0 and got.rp.size == 1
    # rectangular, empty rows and columns, one dense row
    pa = I.random_csr(300, 700, 0.02, 5, dtype=None, empty_row_frac=0.3, empty_col_frac=0.2)
    pb = I.random_csr(700, 5000, 0.01, 6, dtype=None, empty_row_frac=0.3)
    A = values_for(sr, pa, 7)
    Bv = values_for(sr, pb, 8)
    check(sr, A, Bv, None, "rect")
    check(sr, A, Bv, TIERS["dense_small_slabs"], "rect dense")
    check(sr, A, Bv, TIERS["all_block"], "rect block")


def test_argument_errors():
    h = api.Handle()
    A = api.DeviceCSR.from_host(I.random_csr(4, 5, 0.5, 1), val_dtype=np.float64)
    B = api.DeviceCSR.from_host(I.random_csr(6, 5, 0.5, 2), val_dtype=np.float64)
    with pytest.raises(api.SpgemmError) as e:
        api.spgemm(api.PLUS_TIMES_F64, A, B, handle=h)
    assert e.value.status == 1
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    c_rp = torch.empty(5, dtype=torch.int64, device="cuda")
    with pytest.raises(api.SpgemmError) as e:
        h.symbolic(api.PLUS_TIMES_F64, A, A.__class__(5, 4, B.rp[:6], B.col, B.val), c_rp, ws)
    assert e.value.status in (1, 8)


def test_validate_csr():
    h = api.Handle()
    ws = torch.zeros(64, dtype=torch.uint8, device="cuda")
    good = api.DeviceCSR.from_host(I.random_csr(50, 40, 0.2, 1), val_dtype=np.float64)
    h.validate(good, ws)
    bad = I.random_csr(50, 40, 0.2, 1)
    col = bad.col.copy()
    r = int(np.argmax(np.diff(bad.rp) >= 2))
    col[bad.rp[r]], col[bad.rp[r] + 1] = col[bad.rp[r] + 1], col[bad.rp[r]]   # unsorted row
    dbad = api.DeviceCSR.from_host(bad.with_values(bad.val).__class__(50, 40, bad.rp, col, bad.val),
                                   val_dtype=np.float64)
    with pytest.raises(api.SpgemmError) as e:
        h.validate(dbad, ws)
    assert e.value.status == 2


def test_repeated_calls_same_handle_and_workspace():
    """Two calls in a row on one workspace give identical results (counters reset)."""
    pat = I.rmat(10, seed=9, dtype=np.float32)
    h = api.Handle()
    dA = api.DeviceCSR.from_host(pat, val_dtype=np.float32)
    ws = torch.empty(h.workspace_size(api.MIN_PLUS_F32, dA, dA), dtype=torch.uint8, device="cuda")
    r1 = api.to_host(api.spgemm(api.MIN_PLUS_F32, dA, dA, handle=h, ws=ws), api.MIN_PLUS_F32)
    r2 = api.to_host(api.spgemm(api.MIN_PLUS_F32, dA, dA, handle=h, ws=ws), api.MIN_PLUS_F32)
    assert np.array_equal(r1.col, r2.col) and np.array_equal(r1.val, r2.val)


def entry_mode_rows(seed):
    """Rows of 32, 33, 1024, 1025 and 3000 entries (and an empty one) over B rows
    of 24 random columns out of 120,000: the dense tier's row-entry modes (one
    entry per lane, per thread, batched) and, for the long rows, more outputs
    than one value pass holds."""
    rng = np.random.default_rng(seed)
    degs = [32, 33, 1024, 1025, 3000, 0]
    K, N, per_b = 4000, 120_000, 24
    a_rows = np.repeat(np.arange(len(degs)), degs)
    a_cols = np.concatenate([np.sort(rng.choice(K, d, replace=False)) for d in degs if d])
    A = I._from_sorted_coo(len(degs), K, a_rows, a_cols, None)
    b_rows = np.repeat(np.arange(K), per_b)
    b_cols = np.concatenate([np.sort(rng.choice(N, per_b, replace=False)) for _ in range(K)])
    B = I._from_sorted_coo(K, N, b_rows, b_cols, None)
    return A, B


@pytest.mark.parametrize("tier", ["default", "all_dense", "dense_rebuild",
                                  "dense_small_slabs_rank"])
@pytest.mark.parametrize("sr", [api.MIN_PLUS_F32, api.PLUS_TIMES_F64, api.BOOL_OR_AND,
                                api.OVERLAP_I32])
def test_dense_row_entry_modes_and_value_passes(sr, tier):
    A, B = entry_mode_rows(11)
    A = values_for(sr, A, 12)
    B = values_for(sr, B, 13)
    got, h = check(sr, A, B, TIERS[tier], tier)
    # the 3000-entry row has more outputs than one value pass of the rank
    # kernel holds (about 18K at 8 bytes per output)
    assert got.rp[5] - got.rp[4] > 40_000


def light_dense_rows(seed):
    """Rows of 40, 300, 520 and 600 entries over B rows of 8 random columns out
    of 120,000: a few thousand products and outputs each (ub <= 4,800), i.e.
    dense-tier rows light enough for the 512-thread rank kernel, with one
    entry per lane, per thread, and in two batches of entries."""
    rng = np.random.default_rng(seed)
    degs = [40, 300, 520, 600, 0]
    K, N, per_b = 3000, 120_000, 8
    a_rows = np.repeat(np.arange(len(degs)), degs)
    a_cols = np.concatenate([np.sort(rng.choice(K, d, replace=False)) for d in degs if d])
    A = I._from_sorted_coo(len(degs), K, a_rows, a_cols, None)
    b_rows = np.repeat(np.arange(K), per_b)
    b_cols = np.concatenate([np.sort(rng.choice(N, per_b, replace=False)) for _ in range(K)])
    B = I._from_sorted_coo(K, N, b_rows, b_cols, None)
    return A, B


@pytest.mark.parametrize("tier", ["default", "all_dense", "dense_rebuild"])
@pytest.mark.parametrize("sr", [api.MIN_PLUS_F32, api.PLUS_TIMES_F64, api.BOOL_OR_AND,
                                api.OVERLAP_I32])
def test_light_dense_rows(sr, tier):
    A, B = light_dense_rows(17)
    A = values_for(sr, A, 18)
    B = values_for(sr, B, 19)
    got, h = check(sr, A, B, TIERS[tier], tier)
    n = np.diff(got.rp)
    assert n[3] > 4000 and n[2] > 2048   # above the block tier: dense rows


@pytest.mark.parametrize("top", [65535, 65536, 2**31 - 1])
def test_overlap_compact_and_wide_positions(top):
    """The overlap semiring's CTA hash tier packs pairs in 32 bits when every
    position of A and B is below 2^16 and keeps 64-bit pairs otherwise: rows
    of a few thousand outputs, positions drawn up to `top` (one entry of B set
    to `top` exactly), against the oracle."""
    rng = np.random.default_rng(top % 1000)
    # 12,000 reads: every row has 2,000-7,400 outputs (the compact tier below
    # 6,144, the rank tier above)
    A = I.kmer(12000, 1 << 17, len_lo=100, len_hi=300, col_cap=64, seed=4)
    At = oracle.transpose(A, np.int32)
    a_val = rng.integers(0, min(top, 65535) + 1, A.nnz).astype(np.int32)
    b_val = rng.integers(0, top, At.nnz, dtype=np.int64).astype(np.int32)
    b_val[At.nnz // 2] = top
    A = A.with_values(a_val)
    B = I.CSR(At.nrows, At.ncols, At.rp, At.col, b_val)
    got, h = check(api.OVERLAP_I32, A, B, None, f"positions up to {top}")
    n = np.diff(got.rp)
    assert n.max() > 2048   # rows beyond the 24-byte hash tier's limit
