"""Parity at the full sizes of the benchmark configurations, plus properties
that hold at any size.

* R-MAT 18 A^2 (262,144 vertices), min-plus FP32 and boolean: exactly the
  bench product and launch configuration; EVERY row of C is compared with
  the oracle, streamed in row panels (the oracle computes a panel's rows on
  all host cores, the GPU panel is copied to the host, both are compared
  and freed).
* k-mer reads x k-mers (200,000 x 2^24), C = A A^T over the overlap semiring,
  A^T by the GPU transpose; every row against the oracle, streamed.
* 5-point Laplacian on a 2048 x 2048 grid, A^2 plus-times FP64: every entry
  against the closed form.
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


def sample_rows(ub, k_heavy=20, k_rand=300, seed=0, max_products=3e8):
    """The heaviest rows, random non-empty rows, a few empty rows; bounded work."""
    rng = np.random.default_rng(seed)
    order = np.argsort(-ub, kind="stable")
    heavy = order[:k_heavy]
    nz = np.nonzero(ub > 0)[0]
    rand = rng.choice(nz, min(k_rand, nz.size), replace=False)
    empty = np.nonzero(ub == 0)[0][:5]
    rows = np.unique(np.concatenate([heavy, rand, empty]))
    # keep the work bounded: drop the heaviest first while over budget
    while ub[rows].sum() > max_products and rows.size > 10:
        rows = rows[rows != rows[np.argmax(ub[rows])]]
    return rows


def check_rows(sr, A, B, C_dev, rows, row_offset=0):
    got = api.to_host_rows(C_dev, sr, np.asarray(rows) - row_offset)
    exp = oracle.spgemm(sr, A, B, rows=rows)
    assert_pattern_equal(got.rp, got.col, exp.rp, exp.col, f"{len(rows)} sampled rows")
    if sr == api.PLUS_TIMES_F64:
        bound = oracle.spgemm(sr, abs_csr(A), abs_csr(B), rows=rows)
        assert_values(sr, got.val, exp.val, bound=bound.val)
    elif sr != api.BOOL_OR_AND:
        assert_values(sr, got.val, exp.val)


def compare_all_rows_streamed(sr, A, B, C, ub, panel_products=6e8):
    """Every row of C against the oracle, in contiguous row panels of about
    panel_products products each."""
    rp = C.rp.cpu().numpy()
    csum = np.concatenate([[0], np.cumsum(ub)])
    r0, npanels = 0, 0
    while r0 < A.nrows:
        r1 = int(np.searchsorted(csum, csum[r0] + panel_products, side="right")) - 1
        r1 = min(max(r1, r0 + 1), A.nrows)
        exp = oracle.spgemm(sr, A, B, rows=np.arange(r0, r1))
        a, b = int(rp[r0]), int(rp[r1])
        assert_pattern_equal(rp[r0:r1 + 1] - a, C.col[a:b].cpu().numpy(), exp.rp, exp.col,
                             f"rows [{r0}, {r1})")
        if sr != api.BOOL_OR_AND:
            got = C.val[a:b].cpu().numpy()
            if sr == api.OVERLAP_I32:
                got = np.ascontiguousarray(got).view(api.OVERLAP_NP).reshape(-1)
            assert_values(sr, got, exp.val, what=f"rows [{r0}, {r1})")
        del exp
        r0 = r1
        npanels += 1
    return npanels


@pytest.mark.parametrize("sr", [api.MIN_PLUS_F32, api.BOOL_OR_AND])
def test_rmat18_bench_product(sr):
    A = I.rmat(18, dtype=np.float32, seed=1)
    if sr == api.BOOL_OR_AND:
        A = A.with_values(None)
    h = api.Handle()
    dA = api.DeviceCSR.from_host(A, val_dtype=api.IN_NP[sr])
    C = api.spgemm(sr, dA, dA, handle=h)
    st = h.stats()
    assert st["products"] == 9480977744
    assert C.nnz == 2957756203
    ub = oracle.row_upper_bounds(A, A)
    # row sums of the counts equal the scanned row pointers' differences
    rp = C.rp.cpu().numpy()
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and np.all(np.diff(rp) <= ub)
    assert compare_all_rows_streamed(sr, A, A, C, ub) > 1
    if sr == api.MIN_PLUS_F32:   # symmetric weights: C[i,i] = 2 x lightest edge
        rows = sample_rows(ub, k_rand=2000, seed=5)
        rows = rows[ub[rows] > 0]
        got = api.to_host_rows(C, sr, rows)
        for t, i in enumerate(rows):
            seg = got.col[got.rp[t]:got.rp[t + 1]]
            p = np.searchsorted(seg, i)
            assert seg[p] == i
            w = A.val[A.rp[i]:A.rp[i + 1]]
            assert got.val[got.rp[t] + p] == np.float32(2) * w.min()


def test_kmer_full_overlap():
    A = I.kmer(seed=1)                     # 200,000 x 2^24, ~25M nnz
    h = api.Handle()
    dA = api.DeviceCSR.from_host(A, val_dtype=np.int32)
    dAt = h.transpose(dA, 4)
    C = api.spgemm(api.OVERLAP_I32, dA, dAt, handle=h)
    At = oracle.transpose(A, np.int32)
    ub = oracle.row_upper_bounds(A, At)
    assert compare_all_rows_streamed(api.OVERLAP_I32, A, At, C, ub, panel_products=2e8) > 1
    rows = sample_rows(ub, k_heavy=20, k_rand=400)
    # diagonal of every sampled row: {len, (0,0), (1,1)}
    got = api.to_host_rows(C, api.OVERLAP_I32, rows)
    for t, i in enumerate(rows):
        seg = got.col[got.rp[t]:got.rp[t + 1]]
        p = np.searchsorted(seg, i)
        r = got.val[got.rp[t] + p]
        assert (r["count"], r["a0"], r["b0"], r["a1"], r["b1"]) == (A.rp[i + 1] - A.rp[i], 0, 0, 1, 1)


def test_laplacian2048_closed_form():
    g = 2048
    L = I.laplacian(g)
    dL = api.DeviceCSR.from_host(L, val_dtype=np.float64)
    C = api.to_host(api.spgemm(api.PLUS_TIMES_F64, dL, dL), api.PLUS_TIMES_F64)
    assert C.nnz == g * g + 4 * g * (g - 1) + 4 * g * (g - 2) + 4 * (g - 1) ** 2
    n = g * g
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(C.rp))
    x, y = rows % g, rows // g
    cx, cy = C.col.astype(np.int64) % g, C.col.astype(np.int64) // g
    dx, dy = cx - x, cy - y
    nb = (x > 0).astype(int) + (x < g - 1) + (y > 0) + (y < g - 1)
    exp = np.where((dx == 0) & (dy == 0), 16.0 + nb,
          np.where(np.abs(dx) + np.abs(dy) == 1, -8.0,
          np.where((np.abs(dx) == 1) & (np.abs(dy) == 1), 2.0,
          np.where(((np.abs(dx) == 2) & (dy == 0)) | ((dx == 0) & (np.abs(dy) == 2)), 1.0, np.nan))))
    assert np.array_equal(C.val, exp)   # small integers: exact in FP64


def _sample_by_panel(ub, cuts, k_heavy, k_rand, seed):
    """The heaviest rows and random non-empty rows, grouped by panel."""
    rows = sample_rows(ub, k_heavy=k_heavy, k_rand=k_rand, seed=seed, max_products=4e8)
    return {(a, b): rows[(rows >= a) & (rows < b)] for a, b in zip(cuts[:-1], cuts[1:])}


def _check_fp64_rows(A, rows, got_rp, got_col, got_val):
    exp = oracle.spgemm(api.PLUS_TIMES_F64, A, A, rows=rows)
    assert_pattern_equal(got_rp, got_col, exp.rp, exp.col, f"{len(rows)} rows")
    # inputs are non-negative: sum_k |a b| is the value itself
    assert_values(api.PLUS_TIMES_F64, got_val, exp.val, bound=exp.val)


def test_rmat20_summa_panels_sampled_rows():
    """R-MAT 20 A^2 over plus-times FP64 as the 4 x 4 Sparse-SUMMA emulation in
    row panels (C is about 294 GB): sampled rows of every panel, assembled from
    the panel's C blocks, against the oracle."""
    from paper_2504_06408_gb300.summa import summa_panels
    A = I.rmat(20, dtype=np.float64, seed=1, lo=0.0, hi=1.0)
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float64)
    ub = oracle.row_upper_bounds(A, A)
    h = api.Handle()
    checked = []

    def on_panel(r0, r1, sm):
        rows = sample[(r0, r1)]
        if rows.size == 0:
            return
        parts_rp, parts_col, parts_val = [0], [], []
        for r in rows:
            Ib = int(np.searchsorted(sm.row_cuts, r - r0, side="right")) - 1
            i = r - r0 - sm.row_cuts[Ib]
            for Jb in range(sm.q):
                blk = sm.block(Ib, Jb)
                a, b = int(blk.rp[i].item()), int(blk.rp[i + 1].item())
                parts_col.append(blk.col[a:b].cpu().numpy() + sm.col_cuts[Jb])
                parts_val.append(blk.val[a:b].cpu().numpy())
            parts_rp.append(sum(x.size for x in parts_col))
        _check_fp64_rows(A, rows, np.array(parts_rp), np.concatenate(parts_col),
                         np.concatenate(parts_val))
        checked.append(rows.size)

    budget = 24 << 30
    # the panel cuts of summa_panels, known in advance from the row counts
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda")
    ws = torch.empty(h.workspace_size(api.PLUS_TIMES_F64, dA, dA), dtype=torch.uint8, device="cuda")
    h.symbolic(api.PLUS_TIMES_F64, dA, dA, c_rp, ws)
    del ws
    cuts = api.panel_cuts(c_rp.cpu().numpy(), A.nrows, budget // 12)
    sample = _sample_by_panel(ub, cuts, 12, 200, 21)
    npanels = summa_panels(h, api.PLUS_TIMES_F64, dA, dA, budget, on_panel, q=4)
    assert npanels == len(cuts) - 1 >= 8
    assert sum(checked) >= 200


def test_rmat21_learned_panels_sampled_rows():
    """R-MAT 21 A^2 over plus-times FP64 through the learned-sizing path with
    the trained network, in row panels (C is about 757 GB): sampled rows of
    every panel against the oracle."""
    from paper_2504_06408_gb300 import learned as L
    A = I.rmat(21, dtype=np.float64, seed=1, lo=0.0, hi=1.0)
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float64)
    ub = oracle.row_upper_bounds(A, A)
    params, meta = L.load()
    h = api.Handle()
    budget = 24 << 30
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda")
    ws = torch.empty(h.workspace_size(api.PLUS_TIMES_F64, dA, dA), dtype=torch.uint8, device="cuda")
    h.symbolic(api.PLUS_TIMES_F64, dA, dA, c_rp, ws)
    del ws
    cuts = api.panel_cuts(c_rp.cpu().numpy(), A.nrows, budget // 12)
    sample = _sample_by_panel(ub, cuts, 12, 200, 22)
    checked = []

    def on_panel(r0, r1, C):
        rows = sample[(r0, r1)]
        if rows.size == 0:
            return
        got = api.to_host_rows(C, api.PLUS_TIMES_F64, rows - r0)
        _check_fp64_rows(A, rows, got.rp, got.col, got.val)
        checked.append(rows.size)

    total, npanels = api.panel_product(
        api.PLUS_TIMES_F64, dA, dA, budget, on_panel, handle=h,
        learned={"model": params, "margin": meta["margin"], "exact_max_ub": meta["exact_max_ub"]})
    assert npanels == len(cuts) - 1 >= 20
    assert total == int(c_rp[-1].item())
    assert sum(checked) >= 200
