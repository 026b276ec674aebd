"""GPU parity of the Sparse-SUMMA emulation pieces against the CPU oracle:
column split, batched products, merge of stage partials, the whole 4 x 4
block-grid product (batched, unbatched and CUDA-graph replay)."""
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
from paper_2504_06408_gb300.summa import Summa  # noqa: E402

from test_gpu_spgemm import SR, values_for  # noqa: E402


def host(C, sr):
    return api.to_host(C, sr)


def vbytes(sr):
    return 0 if api.IN_NP[sr] is None else np.dtype(api.IN_NP[sr]).itemsize


def test_split_columns_matches_oracle_blocks():
    h = api.Handle()
    M = I.random_csr(300, 1000, 0.03, 4, empty_row_frac=0.2, empty_col_frac=0.1)
    cuts = [0, 7, 400, 401, 1000]
    parts = h.split_columns(api.DeviceCSR.from_host(M, val_dtype=np.float64), cuts, 8)
    ref = oracle.summa_blocks(M, [0, 300], cuts)[0]
    for p, r in zip(parts, ref):
        got = host(p, api.PLUS_TIMES_F64)
        assert_pattern_equal(got.rp, got.col, r.rp, r.col)
        assert np.array_equal(got.val, r.val)


def _partials(sr, S, seed, shape=(60, 40, 70), density=(0.1, 0.1)):
    """S partials of one shape with output-type values (products of random
    factors, so the overlap records are genuine)."""
    out = []
    m, k, n = shape
    for s in range(S):
        pa = I.random_csr(m, k, density[0], seed + 10 * s, dtype=None, empty_row_frac=0.2)
        pb = I.random_csr(k, n, density[1], seed + 10 * s + 1, dtype=None)
        a, b = values_for(sr, pa, seed + s), values_for(sr, pb, seed + s + 5)
        out.append(oracle.spgemm(sr, a, b))
    return out


# (number of partials per merge, shape of the factors, densities): light rows
# (at most 32 entries over all stages), heavy rows (hundreds of entries, the
# bitmap kernel) and a merge wider than 2^18 columns (the sequence-sort path)
MERGE_CASES = {
    "light": [((1, (60, 40, 70), (0.1, 0.1))), ((3, (60, 40, 70), (0.1, 0.1))),
              ((5, (60, 40, 70), (0.1, 0.1)))],
    "heavy": [((4, (50, 30, 3000), (0.3, 0.05))), ((16, (20, 30, 500), (0.2, 0.1))),
              ((2, (40, 60, 5000), (0.2, 0.02)))],
    "wide": [((3, (30, 20, 300_000), (0.3, 0.0004))), ((2, (30, 20, 300_000), (0.3, 0.0004)))],
}


@pytest.mark.parametrize("case", list(MERGE_CASES))
@pytest.mark.parametrize("sr", SR)
def test_merge_stages_matches_oracle(sr, case):
    h = api.Handle()
    groups_host = [_partials(sr, S, 10 * S + k, shape, dens)
                   for k, (S, shape, dens) in enumerate(MERGE_CASES[case])]
    dt = oracle.OUT_DTYPE[sr]
    dev_groups = []
    for g in groups_host:
        dg = []
        for P in g:
            val = None
            if P.val is not None:
                raw = np.ascontiguousarray(P.val).view(np.uint8)
                val = torch.from_numpy(raw.copy()).cuda()
            dg.append(api.DeviceCSR(P.nrows, P.ncols, torch.from_numpy(P.rp).cuda(),
                                    torch.from_numpy(P.col).cuda(), val))
        dev_groups.append(dg)
    ws = torch.empty(h.merge_workspace_size(sr, dev_groups), dtype=torch.uint8, device="cuda")
    c_rp = [torch.empty(g[0].nrows + 1, dtype=torch.int64, device="cuda") for g in dev_groups]
    nnz = h.merge_count(sr, dev_groups, c_rp, ws)
    ob = api.OUT_BYTES[sr]
    c_col = [torch.empty(max(n, 1), dtype=torch.int32, device="cuda") for n in nnz]
    c_val = [torch.empty(max(n, 1) * ob, dtype=torch.uint8, device="cuda") for n in nnz] if ob else None
    h.merge_write(sr, dev_groups, c_rp, c_col, c_val, ws)
    h.check(ws)
    for k, g in enumerate(groups_host):
        exp = oracle.merge(sr, g)
        assert nnz[k] == exp.nnz
        assert np.array_equal(c_rp[k].cpu().numpy(), exp.rp)
        assert np.array_equal(c_col[k][:nnz[k]].cpu().numpy(), exp.col)
        if ob:
            got = c_val[k][:nnz[k] * ob].cpu().numpy().view(dt)
            # the GPU folds in stage order like the oracle: bit-identical, floats included
            assert np.array_equal(got.view(np.uint8), np.ascontiguousarray(exp.val).view(np.uint8))


@pytest.mark.parametrize("sr", [api.PLUS_TIMES_F64, api.BOOL_OR_AND, api.MIN_PLUS_F32,
                                api.OVERLAP_I32])
def test_batched_equals_single_calls(sr):
    pat = I.rmat(11, seed=4, dtype=None)
    A = values_for(sr, pat, 1)
    B = values_for(sr, pat, 2) if sr != api.OVERLAP_I32 else I.positions_csr(pat, 2)
    h = api.Handle()
    dA = api.DeviceCSR.from_host(A, val_dtype=api.IN_NP[sr])
    dB = api.DeviceCSR.from_host(B, val_dtype=api.IN_NP[sr])
    spans = [(0, 2048), (0, 700), (700, 2048), (100, 101)]
    As = [dA if (r0, r1) == (0, 2048) else dA.rows(r0, r1) for r0, r1 in spans]
    Bs = [dB, dB, dB, dB]
    ws = torch.empty(h.workspace_size_batched(sr, As, Bs), dtype=torch.uint8, device="cuda")
    rps = [torch.empty(a.nrows + 1, dtype=torch.int64, device="cuda") for a in As]
    nnz = h.symbolic_batched(sr, As, Bs, rps, ws)
    cols = [torch.empty(max(n, 1), dtype=torch.int32, device="cuda") for n in nnz]
    vals = [api.out_tensor(sr, max(n, 1)) for n in nnz]
    h.numeric_batched(sr, As, Bs, rps, cols, vals if sr != api.BOOL_OR_AND else None, ws)
    h.check(ws)
    for (r0, r1), a, n, rp, c, v in zip(spans, As, nnz, rps, cols, vals):
        one = host(api.spgemm(sr, a, dB, handle=h), sr)
        assert n == one.nnz
        assert np.array_equal(rp.cpu().numpy(), one.rp)
        assert np.array_equal(c[:n].cpu().numpy(), one.col)
        if sr != api.BOOL_OR_AND:
            got = host(api.DeviceCSR(a.nrows, dB.ncols, rp, c[:n], v[:n]), sr).val
            if sr == api.PLUS_TIMES_F64:
                # atomic accumulation order differs between the calls: both within
                # the parity bound of the oracle
                rows = np.arange(r0, r1)
                exp = oracle.spgemm(sr, A, B, rows=rows)
                bound = oracle.spgemm(sr, abs_csr(A), abs_csr(B), rows=rows)
                assert_values(sr, got, exp.val, bound=bound.val)
                assert_values(sr, one.val, exp.val, bound=bound.val)
            else:
                assert np.array_equal(np.ascontiguousarray(got).view(np.uint8),
                                      np.ascontiguousarray(one.val).view(np.uint8))


def _check_blocks(sm, sr, A, B):
    C = oracle.spgemm(sr, A, B)
    Cb = oracle.summa_blocks(C, sm.row_cuts, sm.col_cuts)
    bound = None
    if sr == api.PLUS_TIMES_F64:
        bound = oracle.summa_blocks(oracle.spgemm(sr, abs_csr(A), abs_csr(B)), sm.row_cuts,
                                    sm.col_cuts)
    for Ib in range(sm.q):
        for Jb in range(sm.q):
            got = host(sm.block(Ib, Jb), sr)
            exp = Cb[Ib][Jb]
            assert_pattern_equal(got.rp, got.col, exp.rp, exp.col, f"block {Ib},{Jb}")
            if sr == api.PLUS_TIMES_F64:
                assert_values(sr, got.val, exp.val, bound=bound[Ib][Jb].val)
            elif sr == api.PLUS_TIMES_F32:
                assert np.allclose(got.val, exp.val, rtol=1e-5, atol=1e-5)
            elif sr != api.BOOL_OR_AND:
                assert_values(sr, got.val, exp.val)


@pytest.mark.parametrize("sr", SR)
@pytest.mark.parametrize("batched", [True, False])
def test_summa_4x4_matches_oracle(sr, batched):
    pat = I.rmat(11, seed=6, dtype=None)
    A = values_for(sr, pat, 3)
    B = values_for(sr, pat, 4) if sr != api.OVERLAP_I32 else I.positions_csr(pat, 4)
    h = api.Handle()
    dA = api.DeviceCSR.from_host(A, val_dtype=api.IN_NP[sr])
    dB = api.DeviceCSR.from_host(B, val_dtype=api.IN_NP[sr])
    cuts = [0, 64, 300, 1100, 2048]          # uneven blocks, hubs in the first
    sm = Summa(h, sr, dA, dB, q=4, row_cuts=cuts, inner_cuts=[0, 200, 900, 1500, 2048],
               col_cuts=cuts, batched=batched)
    sm.plan()
    sm.run()
    sm.check()
    torch.cuda.synchronize()
    _check_blocks(sm, sr, A, B)


@pytest.mark.parametrize("batched", [True, False])
def test_summa_dense_tier_blocks(batched):
    """Every block row in the dense tiers (symbolic bitmap cache kept): in the
    plain form each block product needs its own workspace."""
    from test_gpu_spgemm import TIERS
    sr = api.MIN_PLUS_F32
    pat = I.rmat(12, seed=2, dtype=None)
    A = values_for(sr, pat, 7)
    h = api.Handle(tuning=TIERS["all_dense"])
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float32)
    sm = Summa(h, sr, dA, dA, q=4, batched=batched, tuning=TIERS["all_dense"])
    sm.plan()
    sm.run()
    sm.check()
    torch.cuda.synchronize()
    _check_blocks(sm, sr, A, A)


@pytest.mark.parametrize("sr", [api.PLUS_TIMES_F64, api.MIN_PLUS_F32, api.OVERLAP_I32])
def test_summa_2_5d_half_stages(sr):
    """2.5D split: every stage in halves, 8 partials per C block merged."""
    pat = I.rmat(11, seed=9, dtype=None)
    A = values_for(sr, pat, 1)
    B = values_for(sr, pat, 2) if sr != api.OVERLAP_I32 else I.positions_csr(pat, 2)
    h = api.Handle()
    dA = api.DeviceCSR.from_host(A, val_dtype=api.IN_NP[sr])
    dB = api.DeviceCSR.from_host(B, val_dtype=api.IN_NP[sr])
    sm = Summa(h, sr, dA, dB, q=4, stages=8)
    assert sm.stages == 8 and len(sm.blocks) == 128
    sm.plan()
    sm.capture()
    sm.run()
    sm.check()
    torch.cuda.synchronize()
    _check_blocks(sm, sr, A, B)


def test_summa_graph_replay_matches():
    sr = api.MIN_PLUS_F32
    pat = I.rmat(12, seed=8, dtype=None)
    A = values_for(sr, pat, 5)
    h = api.Handle()
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float32)
    sm = Summa(h, sr, dA, dA, q=4)
    sm.plan()
    sm.capture()
    for _ in range(2):
        for k in range(len(sm.c_col)):
            sm.c_col[k].fill_(-1)
        sm.run()
        torch.cuda.synchronize()
        _check_blocks(sm, sr, A, A)


@pytest.mark.parametrize("sr", [api.MIN_PLUS_F32, api.PLUS_TIMES_F64, api.OVERLAP_I32])
def test_summa_full_graph_replay_matches(sr):
    """One CUDA graph over the whole batched product (row analysis, symbolic
    phase, scan, numeric phase, merge count and merge write; no host
    synchronisation inside): every replay recomputes the row pointers, the
    partials and C from scratch and matches the oracle."""
    pat = I.rmat(12, seed=13, dtype=None)
    A = values_for(sr, pat, 5)
    B = values_for(sr, pat, 6) if sr != api.OVERLAP_I32 else I.positions_csr(pat, 6)
    h = api.Handle()
    dA = api.DeviceCSR.from_host(A, val_dtype=api.IN_NP[sr])
    dB = api.DeviceCSR.from_host(B, val_dtype=api.IN_NP[sr])
    sm = Summa(h, sr, dA, dB, q=4)
    sm.plan()
    sm.capture(full=True)
    for _ in range(2):
        for rp in sm.p_rp + sm.c_rp:
            rp.fill_(-1)
        for k in range(len(sm.c_col)):
            sm.c_col[k].fill_(-1)
        sm._pcol.fill_(-1)
        sm.run()
        sm.check()
        torch.cuda.synchronize()
        _check_blocks(sm, sr, A, B)
