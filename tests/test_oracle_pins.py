"""Pins for the CPU oracle: each test checks it against something other than itself.

* dense brute force on tiny inputs, every semiring, bit-identical;
* boolean A^2 = 2-hop reachability (set-based graph walk);
* min-plus A^2 = one Bellman-Ford relaxation from the 1-hop distances, and the
  diagonal of a symmetric graph = twice the lightest incident edge;
* plus-times = dense GEMM (BLAS) within 1e-12, and the closed form of the
  squared 5-point Laplacian (exact in FP64);
* identity and permutation invariants;
* k-mer overlap: counts = set intersections, two smallest pairs by brute force,
  C[j,i] = C[i,j] with pairs swapped, and the diagonal;
* transpose identity AB = (B^T A^T)^T for commutative semirings (Section 3.1);
* merge: the block-grid (Sparse SUMMA, Section 2.1) products merged over
  stages equal the unblocked product;
* hand-worked golden examples under tests/golden/.
"""
import json
import os

import numpy as np
import pytest

import oracle
from _util import abs_csr, assert_pattern_equal, assert_values
from paper_2504_06408_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALL_SR = [oracle.SR_PT_F64, oracle.SR_BOOL, oracle.SR_MP_F32, oracle.SR_OVERLAP,
          oracle.SR_PT_I64, oracle.SR_PT_F32]


def _vals_for(sr, M, seed):
    """Values of semiring sr's input type on M's pattern."""
    rng = np.random.default_rng(seed)
    if sr == oracle.SR_BOOL:
        return M.with_values(None)
    if sr == oracle.SR_OVERLAP:
        return I.positions_csr(M, seed)
    if sr == oracle.SR_PT_I64:
        return M.with_values(rng.integers(-2**40, 2**40, M.nnz).astype(np.int64))
    if sr == oracle.SR_MP_F32:
        return M.with_values((rng.random(M.nnz) * 200 - 100).astype(np.float32))
    if sr == oracle.SR_PT_F32:
        return M.with_values((rng.random(M.nnz) * 2 - 1).astype(np.float32))
    return M.with_values(rng.random(M.nnz) * 2 - 1)


# ---- independent dense brute force -------------------------------------------------

def _dense_ops(sr):
    NP = (2**31 - 1, 2**31 - 1)
    if sr == oracle.SR_PT_F64:
        return (lambda a, b: float(a) * float(b)), (lambda x, y: x + y)
    if sr == oracle.SR_PT_F32:
        return (lambda a, b: np.float32(a) * np.float32(b)), (lambda x, y: np.float32(x + y))
    if sr == oracle.SR_MP_F32:
        def mn(x, y):
            if y < x:
                return y
            if x < y:
                return x
            return y if (np.signbit(y) and not np.signbit(x)) else x
        return (lambda a, b: np.float32(np.float32(a) + np.float32(b))), mn
    if sr == oracle.SR_PT_I64:
        M = 2**64
        def wrap(v):
            v %= M
            return v - M if v >= 2**63 else v
        return (lambda a, b: wrap(int(a) * int(b))), (lambda x, y: wrap(x + y))
    if sr == oracle.SR_BOOL:
        return (lambda a, b: True), (lambda x, y: True)
    if sr == oracle.SR_OVERLAP:
        def mul(a, b):
            return (1, [(int(a), int(b))])
        def add(x, y):
            pairs = sorted(x[1] + y[1])[:2]
            return (x[0] + y[0], pairs)
        return mul, add
    raise ValueError(sr)


def dense_bruteforce(sr, A, B):
    """Dense triple loop with a touched mask; k ascending per (i, j)."""
    mul, add = _dense_ops(sr)
    Ad = {}
    for i in range(A.nrows):
        for p in range(A.rp[i], A.rp[i + 1]):
            Ad[(i, int(A.col[p]))] = None if A.val is None else A.val[p]
    Bd = {}
    for k in range(B.nrows):
        for p in range(B.rp[k], B.rp[k + 1]):
            Bd[(k, int(B.col[p]))] = None if B.val is None else B.val[p]
    out = {}
    for i in range(A.nrows):
        for j in range(B.ncols):
            acc = None
            for k in range(A.ncols):
                if (i, k) in Ad and (k, j) in Bd:
                    pr = mul(Ad[(i, k)], Bd[(k, j)])
                    acc = pr if acc is None else add(acc, pr)
            if acc is not None:
                out[(i, j)] = acc
    return out


def _as_dict(sr, C):
    d = {}
    for i in range(C.nrows):
        for p in range(C.rp[i], C.rp[i + 1]):
            j = int(C.col[p])
            if sr == oracle.SR_BOOL:
                v = True
            elif sr == oracle.SR_OVERLAP:
                r = C.val[p]
                pairs = [(int(r["a0"]), int(r["b0"]))]
                if (int(r["a1"]), int(r["b1"])) != (2**31 - 1, 2**31 - 1):
                    pairs.append((int(r["a1"]), int(r["b1"])))
                v = (int(r["count"]), pairs)
            else:
                v = C.val[p]
            d[(i, j)] = v
    return d


def _same_scalar(sr, x, y):
    if sr in (oracle.SR_PT_F64,):
        return np.float64(x).tobytes() == np.float64(y).tobytes()
    if sr in (oracle.SR_MP_F32, oracle.SR_PT_F32):
        return np.float32(x).tobytes() == np.float32(y).tobytes()
    if sr == oracle.SR_PT_I64:
        return int(x) == int(y)
    return x == y


@pytest.mark.parametrize("sr", ALL_SR)
@pytest.mark.parametrize("case", [
    dict(m=7, k=9, n=6, dens=0.3, seed=1),
    dict(m=16, k=16, n=16, dens=0.5, seed=2),
    dict(m=20, k=12, n=24, dens=0.15, seed=3, erow=0.3, ecol=0.3),
    dict(m=5, k=5, n=5, dens=0.0, seed=4),
    dict(m=1, k=30, n=1, dens=0.9, seed=5),
])
def test_oracle_matches_dense_bruteforce(sr, case):
    pa = I.random_csr(case["m"], case["k"], case["dens"], case["seed"], dtype=None,
                      empty_row_frac=case.get("erow", 0), empty_col_frac=case.get("ecol", 0))
    pb = I.random_csr(case["k"], case["n"], case["dens"], case["seed"] + 100, dtype=None,
                      empty_row_frac=case.get("erow", 0), empty_col_frac=case.get("ecol", 0))
    A = _vals_for(sr, pa, case["seed"] + 7)
    B = _vals_for(sr, pb, case["seed"] + 8)
    C = oracle.spgemm(sr, A, B)
    # rows strictly ascending, structural pattern
    for i in range(C.nrows):
        seg = C.col[C.rp[i]:C.rp[i + 1]]
        assert np.all(np.diff(seg) > 0)
    got = _as_dict(sr, C)
    exp = dense_bruteforce(sr, A, B)
    assert set(got) == set(exp)
    for key, v in exp.items():
        assert _same_scalar(sr, got[key], v), (key, got[key], v)


def test_mutated_dense_bruteforce_is_sensitive():
    """The brute force itself differs from a transposed-operand product."""
    pa = I.random_csr(9, 9, 0.4, 11, dtype=None)
    A = _vals_for(oracle.SR_PT_F64, pa, 1)
    B = _vals_for(oracle.SR_PT_F64, I.random_csr(9, 9, 0.4, 12, dtype=None), 2)
    C = oracle.spgemm(oracle.SR_PT_F64, A, B)
    CT = oracle.spgemm(oracle.SR_PT_F64, B, A)
    assert _as_dict(0, C) != _as_dict(0, CT)


# ---- golden, hand-worked ---------------------------------------------------------------

def _golden_graph():
    g = json.load(open(os.path.join(GOLDEN, "semiring_4vertex.json")))
    n = g["n"]
    e = sorted(g["edges"])
    rows = np.array([x[0] for x in e], np.int64)
    cols = np.array([x[1] for x in e], np.int32)
    w = np.array([x[2] for x in e], np.float64)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    return g, I.CSR(n, n, rp, cols, w)


def test_golden_min_plus_plus_times_bool():
    g, W = _golden_graph()
    C = oracle.spgemm(oracle.SR_MP_F32, W.with_values(W.val.astype(np.float32)),
                      W.with_values(W.val.astype(np.float32)))
    assert sorted((i, int(j), float(v)) for i in range(4)
                  for j, v in zip(C.col[C.rp[i]:C.rp[i + 1]], C.val[C.rp[i]:C.rp[i + 1]])) == \
        sorted(tuple(x) for x in g["min_plus"])
    C = oracle.spgemm(oracle.SR_PT_F64, W, W)
    assert sorted((i, int(j), float(v)) for i in range(4)
                  for j, v in zip(C.col[C.rp[i]:C.rp[i + 1]], C.val[C.rp[i]:C.rp[i + 1]])) == \
        sorted(tuple(x) for x in g["plus_times"])
    C = oracle.spgemm(oracle.SR_BOOL, W.with_values(None), W.with_values(None))
    assert sorted((i, int(j)) for i in range(4) for j in C.col[C.rp[i]:C.rp[i + 1]]) == \
        sorted(tuple(x) for x in g["bool_pattern"])


def test_golden_overlap():
    g = json.load(open(os.path.join(GOLDEN, "overlap_3reads.json")))
    rows, cols, vals = [], [], []
    for i, read in enumerate(g["reads"]):
        for c, pos in sorted(read):
            rows.append(i)
            cols.append(c)
            vals.append(pos)
    n = g["nrows"]
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(np.array(rows), minlength=n), out=rp[1:])
    A = I.CSR(n, g["ncols"], rp, np.array(cols, np.int32), np.array(vals, np.int32))
    At = oracle.transpose(A, np.int32)
    C = oracle.spgemm(oracle.SR_OVERLAP, A, At)
    got = []
    for i in range(n):
        for p in range(C.rp[i], C.rp[i + 1]):
            r = C.val[p]
            got.append([i, int(C.col[p]), int(r["count"]), int(r["a0"]), int(r["b0"]),
                        int(r["a1"]), int(r["b1"])])
    assert got == g["C"]


# ---- graph algorithms ----------------------------------------------------------------

def _adj_sets(M):
    return [set(int(c) for c in M.col[M.rp[i]:M.rp[i + 1]]) for i in range(M.nrows)]


@pytest.mark.parametrize("seed", [1, 2])
def test_bool_is_two_hop_reachability(seed):
    A = I.rmat(10, seed=seed, dtype=None)
    C = oracle.spgemm(oracle.SR_BOOL, A, A)
    adj = _adj_sets(A)
    for i in range(A.nrows):
        reach = set()
        for k in adj[i]:
            reach |= adj[k]
        assert set(int(c) for c in C.col[C.rp[i]:C.rp[i + 1]]) == reach
        # i -> k -> i walks: the diagonal is set iff the row is non-empty
        assert (i in reach) == (len(adj[i]) > 0)


def test_min_plus_is_bellman_ford_relaxation():
    A = I.rmat(9, seed=3, dtype=np.float32)
    n = A.nrows
    W = np.full((n, n), np.inf, dtype=np.float32)
    for i in range(n):
        W[i, A.col[A.rp[i]:A.rp[i + 1]]] = A.val[A.rp[i]:A.rp[i + 1]]
    C = oracle.spgemm(oracle.SR_MP_F32, A, A)
    for i in range(n):
        d1 = W[i]                        # one-hop distances (no d[i] = 0)
        d2 = np.min(d1[:, None] + W, axis=0)   # one relaxation over every edge
        cols = C.col[C.rp[i]:C.rp[i + 1]]
        exp_cols = np.nonzero(np.isfinite(d2))[0]
        assert np.array_equal(cols, exp_cols)
        assert np.array_equal(C.val[C.rp[i]:C.rp[i + 1]], d2[exp_cols])


def test_min_plus_symmetric_diagonal_is_twice_lightest_edge():
    A = I.rmat(12, seed=1, dtype=np.float32)
    C = oracle.spgemm(oracle.SR_MP_F32, A, A)
    for i in range(A.nrows):
        a0, a1 = A.rp[i], A.rp[i + 1]
        seg = C.col[C.rp[i]:C.rp[i + 1]]
        if a0 == a1:
            assert i not in seg
            continue
        p = np.searchsorted(seg, i)
        assert seg[p] == i
        assert C.val[C.rp[i] + p] == np.float32(2) * A.val[a0:a1].min()


# ---- plus-times --------------------------------------------------------------------

def test_plus_times_matches_dense_gemm_er4096():
    A = I.er(4096, 8, seed=1)
    C = oracle.spgemm(oracle.SR_PT_F64, A, A)
    D = np.zeros((4096, 4096))
    rows = np.repeat(np.arange(4096), 8)
    D[rows, A.col] = A.val
    G = D @ D
    P = (D != 0).astype(np.float64)
    pattern = (P @ P) > 0
    Cd = np.zeros((4096, 4096))
    crow = np.repeat(np.arange(4096), np.diff(C.rp))
    mask = np.zeros((4096, 4096), bool)
    mask[crow, C.col] = True
    Cd[crow, C.col] = C.val
    assert np.array_equal(mask, pattern)
    assert np.all(np.abs(Cd - G) <= 1e-12 * (np.abs(D) @ np.abs(D)))


def _laplacian_sq_closed_form(g):
    """Entries of L^2 for the Dirichlet 5-point L: diag 16 + (#neighbours),
    axis neighbours -8, diagonal neighbours 2, distance-2 axis entries 1."""
    out = {}
    for y in range(g):
        for x in range(g):
            i = y * g + x
            nb = sum(1 for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1))
                     if 0 <= x + dx < g and 0 <= y + dy < g)
            out[(i, i)] = 16.0 + nb
            for dx, dy, v in ((1, 0, -8.0), (-1, 0, -8.0), (0, 1, -8.0), (0, -1, -8.0),
                              (1, 1, 2.0), (1, -1, 2.0), (-1, 1, 2.0), (-1, -1, 2.0),
                              (2, 0, 1.0), (-2, 0, 1.0), (0, 2, 1.0), (0, -2, 1.0)):
                if 0 <= x + dx < g and 0 <= y + dy < g:
                    out[(i, (y + dy) * g + x + dx)] = v
    return out


@pytest.mark.parametrize("g", [1, 2, 3, 17])
def test_laplacian_square_closed_form(g):
    L = I.laplacian(g)
    C = oracle.spgemm(oracle.SR_PT_F64, L, L)
    got = {}
    for i in range(C.nrows):
        for p in range(C.rp[i], C.rp[i + 1]):
            got[(i, int(C.col[p]))] = float(C.val[p])
    assert got == _laplacian_sq_closed_form(g)
    assert C.nnz == g * g + 4 * g * (g - 1) + 4 * g * max(g - 2, 0) + 4 * (g - 1) ** 2


# ---- identity and permutation invariants -------------------------------------------

def _identity(n, sr):
    one = {oracle.SR_PT_F64: 1.0, oracle.SR_MP_F32: np.float32(0.0), oracle.SR_PT_I64: 1,
           oracle.SR_PT_F32: np.float32(1.0)}
    rp = np.arange(n + 1, dtype=np.int64)
    col = np.arange(n, dtype=np.int32)
    if sr == oracle.SR_BOOL:
        return I.CSR(n, n, rp, col, None)
    return I.CSR(n, n, rp, col, np.full(n, one[sr], dtype=oracle.IN_DTYPE[sr]))


@pytest.mark.parametrize("sr", [oracle.SR_PT_F64, oracle.SR_BOOL, oracle.SR_MP_F32,
                                oracle.SR_PT_I64, oracle.SR_PT_F32])
def test_identity(sr):
    A = _vals_for(sr, I.random_csr(40, 30, 0.2, 9, dtype=None, empty_row_frac=0.2), 3)
    for C in (oracle.spgemm(sr, A, _identity(30, sr)), oracle.spgemm(sr, _identity(40, sr), A)):
        assert_pattern_equal(C.rp, C.col, A.rp, A.col)
        if sr != oracle.SR_BOOL:
            assert np.array_equal(C.val.view(np.uint8), A.val.view(np.uint8))


def _permute(M, prow, pcol):
    """M' with M'[prow[i], pcol[j]] = M[i, j]."""
    rows = np.repeat(np.arange(M.nrows), np.diff(M.rp))
    r2 = prow[rows]
    c2 = pcol[M.col.astype(np.int64)]
    order = np.lexsort((c2, r2))
    rp = np.zeros(M.nrows + 1, np.int64)
    np.cumsum(np.bincount(r2, minlength=M.nrows), out=rp[1:])
    return I.CSR(M.nrows, M.ncols, rp, c2[order].astype(np.int32),
                 None if M.val is None else M.val[order])


@pytest.mark.parametrize("sr", ALL_SR)
def test_permutation_invariance(sr):
    rng = np.random.default_rng(5)
    A = _vals_for(sr, I.random_csr(50, 40, 0.15, 21, dtype=None), 1)
    B = _vals_for(sr, I.random_csr(40, 45, 0.15, 22, dtype=None), 2)
    p, q, r = rng.permutation(50), rng.permutation(40), rng.permutation(45)
    C = oracle.spgemm(sr, A, B)
    C2 = oracle.spgemm(sr, _permute(A, p, q), _permute(B, q, r))
    Cp = _permute(I.CSR(C.nrows, C.ncols, C.rp, C.col, C.val), p, r)
    assert_pattern_equal(C2.rp, C2.col, Cp.rp, Cp.col)
    if sr == oracle.SR_PT_F64:
        bound = oracle.spgemm(sr, abs_csr(A), abs_csr(B))
        bp = _permute(I.CSR(bound.nrows, bound.ncols, bound.rp, bound.col, bound.val), p, r)
        assert_values(sr, C2.val, Cp.val, bound=bp.val)
    elif sr == oracle.SR_PT_F32:
        bound = oracle.spgemm(oracle.SR_PT_F64, abs_csr(A).__class__(
            nrows=A.nrows, ncols=A.ncols, rp=A.rp, col=A.col, val=np.abs(A.val).astype(np.float64)),
            abs_csr(B).__class__(nrows=B.nrows, ncols=B.ncols, rp=B.rp, col=B.col,
                                 val=np.abs(B.val).astype(np.float64)))
        bp = _permute(I.CSR(bound.nrows, bound.ncols, bound.rp, bound.col, bound.val), p, r)
        terms = oracle.spgemm(oracle.SR_OVERLAP, I.positions_csr(A, 1), I.positions_csr(B, 2))
        tp = _permute(I.CSR(terms.nrows, terms.ncols, terms.rp, terms.col,
                            terms.val["count"].astype(np.float64)), p, r)
        assert_values(sr, C2.val, Cp.val, bound=bp.val, terms=tp.val)
    elif sr == oracle.SR_OVERLAP:
        # pairs hold positions in rows of A and B; permuting rows and columns
        # keeps them, so the records are identical
        assert_values(sr, C2.val, Cp.val)
    else:
        assert_values(sr, C2.val, Cp.val)


# ---- overlap invariants --------------------------------------------------------------

def test_overlap_invariants_kmer():
    A = I.kmer(300, 4096, len_lo=5, len_hi=40, col_cap=8, seed=4)
    At = oracle.transpose(A, np.int32)
    C = oracle.spgemm(oracle.SR_OVERLAP, A, At)
    pos = [dict(zip(A.col[A.rp[i]:A.rp[i + 1]].tolist(), A.val[A.rp[i]:A.rp[i + 1]].tolist()))
           for i in range(A.nrows)]
    NP = 2**31 - 1
    rec = {}
    for i in range(C.nrows):
        for p in range(C.rp[i], C.rp[i + 1]):
            r = C.val[p]
            rec[(i, int(C.col[p]))] = (int(r["count"]), (int(r["a0"]), int(r["b0"])),
                                       (int(r["a1"]), int(r["b1"])))
    for i in range(A.nrows):
        for j in range(A.nrows):
            shared = set(pos[i]) & set(pos[j])
            if not shared:
                assert (i, j) not in rec
                continue
            pairs = sorted((pos[i][k], pos[j][k]) for k in shared)
            exp = (len(shared), pairs[0], pairs[1] if len(pairs) > 1 else (NP, NP))
            assert rec[(i, j)] == exp
            # symmetry: C[j,i] holds the same pairs swapped
            swapped = sorted((b, a) for a, b in pairs)
            assert rec[(j, i)][1] == swapped[0]
            if i == j:
                ln = len(pos[i])
                assert rec[(i, i)] == (ln, (0, 0), (1, 1) if ln > 1 else (NP, NP))


# ---- transpose and the transpose identity ----------------------------------------

def test_transpose_matches_dense():
    A = I.random_csr(23, 31, 0.2, 5)
    T = oracle.transpose(A, np.float64)
    D = np.zeros((23, 31))
    rows = np.repeat(np.arange(23), np.diff(A.rp))
    D[rows, A.col] = A.val
    Dt = np.zeros((31, 23))
    trow = np.repeat(np.arange(31), np.diff(T.rp))
    Dt[trow, T.col] = T.val
    assert np.array_equal(Dt, D.T)
    assert T.nnz == A.nnz
    for i in range(31):
        assert np.all(np.diff(T.col[T.rp[i]:T.rp[i + 1]]) > 0)


@pytest.mark.parametrize("sr", [oracle.SR_PT_F64, oracle.SR_BOOL, oracle.SR_MP_F32,
                                oracle.SR_PT_I64])
def test_transpose_identity(sr):
    A = _vals_for(sr, I.random_csr(30, 25, 0.2, 31, dtype=None), 1)
    B = _vals_for(sr, I.random_csr(25, 35, 0.2, 32, dtype=None), 2)
    dt = oracle.IN_DTYPE[sr]
    C = oracle.spgemm(sr, A, B)
    Ct = oracle.spgemm(sr, oracle.transpose(B, dt), oracle.transpose(A, dt))
    C2 = oracle.transpose(Ct, dt)
    assert_pattern_equal(C2.rp, C2.col, C.rp, C.col)
    if sr != oracle.SR_BOOL:
        # same k order and commutative (x): bit-identical even for plus-times
        assert np.array_equal(C2.val.view(np.uint8), C.val.view(np.uint8))


# ---- merge of stage partials (block-grid Sparse SUMMA) -----------------------------

@pytest.mark.parametrize("sr", ALL_SR)
def test_block_grid_merge_equals_unblocked(sr):
    n = 64
    pat = I.rmat(6, seed=2, dtype=None)
    A = _vals_for(sr, pat, 3)
    B = _vals_for(sr, pat, 4) if sr != oracle.SR_OVERLAP else I.positions_csr(pat, 4)
    cuts = [0, 5, 21, 40, 64]
    Ab = oracle.summa_blocks(A, cuts, cuts)
    Bb = oracle.summa_blocks(B, cuts, cuts)
    C = oracle.spgemm(sr, A, B)
    for Ib in range(4):
        for Jb in range(4):
            parts = [oracle.spgemm(sr, Ab[Ib][s], Bb[s][Jb]) for s in range(4)]
            M = oracle.merge(sr, parts)
            Cb = oracle.summa_blocks(C, cuts, cuts)[Ib][Jb]
            assert_pattern_equal(M.rp, M.col, Cb.rp, Cb.col, f"block {Ib},{Jb}")
            if sr == oracle.SR_PT_F64:
                bnd = oracle.summa_blocks(oracle.spgemm(sr, abs_csr(A), abs_csr(B)), cuts, cuts)
                assert_values(sr, M.val, Cb.val, bound=bnd[Ib][Jb].val)
            elif sr == oracle.SR_PT_F32:
                assert np.allclose(M.val, Cb.val, rtol=1e-5, atol=1e-5)
            else:
                assert_values(sr, M.val, Cb.val)


def test_merge_is_fold_in_stage_order():
    """Three one-entry partials: the merge is ((p0 (+) p1) (+) p2)."""
    parts = []
    for v in (0.1, 0.2, 0.3):
        parts.append(I.CSR(1, 4, np.array([0, 1], np.int64), np.array([2], np.int32),
                           np.array([v])))
    M = oracle.merge(oracle.SR_PT_F64, parts)
    assert M.val[0] == (0.1 + 0.2) + 0.3
    ov = []
    for c, a in ((1, 5), (1, 3), (2, 4)):
        rec = np.zeros(1, oracle.OVERLAP_DTYPE)
        rec["count"], rec["a0"], rec["b0"], rec["a1"], rec["b1"] = c, a, 0, 2**31 - 1, 2**31 - 1
        ov.append(I.CSR(1, 4, np.array([0, 1], np.int64), np.array([2], np.int32), rec))
    M = oracle.merge(oracle.SR_OVERLAP, ov)
    r = M.val[0]
    assert (r["count"], r["a0"], r["b0"], r["a1"], r["b1"]) == (4, 3, 0, 4, 0)


# ---- row analysis ------------------------------------------------------------------

def test_row_upper_bounds_by_loop():
    A = I.random_csr(40, 30, 0.2, 1, empty_row_frac=0.2)
    B = I.random_csr(30, 50, 0.3, 2, empty_row_frac=0.2)
    ub = oracle.row_upper_bounds(A, B)
    for i in range(40):
        s = 0
        for p in range(A.rp[i], A.rp[i + 1]):
            k = A.col[p]
            s += B.rp[k + 1] - B.rp[k]
        assert ub[i] == s
    # the number of oracle products equals the upper bound (overlap counts products)
    C = oracle.spgemm(oracle.SR_OVERLAP, I.positions_csr(A, 1), I.positions_csr(B, 2))
    tot = np.add.reduceat(np.r_[C.val["count"], 0].astype(np.int64),
                          np.minimum(C.rp[:-1], C.nnz)) * (np.diff(C.rp) > 0)
    assert np.array_equal(tot, ub)


def test_generators_deterministic_and_valid():
    for make in (lambda: I.er(512, 8, seed=7), lambda: I.rmat(9, seed=7),
                 lambda: I.kmer(100, 2048, 5, 20, col_cap=6, seed=7), lambda: I.laplacian(9)):
        a, b = make(), make()
        assert np.array_equal(a.rp, b.rp) and np.array_equal(a.col, b.col)
        assert np.array_equal(a.val, b.val)
        for i in range(a.nrows):
            assert np.all(np.diff(a.col[a.rp[i]:a.rp[i + 1]]) > 0)
        assert a.col.min() >= 0 and a.col.max() < a.ncols
    K = I.kmer(100, 2048, 5, 20, col_cap=6, seed=7)
    assert np.bincount(K.col, minlength=2048).max() <= 6
    for i in range(K.nrows):
        assert sorted(K.val[K.rp[i]:K.rp[i + 1]].tolist()) == list(range(K.rp[i + 1] - K.rp[i]))
    R = I.rmat(9, seed=7)
    D = np.zeros((512, 512), np.float32)
    rows = np.repeat(np.arange(512), np.diff(R.rp))
    D[rows, R.col] = R.val
    assert np.array_equal(D, D.T) and np.all(np.diag(D) == 0)


# ---- masked product (oracle.masked) ------------------------------------------

def _lower(A):
    rows, cols = [], []
    for i in range(A.nrows):
        c = A.col[A.rp[i]:A.rp[i + 1]]
        c = c[c < i]
        rows.append(np.full(c.size, i, dtype=np.int64))
        cols.append(c)
    r = np.concatenate(rows)
    c = np.concatenate(cols).astype(np.int32)
    rp = np.zeros(A.nrows + 1, dtype=np.int64)
    np.add.at(rp, r + 1, 1)
    return I.CSR(A.nrows, A.ncols, np.cumsum(rp), c, np.ones(c.size, dtype=np.int64))


def test_masked_triangle_count_matches_trace():
    """sum of (L L) o L over plus-times = number of triangles = trace(A^3) / 6."""
    A = I.rmat(8, seed=5, dtype=None)
    L = _lower(A)
    C = oracle.masked(oracle.SR_PT_I64, L, L, L)
    D = np.zeros((A.nrows, A.nrows), dtype=np.int64)
    for i in range(A.nrows):
        D[i, A.col[A.rp[i]:A.rp[i + 1]]] = 1
    assert int(C.val.sum()) == int(np.trace(D @ D @ D)) // 6
    assert int(C.val.sum()) > 0


def test_masked_dense_brute_force_and_limits():
    rng = np.random.default_rng(3)
    A = I.random_csr(20, 15, 0.3, 1, dtype=np.float64, empty_row_frac=0.1)
    B = I.random_csr(15, 25, 0.3, 2, dtype=np.float64)
    M = I.random_csr(20, 25, 0.4, 3, dtype=None)
    C = oracle.masked(oracle.SR_PT_F64, A, B, M)
    Ad, Bd = np.zeros((20, 15)), np.zeros((15, 25))
    Ph = np.zeros((20, 25), dtype=bool)   # has a product
    for i in range(20):
        for p in range(A.rp[i], A.rp[i + 1]):
            k = A.col[p]
            Ad[i, k] = A.val[p]
            for q in range(B.rp[k], B.rp[k + 1]):
                Ph[i, B.col[q]] = True
    for k in range(15):
        Bd[k, B.col[B.rp[k]:B.rp[k + 1]]] = B.val[B.rp[k]:B.rp[k + 1]]
    Md = np.zeros((20, 25), dtype=bool)
    for i in range(20):
        Md[i, M.col[M.rp[i]:M.rp[i + 1]]] = True
    want = Ph & Md
    got = np.zeros((20, 25), dtype=bool)
    vals = np.zeros((20, 25))
    for i in range(20):
        got[i, C.col[C.rp[i]:C.rp[i + 1]]] = True
        vals[i, C.col[C.rp[i]:C.rp[i + 1]]] = C.val[C.rp[i]:C.rp[i + 1]]
    assert np.array_equal(got, want)
    assert np.allclose(vals[want], (Ad @ Bd)[want], rtol=1e-12, atol=1e-15)
    # mask = C's own pattern gives C; an empty mask gives nothing
    full = oracle.spgemm(oracle.SR_PT_F64, A, B)
    same = oracle.masked(oracle.SR_PT_F64, A, B, full)
    assert np.array_equal(same.rp, full.rp) and np.array_equal(same.val, full.val)
    empty = I.random_csr(20, 25, 0.0, 4, dtype=None)
    assert oracle.masked(oracle.SR_PT_F64, A, B, empty).nnz == 0
    del rng
