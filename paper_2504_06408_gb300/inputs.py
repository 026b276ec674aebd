"""Seeded synthetic input generators (host side, numpy).

This module is the one piece shared by the CUDA path, the CPU oracle and the
benchmark: it only draws matrices.  It holds none of the multiplication,
merge or transpose arithmetic, so the oracle and the kernels stay independent.

Workloads (stand-ins for the paper's SuiteSparse graph/PDE matrices and the
genomics use case of the introduction, Section 1 and Table 2):

* ``er``        Erdos-Renyi: exactly ``per_row`` distinct uniform columns a row.
* ``rmat``      R-MAT (a, b, c, d) recursive edges, symmetrised, self loops and
                duplicates removed, one weight per undirected edge.
* ``kmer``      k-mer-style reads x k-mers matrix: row length uniform in
                [lo, hi], column ids Zipf(s) over ``ncols`` ranks mapped through
                a seeded permutation, at most ``col_cap`` entries per column,
                value = position of the k-mer in generation order.
* ``laplacian`` Dirichlet 5-point stencil on a g x g grid (4 on the diagonal,
                -1 for each grid neighbour).
* ``random_csr`` small irregular matrices for edge-case tests (empty rows,
                empty columns, chosen density).

Every matrix is a :class:`CSR` with int64 row pointers, int32 column ids
strictly ascending within a row, and a value array (or ``None`` for the
pattern-only boolean semiring).
"""
from __future__ import annotations

import hashlib
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class CSR:
    nrows: int
    ncols: int
    rp: np.ndarray            # int64, nrows + 1
    col: np.ndarray           # int32, nnz
    val: Optional[np.ndarray]  # nnz values (dtype per semiring) or None

    @property
    def nnz(self) -> int:
        return int(self.rp[-1])

    def with_values(self, val: Optional[np.ndarray]) -> "CSR":
        return CSR(self.nrows, self.ncols, self.rp, self.col, val)


# Large generated matrices are kept on disk between processes (the tests and
# the benchmark draw the same seeded inputs); the directory is outside the
# repository.  SPGEMM_INPUT_CACHE="" turns the cache off.
_CACHE_DIR = os.environ.get("SPGEMM_INPUT_CACHE", "/tmp/spgemm_inputs")
_CACHE_MIN_NNZ = 4_000_000


def _cached(name: str, key: tuple, make):
    """make() on a miss; the CSR's arrays are stored under a name derived from
    the generator's arguments and read back on later calls."""
    if not _CACHE_DIR:
        return make()
    tag = hashlib.sha256(repr((name, key)).encode()).hexdigest()[:20]
    path = os.path.join(_CACHE_DIR, f"{name}_{tag}.npz")
    try:
        with np.load(path, allow_pickle=False) as z:
            val = z["val"] if "val" in z.files else None
            return CSR(int(z["shape"][0]), int(z["shape"][1]), z["rp"], z["col"], val)
    except (OSError, KeyError, ValueError):
        pass
    M = make()
    if M.nnz >= _CACHE_MIN_NNZ:
        try:
            os.makedirs(_CACHE_DIR, exist_ok=True)
            tmp = f"{path}.{os.getpid()}.tmp.npz"
            arrays = {"shape": np.array([M.nrows, M.ncols], np.int64), "rp": M.rp, "col": M.col}
            if M.val is not None:
                arrays["val"] = M.val
            np.savez(tmp, **arrays)
            os.replace(tmp, path)
        except OSError:
            pass
    return M


def _from_sorted_coo(nrows: int, ncols: int, rows: np.ndarray, cols: np.ndarray,
                     vals: Optional[np.ndarray]) -> CSR:
    """Build a CSR from COO triples already sorted by (row, col), no duplicates."""
    counts = np.bincount(rows, minlength=nrows).astype(np.int64)
    rp = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return CSR(nrows, ncols, rp, cols.astype(np.int32, copy=False), vals)


def _uniform(rng: np.random.Generator, n: int, lo: float, hi: float, dtype) -> np.ndarray:
    """n draws uniform in [lo, hi) rounded to ``dtype``, never equal to hi."""
    x = (lo + (hi - lo) * rng.random(n)).astype(dtype)
    top = np.nextafter(dtype(hi), dtype(lo))
    np.minimum(x, top, out=x)
    return x


def er(n: int = 4096, per_row: int = 8, seed: int = 1, dtype=np.float64,
       lo: float = 0.0, hi: float = 1.0) -> CSR:
    """n x n matrix, exactly ``per_row`` distinct uniform columns per row."""
    rng = np.random.default_rng(seed)
    cols = np.empty((n, per_row), dtype=np.int64)
    for i in range(n):
        cols[i] = np.sort(rng.choice(n, size=per_row, replace=False))
    rp = np.arange(0, n * per_row + 1, per_row, dtype=np.int64)
    val = None if dtype is None else _uniform(rng, n * per_row, lo, hi, dtype)
    return CSR(n, n, rp, cols.reshape(-1).astype(np.int32), val)


def rmat_edges(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
               c: float = 0.19, seed: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """Directed R-MAT edge list (no noise, no relabelling: low ids are hubs)."""
    rng = np.random.default_rng(seed)
    m = edge_factor << scale
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for level in range(scale):
        u = rng.random(m)
        bit = np.int64(1) << (scale - 1 - level)
        row_bit = u >= ab                       # quadrants c, d
        col_bit = ((u >= a) & (u < ab)) | (u >= abc)  # quadrants b, d
        src += row_bit * bit
        dst += col_bit * bit
    return src, dst


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, dtype=np.float32, lo: float = 1.0,
         hi: float = 100.0) -> CSR:
    """Symmetric R-MAT adjacency matrix with one weight per undirected edge
    (see _rmat); large ones are kept in the input cache."""
    make = lambda: _rmat(scale, edge_factor, a, b, c, seed, dtype, lo, hi)  # noqa: E731
    if scale < 17:
        return make()
    key = (scale, edge_factor, a, b, c, seed, None if dtype is None else np.dtype(dtype).str,
           lo, hi)
    return _cached("rmat", key, make)


def _rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int, dtype,
          lo: float, hi: float) -> CSR:
    """Symmetric R-MAT adjacency matrix with one weight per undirected edge.

    ``dtype=None`` gives a pattern-only matrix.
    """
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor, a, b, c, seed)
    keep = src != dst
    lo_v = np.minimum(src[keep], dst[keep])
    hi_v = np.maximum(src[keep], dst[keep])
    und = np.unique(lo_v * n + hi_v)          # undirected edges, sorted
    del src, dst, keep, lo_v, hi_v
    u_ = und // n
    v_ = und - u_ * n
    rng = np.random.default_rng(seed + 0x5EED)
    w = None if dtype is None else _uniform(rng, und.size, lo, hi, dtype)
    rows = np.concatenate([u_, v_])
    cols = np.concatenate([v_, u_])
    order = np.argsort(rows * n + cols, kind="stable")
    rows = rows[order]
    cols = cols[order]
    vals = None if w is None else np.concatenate([w, w])[order]
    return _from_sorted_coo(n, n, rows, cols, vals)


def laplacian(g: int = 2048, dtype=np.float64) -> CSR:
    """Dirichlet 5-point stencil on a g x g grid, row-major vertex order."""
    n = g * g
    idx = np.arange(n, dtype=np.int64)
    x = idx % g
    y = idx // g
    offs = [(-g, y > 0), (-1, x > 0), (0, np.ones(n, bool)), (1, x < g - 1), (g, y < g - 1)]
    cols = np.full((n, 5), -1, dtype=np.int64)
    vals = np.zeros((n, 5), dtype=np.float64)
    for t, (d, ok) in enumerate(offs):
        cols[ok, t] = idx[ok] + d
        vals[ok, t] = 4.0 if d == 0 else -1.0
    mask = cols >= 0
    counts = mask.sum(axis=1)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    v = None if dtype is None else vals[mask].astype(dtype)
    return CSR(n, n, rp, cols[mask].astype(np.int32), v)


def trigrid(g: int, dtype=np.float32, seed: int = 1) -> CSR:
    """Triangular lattice on a g x g grid: every vertex joined to its 6
    neighbours (x +- 1, y +- 1, and the diagonal (x + 1, y - 1), (x - 1, y + 1)),
    no diagonal entries, weights U[0, 1) per undirected edge.  Stand-in for a
    planar Delaunay triangulation (delaunay_n22: 4.19M rows, 6.0 entries per
    row)."""
    n = g * g
    idx = np.arange(n, dtype=np.int64)
    x, y = idx % g, idx // g
    deltas = sorted([(1, -1), (0, -1), (-1, 0), (1, 0), (0, 1), (-1, 1)],
                    key=lambda d: d[1] * g + d[0])
    cols = np.full((n, 6), -1, dtype=np.int64)
    for t, (dx, dy) in enumerate(deltas):
        ok = (x + dx >= 0) & (x + dx < g) & (y + dy >= 0) & (y + dy < g)
        cols[ok, t] = idx[ok] + dy * g + dx
    mask = cols >= 0
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=rp[1:])
    col = cols[mask]
    if dtype is None:
        return CSR(n, n, rp, col.astype(np.int32), None)
    # one weight per undirected edge {min, max}: symmetric values
    rows = np.repeat(idx, mask.sum(axis=1))
    lo, hi = np.minimum(rows, col), np.maximum(rows, col)
    rng = np.random.default_rng(seed)
    w_edge = _uniform(rng, n * 3 + 1, 0.0, 1.0, np.float64)
    key = lo * 3 + np.select([hi - lo == 1, hi - lo == g - 1], [0, 1], 2)
    return CSR(n, n, rp, col.astype(np.int32), w_edge[key].astype(dtype))


def stencil3d(g: int, points: int = 7, dtype=np.float32) -> CSR:
    """Dirichlet 3D stencil on a g x g x g grid (x fastest): 7 points (faces,
    value 6 on the diagonal and -1 off it) or 27 points (the full 3 x 3 x 3
    neighbourhood, 26 and -1).  Stand-ins for the PDE matrices of the
    paper's experiments (atmosmodd: 1.27M rows, 8.8M entries, about a 7-point
    108^3 grid; Long_dt_Coup0: a 3D coupled problem)."""
    if points not in (7, 27):
        raise ValueError("points must be 7 or 27")
    n = g * g * g
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % g, (idx // g) % g, idx // (g * g)
    if points == 7:
        deltas = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    else:
        deltas = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    # ascending column order: offsets dz * g^2 + dy * g + dx are increasing in this order
    deltas.sort(key=lambda d: d[2] * g * g + d[1] * g + d[0])
    cols = np.full((n, len(deltas)), -1, dtype=np.int64)
    vals = np.zeros((n, len(deltas)), dtype=np.float64)
    for t, (dx, dy, dz) in enumerate(deltas):
        ok = ((x + dx >= 0) & (x + dx < g) & (y + dy >= 0) & (y + dy < g) &
              (z + dz >= 0) & (z + dz < g))
        cols[ok, t] = idx[ok] + dz * g * g + dy * g + dx
        vals[ok, t] = (len(deltas) - 1.0) if (dx, dy, dz) == (0, 0, 0) else -1.0
    mask = cols >= 0
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=rp[1:])
    v = None if dtype is None else vals[mask].astype(dtype)
    return CSR(n, n, rp, cols[mask].astype(np.int32), v)


def _zipf_cdf(nranks: int, s: float) -> np.ndarray:
    w = np.arange(1, nranks + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    return cdf


def kmer(nrows: int = 200_000, ncols: int = 1 << 24, len_lo: int = 50, len_hi: int = 200,
         s: float = 1.1, col_cap: int = 64, seed: int = 1, max_rounds: int = 100000) -> CSR:
    """Reads x k-mers matrix (see _kmer), kept in the input cache."""
    return _cached("kmer", (nrows, ncols, len_lo, len_hi, s, col_cap, seed, max_rounds),
                   lambda: _kmer(nrows, ncols, len_lo, len_hi, s, col_cap, seed, max_rounds))


def _kmer(nrows: int, ncols: int, len_lo: int, len_hi: int, s: float, col_cap: int, seed: int,
          max_rounds: int) -> CSR:
    """Reads x k-mers matrix; value = position of the k-mer in its read.

    Row lengths are uniform in [len_lo, len_hi].  Each slot draws a Zipf(s)
    rank over ``ncols`` ranks, mapped to a column id by a seeded permutation.
    A draw that repeats a column already in the row, or hits a column that
    already holds ``col_cap`` entries, is redrawn, until every row is full.
    Positions 0..len-1 follow generation (draw) order, so after sorting the
    row by column the values are a permutation of 0..len-1.
    """
    rng = np.random.default_rng(seed)
    lens = rng.integers(len_lo, len_hi + 1, size=nrows).astype(np.int64)
    if int(lens.sum()) > ncols * col_cap:
        raise ValueError("row lengths exceed total column capacity")
    perm = rng.permutation(ncols).astype(np.int64)
    cdf = _zipf_cdf(ncols, s)
    filled = np.zeros(nrows, dtype=np.int64)
    col_count = np.zeros(ncols, dtype=np.int64)
    # accepted (row, col, position) triples
    acc_rows, acc_cols, acc_pos = [], [], []
    seen_keys = np.zeros(0, dtype=np.int64)   # sorted row * ncols + col of accepted
    for _ in range(max_rounds):
        need = lens - filled
        todo = np.nonzero(need > 0)[0]
        if todo.size == 0:
            break
        reps = need[todo]
        r = np.repeat(todo, reps)
        u = rng.random(r.size)
        cidx = perm[np.minimum(np.searchsorted(cdf, u, side="right"), ncols - 1)]
        key = r * ncols + cidx
        # drop repeats of a column already accepted in the row
        if seen_keys.size:
            at = np.searchsorted(seen_keys, key)
            at = np.minimum(at, seen_keys.size - 1)
            fresh = seen_keys[at] != key
        else:
            fresh = np.ones(r.size, bool)
        # drop repeats within this round (keep the first draw in slot order)
        _, first = np.unique(key, return_index=True)
        uniq = np.zeros(r.size, bool)
        uniq[first] = True
        ok = fresh & uniq
        # column cap: within each column accept draws in slot order up to capacity
        cand = np.nonzero(ok)[0]
        cc = cidx[cand]
        order = np.lexsort((cand, cc))
        cand = cand[order]
        cc = cc[order]
        bounds = np.r_[0, np.nonzero(np.diff(cc))[0] + 1]
        rank = np.arange(cc.size) - np.repeat(bounds, np.diff(np.r_[bounds, cc.size]))
        room = col_cap - col_count[cc]
        take = cand[rank < room]
        if take.size == 0:
            continue
        # an accepted draw keeps its slot only if every earlier slot of its row was
        # accepted too; later accepted slots are renumbered to stay consecutive.
        acc_mask = np.zeros(r.size, bool)
        acc_mask[take] = True
        rr = r[acc_mask]
        # renumber: position = filled[row] + ordinal among accepted draws of the row
        ordn = np.arange(rr.size)
        rstart = np.r_[0, np.nonzero(np.diff(rr))[0] + 1]
        first_of = np.repeat(rstart, np.diff(np.r_[rstart, rr.size]))
        newpos = filled[rr] + (ordn - first_of)
        cols_t = cidx[acc_mask]
        acc_rows.append(rr)
        acc_cols.append(cols_t)
        acc_pos.append(newpos)
        np.add.at(filled, rr, 1)
        np.add.at(col_count, cols_t, 1)
        new_keys = np.sort(rr * ncols + cols_t)
        seen_keys = np.insert(seen_keys, np.searchsorted(seen_keys, new_keys), new_keys)
    else:
        raise RuntimeError("k-mer generator did not fill every row")
    rows = np.concatenate(acc_rows)
    cols = np.concatenate(acc_cols)
    posv = np.concatenate(acc_pos)
    order = np.lexsort((cols, rows))
    return _from_sorted_coo(nrows, ncols, rows[order], cols[order],
                            posv[order].astype(np.int32))


def random_csr(nrows: int, ncols: int, density: float, seed: int, dtype=np.float64,
               lo: float = 0.0, hi: float = 1.0, empty_row_frac: float = 0.0,
               empty_col_frac: float = 0.0, int_vals: bool = False) -> CSR:
    """Small irregular matrix: Bernoulli(density) pattern with forced empty rows/cols.

    ``int_vals`` draws integers in [lo, hi) (stored in ``dtype``), which keeps
    plus-times sums exact for tests that need bit equality.
    """
    rng = np.random.default_rng(seed)
    mask = rng.random((nrows, ncols)) < density
    if empty_row_frac > 0:
        mask[rng.random(nrows) < empty_row_frac, :] = False
    if empty_col_frac > 0:
        mask[:, rng.random(ncols) < empty_col_frac] = False
    rows, cols = np.nonzero(mask)
    if dtype is None:
        vals = None
    elif int_vals:
        vals = rng.integers(int(lo), int(hi), size=rows.size).astype(dtype)
    else:
        vals = _uniform(rng, rows.size, lo, hi, dtype)
    return _from_sorted_coo(nrows, ncols, rows.astype(np.int64), cols, vals)


def positions_csr(pattern: CSR, seed: int) -> CSR:
    """Same pattern, int32 values = a random permutation of 0..len-1 per row
    (the overlap semiring's "position in read" values for arbitrary patterns)."""
    rng = np.random.default_rng(seed)
    val = np.empty(pattern.nnz, dtype=np.int32)
    for i in range(pattern.nrows):
        a, b = int(pattern.rp[i]), int(pattern.rp[i + 1])
        val[a:b] = rng.permutation(b - a)
    return pattern.with_values(val)
