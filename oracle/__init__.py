"""CPU oracle for semiring SpGEMM -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and it
never calls the CUDA library: the two share no code.

The arithmetic lives in ``spgemm_oracle.cpp`` (sorted-map Gustavson, stage
merge, transpose); this module only marshals numpy arrays and adds two plain
numpy definitions:

* :func:`row_upper_bounds` -- ub_i = sum over k in cols(A_i) of nnz(B_k), the
  number of intermediate products of output row i (Gustavson's work count;
  the paper's Section 2.1 defines SpGEMM, the count follows from it).
* :func:`summa_blocks` -- splits a matrix into a q x q block grid, the data
  layout of Sparse SUMMA (Section 2.1): block (I, J) holds rows
  [r_I, r_{I+1}) and columns [c_J, c_{J+1}) with local column ids.

Every function here is pinned by ``tests/test_oracle_pins.py`` against
dense brute force, graph algorithms, dense GEMM, closed forms and algebraic
invariants.
"""
from __future__ import annotations

import ctypes
import os
from types import SimpleNamespace

import numpy as np

from . import build as _build

SR_PT_F64, SR_BOOL, SR_MP_F32, SR_OVERLAP, SR_PT_I64, SR_PT_F32 = 0, 1, 2, 3, 4, 5
IN_DTYPE = {SR_PT_F64: np.float64, SR_BOOL: None, SR_MP_F32: np.float32,
            SR_OVERLAP: np.int32, SR_PT_I64: np.int64, SR_PT_F32: np.float32}
# overlap output record: count, (a0, b0) smallest pair, (a1, b1) second pair
OVERLAP_DTYPE = np.dtype([("count", np.int32), ("a0", np.int32), ("b0", np.int32),
                          ("a1", np.int32), ("b1", np.int32)])
OUT_DTYPE = dict(IN_DTYPE)
OUT_DTYPE[SR_OVERLAP] = OVERLAP_DTYPE
NO_PAIR = np.int32(2**31 - 1)


class _OCsr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64),
                ("rp", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        lib.oracle_spgemm_rows.restype = ctypes.c_void_p
        lib.oracle_spgemm_rows.argtypes = [ctypes.c_int, ctypes.POINTER(_OCsr),
                                           ctypes.POINTER(_OCsr), ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_int]
        lib.oracle_merge.restype = ctypes.c_void_p
        lib.oracle_merge.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_OCsr),
                                     ctypes.c_int]
        lib.oracle_transpose.restype = ctypes.c_void_p
        lib.oracle_transpose.argtypes = [ctypes.POINTER(_OCsr), ctypes.c_int]
        lib.oracle_result_nrows.restype = ctypes.c_int64
        lib.oracle_result_nrows.argtypes = [ctypes.c_void_p]
        lib.oracle_result_nnz.restype = ctypes.c_int64
        lib.oracle_result_nnz.argtypes = [ctypes.c_void_p]
        lib.oracle_result_copy.restype = None
        lib.oracle_result_copy.argtypes = [ctypes.c_void_p] * 4
        lib.oracle_result_free.restype = None
        lib.oracle_result_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


def _csr_struct(M, val_dtype):
    rp = np.ascontiguousarray(M.rp, dtype=np.int64)
    col = np.ascontiguousarray(M.col, dtype=np.int32)
    val = None
    if val_dtype is not None:
        val = np.ascontiguousarray(M.val, dtype=val_dtype)
    keep = (rp, col, val)
    s = _OCsr(M.nrows, M.ncols, rp.ctypes.data, col.ctypes.data,
              None if val is None else val.ctypes.data)
    return s, keep


def _collect(res, ncols, out_dtype):
    lib = _load()
    if not res:
        raise ValueError("oracle rejected its arguments")
    try:
        n = lib.oracle_result_nrows(res)
        nnz = lib.oracle_result_nnz(res)
        rp = np.zeros(n + 1, dtype=np.int64)
        col = np.zeros(nnz, dtype=np.int32)
        val = None if out_dtype is None else np.zeros(nnz, dtype=out_dtype)
        lib.oracle_result_copy(res, rp.ctypes.data, col.ctypes.data,
                               None if val is None else val.ctypes.data)
    finally:
        lib.oracle_result_free(res)
    return SimpleNamespace(nrows=n, ncols=ncols, rp=rp, col=col, val=val, nnz=nnz)


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def spgemm(sr: int, A, B, rows=None, threads: int | None = None):
    """C = A (x).(+) B over semiring ``sr`` (rows of A restricted to ``rows``)."""
    if A.ncols != B.nrows:
        raise ValueError("inner dimensions differ")
    a, ka = _csr_struct(A, IN_DTYPE[sr])
    b, kb = _csr_struct(B, IN_DTYPE[sr])
    sel = None
    nsel = A.nrows
    if rows is not None:
        sel = np.ascontiguousarray(rows, dtype=np.int64)
        nsel = sel.size
    th = default_threads() if threads is None else threads
    res = _load().oracle_spgemm_rows(sr, ctypes.byref(a), ctypes.byref(b), nsel,
                                     None if sel is None else sel.ctypes.data, th)
    return _collect(res, B.ncols, OUT_DTYPE[sr])


def merge(sr: int, parts, threads: int | None = None):
    """(+)-merge of stage partials (same shape), folded in stage order."""
    structs, keep = [], []
    for P in parts:
        s, k = _csr_struct(P, OUT_DTYPE[sr])
        structs.append(s)
        keep.append(k)
    arr = (_OCsr * len(structs))(*structs)
    th = default_threads() if threads is None else threads
    res = _load().oracle_merge(sr, len(structs), arr, th)
    return _collect(res, parts[0].ncols, OUT_DTYPE[sr])


def transpose(A, val_dtype=None):
    """A^T, values carried (``val_dtype`` None: pattern only)."""
    s, k = _csr_struct(A, val_dtype)
    nbytes = 0 if val_dtype is None else np.dtype(val_dtype).itemsize
    res = _load().oracle_transpose(ctypes.byref(s), nbytes)
    out = _collect(res, A.nrows, val_dtype)
    out.ncols = A.nrows
    return out


def row_upper_bounds(A, B) -> np.ndarray:
    """ub_i = sum_{k in cols(A_i)} nnz(B_k) (int64), by its definition."""
    blen = np.diff(np.asarray(B.rp, dtype=np.int64))
    per_entry = blen[np.asarray(A.col, dtype=np.int64)]
    ub = np.zeros(A.nrows, dtype=np.int64)
    rows = np.repeat(np.arange(A.nrows), np.diff(np.asarray(A.rp, dtype=np.int64)))
    np.add.at(ub, rows, per_entry)
    return ub


def summa_blocks(M, row_cuts, col_cuts):
    """Block (I, J) of M: rows [row_cuts[I], row_cuts[I+1]) x cols [col_cuts[J], ...),
    column ids made local to the block.  Returns a nested list [I][J]."""
    rp = np.asarray(M.rp, dtype=np.int64)
    out = []
    for I in range(len(row_cuts) - 1):
        r0, r1 = int(row_cuts[I]), int(row_cuts[I + 1])
        rows = np.repeat(np.arange(r0, r1), np.diff(rp[r0:r1 + 1]))
        cols = np.asarray(M.col[rp[r0]:rp[r1]], dtype=np.int64)
        vals = None if M.val is None else M.val[rp[r0]:rp[r1]]
        line = []
        for J in range(len(col_cuts) - 1):
            c0, c1 = int(col_cuts[J]), int(col_cuts[J + 1])
            m = (cols >= c0) & (cols < c1)
            counts = np.bincount(rows[m] - r0, minlength=r1 - r0)
            brp = np.zeros(r1 - r0 + 1, dtype=np.int64)
            np.cumsum(counts, out=brp[1:])
            line.append(SimpleNamespace(nrows=r1 - r0, ncols=c1 - c0, rp=brp,
                                        col=(cols[m] - c0).astype(np.int32),
                                        val=None if vals is None else vals[m].copy(),
                                        nnz=int(brp[-1])))
        out.append(line)
    return out


def masked(sr, A, B, M):
    """(A (x).(+) B) on the pattern of M, by its definition: the full product,
    then the entries whose (i, j) is in M."""
    C = spgemm(sr, A, B)
    keep = np.zeros(C.nnz, dtype=bool)
    for i in range(C.nrows):
        a, b = int(C.rp[i]), int(C.rp[i + 1])
        m = np.asarray(M.col[int(M.rp[i]):int(M.rp[i + 1])])
        keep[a:b] = np.isin(C.col[a:b], m)
    rp = np.zeros(C.nrows + 1, dtype=np.int64)
    np.cumsum([int(keep[int(C.rp[i]):int(C.rp[i + 1])].sum()) for i in range(C.nrows)], out=rp[1:])
    return SimpleNamespace(nrows=C.nrows, ncols=C.ncols, rp=rp, col=C.col[keep],
                           val=None if C.val is None else C.val[keep], nnz=int(rp[-1]))
