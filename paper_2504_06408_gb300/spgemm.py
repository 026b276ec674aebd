"""Python binding of the C ABI in include/spgemm.h (argument marshalling only).

Every step of the multiplication runs in the CUDA library
``_build/libspgemm.so``; this module passes device pointers (from torch CUDA
tensors), sizes and the current CUDA stream.  There is no CPU fallback: if the
library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libspgemm.so")
# the same library built with -DSPG_CHECKS (inputs validated on the device
# before any product kernel, C's row pointers and ranks checked)
CHECKS_LIB_PATH = os.path.join(HERE, "_build_checks", "libspgemm_checks.so")

# semiring ids (spg_semiring)
PLUS_TIMES_F64, BOOL_OR_AND, MIN_PLUS_F32, OVERLAP_I32, PLUS_TIMES_I64, PLUS_TIMES_F32 = range(6)
SEMIRING_NAMES = {PLUS_TIMES_F64: "plus_times_f64", BOOL_OR_AND: "bool_or_and",
                  MIN_PLUS_F32: "min_plus_f32", OVERLAP_I32: "overlap_i32",
                  PLUS_TIMES_I64: "plus_times_i64", PLUS_TIMES_F32: "plus_times_f32"}
IN_NP = {PLUS_TIMES_F64: np.float64, BOOL_OR_AND: None, MIN_PLUS_F32: np.float32,
         OVERLAP_I32: np.int32, PLUS_TIMES_I64: np.int64, PLUS_TIMES_F32: np.float32}
OVERLAP_NP = np.dtype([("count", np.int32), ("a0", np.int32), ("b0", np.int32),
                       ("a1", np.int32), ("b1", np.int32)])
OUT_BYTES = {PLUS_TIMES_F64: 8, BOOL_OR_AND: 0, MIN_PLUS_F32: 4, OVERLAP_I32: 20,
             PLUS_TIMES_I64: 8, PLUS_TIMES_F32: 4}

STATUS = {0: "SPG_OK", 1: "SPG_ERR_INVALID_ARG", 2: "SPG_ERR_INVALID_CSR", 3: "SPG_ERR_OOM",
          4: "SPG_ERR_CUDA", 5: "SPG_ERR_UNSUPPORTED", 6: "SPG_ERR_OVERFLOW",
          8: "SPG_ERR_WORKSPACE"}


class SpgemmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class spg_csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class spg_tuning(ctypes.Structure):
    _fields_ = [("sym_warp_max_ub", ctypes.c_int64), ("sym_block_max_ub", ctypes.c_int64),
                ("num_warp_max_nnz", ctypes.c_int64), ("num_block_max_nnz", ctypes.c_int64),
                ("dense_slab_cols", ctypes.c_int64), ("sym_slab_cols", ctypes.c_int64),
                ("bitmap_cache_bytes", ctypes.c_int64), ("host_panel_bytes", ctypes.c_int64),
                ("deterministic", ctypes.c_int64), ("host_alloc_limit", ctypes.c_int64),
                ("rank_light_ub", ctypes.c_int64)]


class spg_stats(ctypes.Structure):
    _fields_ = [("products", ctypes.c_int64), ("nnz_c", ctypes.c_int64),
                ("rows_per_tier", ctypes.c_int64 * 4), ("launches", ctypes.c_int64),
                ("learned_rows", ctypes.c_int64), ("overflow_rows", ctypes.c_int64),
                ("staging_entries", ctypes.c_int64), ("learned_nnz", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 1)]


class spg_learned_opts(ctypes.Structure):
    _fields_ = [("model", ctypes.c_void_p), ("margin", ctypes.c_float),
                ("exact_max_ub", ctypes.c_int64), ("learned_max", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 4)]


MLP_PARAMS = 4545   # SPGEMM_MLP_PARAMS


# stage indices of spgemm_get_stage_times
STAGES = ["", "analysis", "sym_dense", "sym_block", "sym_warp", "scan", "num_binning",
          "slab_table", "num_dense", "num_block", "num_warp", "merge", "learned"]


_libs = {}
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_CSR = ctypes.POINTER(spg_csr)


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    sig = {
        "spgemm_create": [ctypes.POINTER(_P)],
        "spgemm_destroy": [_P],
        "spgemm_set_tuning": [_P, ctypes.POINTER(spg_tuning)],
        "spgemm_get_tuning": [_P, ctypes.POINTER(spg_tuning)],
        "spgemm_get_stats": [_P, ctypes.POINTER(spg_stats)],
        "spgemm_workspace_size": [_P, ctypes.c_int, _CSR, _CSR, ctypes.POINTER(ctypes.c_size_t)],
        "spgemm_symbolic": [_P, ctypes.c_int, _CSR, _CSR, _P, ctypes.POINTER(_I64), _P,
                            ctypes.c_size_t, _P],
        "spgemm_numeric": [_P, ctypes.c_int, _CSR, _CSR, _P, _P, _P, _P, ctypes.c_size_t, _P],
        "spgemm_check": [_P, _P, _P],
        "spgemm_validate_csr": [_P, _CSR, _P, ctypes.c_size_t, _P],
        "spgemm_transpose_workspace_size": [_P, _CSR, ctypes.POINTER(ctypes.c_size_t)],
        "spgemm_transpose": [_P, _CSR, ctypes.c_int, _P, _P, _P, _P, ctypes.c_size_t, _P],
        "spgemm_set_timing": [_P, ctypes.c_int],
        "spgemm_get_stage_times": [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int],
        "spgemm_host_symbolic": [_P, ctypes.c_int, _CSR, _CSR, _P, ctypes.POINTER(_I64)],
        "spgemm_host_numeric": [_P, ctypes.c_int, _P, _P],
        "spgemm_transpose_noalloc": [_CSR, ctypes.c_int, _P, _P, _P, _P],
        "spgemm_workspace_size_batched": [_P, ctypes.c_int, ctypes.c_int, _CSR, _CSR,
                                          ctypes.POINTER(ctypes.c_size_t)],
        "spgemm_symbolic_batched": [_P, ctypes.c_int, ctypes.c_int, _CSR, _CSR, _P, _P, _P,
                                    ctypes.c_size_t, _P],
        "spgemm_numeric_batched": [_P, ctypes.c_int, ctypes.c_int, _CSR, _CSR, _P, _P, _P, _P,
                                   ctypes.c_size_t, _P],
        "spgemm_merge_workspace_size": [_P, ctypes.c_int, ctypes.c_int, _P, _CSR,
                                        ctypes.POINTER(ctypes.c_size_t)],
        "spgemm_merge_stages": [_P, ctypes.c_int, ctypes.c_int, _CSR, _P, ctypes.POINTER(_I64),
                                _P, _P, _P, ctypes.c_size_t, _P],
        "spgemm_merge_stages_batched": [_P, ctypes.c_int, ctypes.c_int, _P, _CSR, _P, _P, _P, _P,
                                        _P, ctypes.c_size_t, _P],
        "spgemm_split_workspace_size": [_P, _CSR, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
        "spgemm_split_columns": [_P, _CSR, ctypes.c_int, _P, ctypes.c_int, _P, _P, _P, _P, _P,
                                 ctypes.c_size_t, _P],
        "spgemm_learned_workspace_size": [_P, ctypes.c_int, _CSR, _CSR,
                                          ctypes.POINTER(ctypes.c_size_t)],
        "spgemm_learned_plan": [_P, ctypes.c_int, _CSR, _CSR, ctypes.POINTER(spg_learned_opts),
                                _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), _P],
        "spgemm_learned_symbolic": [_P, ctypes.c_int, _CSR, _CSR, _P, ctypes.POINTER(_I64), _P,
                                    ctypes.c_size_t, _P, ctypes.c_size_t, _P],
        "spgemm_learned_numeric": [_P, ctypes.c_int, _CSR, _CSR, _P, _P, _P, _P, ctypes.c_size_t,
                                   _P, ctypes.c_size_t, _P],
        "spgemm_row_features": [_P, _CSR, _CSR, _P, _P, _P, ctypes.c_size_t, _P],
        "spgemm_mlp_forward": [_P, _P, _I64, _P, _P, _P],
        "spgemm_mlp_grad": [_P, _P, _P, _I64, ctypes.c_float, _P, _P, _P, _P, ctypes.c_size_t,
                            _P],
        "spgemm_mlp_adam": [_P, _P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_int, _P],
        "spgemm_mlp_to_bf16": [_P, _P, _P, _P],
        "spgemm_masked_workspace_size": [_P, ctypes.c_int, _CSR, _CSR, _CSR,
                                         ctypes.POINTER(ctypes.c_size_t)],
        "spgemm_masked_symbolic": [_P, ctypes.c_int, _CSR, _CSR, _CSR, _P, ctypes.POINTER(_I64),
                                   _P, ctypes.c_size_t, _P],
        "spgemm_masked_numeric": [_P, ctypes.c_int, _CSR, _CSR, _CSR, _P, _P, _P, _P,
                                  ctypes.c_size_t, _P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.spgemm_last_error.argtypes = [_P]
    lib.spgemm_last_error.restype = ctypes.c_char_p
    lib.spgemm_mlp_train_workspace_size.argtypes = [_I64]
    lib.spgemm_mlp_train_workspace_size.restype = ctypes.c_size_t
    _libs[path] = lib
    return lib


def exported_symbols() -> list[str]:
    return ["spgemm_create", "spgemm_destroy", "spgemm_last_error", "spgemm_set_tuning",
            "spgemm_get_tuning", "spgemm_get_stats", "spgemm_workspace_size", "spgemm_symbolic",
            "spgemm_numeric", "spgemm_check", "spgemm_validate_csr",
            "spgemm_transpose_workspace_size", "spgemm_transpose", "spgemm_set_timing",
            "spgemm_get_stage_times", "spgemm_host_symbolic", "spgemm_host_numeric",
            "spgemm_transpose_noalloc", "spgemm_workspace_size_batched",
            "spgemm_symbolic_batched", "spgemm_numeric_batched", "spgemm_merge_workspace_size",
            "spgemm_merge_stages", "spgemm_merge_stages_batched", "spgemm_split_workspace_size",
            "spgemm_split_columns", "spgemm_learned_workspace_size", "spgemm_learned_plan",
            "spgemm_learned_symbolic", "spgemm_learned_numeric", "spgemm_row_features",
            "spgemm_mlp_forward", "spgemm_mlp_train_workspace_size", "spgemm_mlp_grad",
            "spgemm_mlp_adam", "spgemm_mlp_to_bf16", "spgemm_masked_workspace_size",
            "spgemm_masked_symbolic", "spgemm_masked_numeric"]


@dataclass
class DeviceCSR:
    """CSR matrix in device memory (torch CUDA tensors): int64 rp, int32 col."""
    nrows: int
    ncols: int
    rp: "object"
    col: "object"
    val: "Optional[object]" = None
    _nnz: "Optional[int]" = None   # entries of a row view (col/val are shared)

    @property
    def nnz(self) -> int:
        return int(self.col.numel()) if self._nnz is None else self._nnz

    def rows(self, r0: int, r1: int) -> "DeviceCSR":
        """Row view [r0, r1): row pointers offset, same column/value arrays
        (the kernels address entries by the absolute offsets in row_ptr)."""
        return DeviceCSR(r1 - r0, self.ncols, self.rp[r0:r1 + 1], self.col, self.val,
                         _nnz=int((self.rp[r1] - self.rp[r0]).item()) if r1 > r0 else 0)

    def c(self) -> spg_csr:
        return spg_csr(self.nrows, self.ncols, self.nnz, self.rp.data_ptr(),
                       self.col.data_ptr() if self.col.numel() else None,
                       None if self.val is None or self.val.numel() == 0 else self.val.data_ptr())

    @staticmethod
    def from_host(M, device="cuda", val_dtype=None) -> "DeviceCSR":
        import torch
        rp = torch.from_numpy(np.ascontiguousarray(M.rp, dtype=np.int64)).to(device)
        col = torch.from_numpy(np.ascontiguousarray(M.col, dtype=np.int32)).to(device)
        val = None
        if M.val is not None and val_dtype is not None:
            val = torch.from_numpy(np.ascontiguousarray(M.val, dtype=val_dtype)).to(device)
        return DeviceCSR(int(M.nrows), int(M.ncols), rp, col, val)


def _stream_ptr(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Handle:
    """spg_handle wrapper; one per thread, reusable across calls."""

    def __init__(self, tuning: Optional[dict] = None, lib_path: Optional[str] = None):
        self.lib = load_library(lib_path or LIB_PATH)
        self._h = ctypes.c_void_p()
        self._ok(self.lib.spgemm_create(ctypes.byref(self._h)))
        if tuning:
            self.set_tuning(**tuning)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and self.lib is not None:
            self.lib.spgemm_destroy(h)
            self._h = None

    def _ok(self, st: int):
        if st != 0:
            msg = self.lib.spgemm_last_error(self._h).decode() if getattr(self, "_h", None) else ""
            raise SpgemmError(st, msg)

    def set_tuning(self, **kw):
        """Set spg_tuning fields by name (0 = library default); an unknown
        name raises instead of being ignored."""
        t = spg_tuning()
        known = {name for name, _ in spg_tuning._fields_}
        for k, v in kw.items():
            if k not in known or k == "reserved":
                raise ValueError(f"unknown tuning field {k!r} (known: {sorted(known - {'reserved'})})")
            setattr(t, k, int(v))
        self._ok(self.lib.spgemm_set_tuning(self._h, ctypes.byref(t)))

    def stats(self) -> dict:
        s = spg_stats()
        self._ok(self.lib.spgemm_get_stats(self._h, ctypes.byref(s)))
        return {"products": s.products, "nnz_c": s.nnz_c,
                "rows_per_tier": list(s.rows_per_tier), "launches": s.launches,
                "learned_rows": s.learned_rows, "overflow_rows": s.overflow_rows,
                "staging_entries": s.staging_entries, "learned_nnz": s.learned_nnz}

    def set_timing(self, enable: bool = True):
        self._ok(self.lib.spgemm_set_timing(self._h, 1 if enable else 0))

    def stage_times(self) -> dict:
        """Milliseconds per stage of the last symbolic or numeric call."""
        buf = (ctypes.c_float * len(STAGES))()
        self._ok(self.lib.spgemm_get_stage_times(self._h, buf, len(STAGES)))
        return {name: buf[i] for i, name in enumerate(STAGES) if name}

    def host_multiply(self, sr: int, A, B, out=None):
        """C = A (x).(+) B for HOST matrices (numpy arrays, ideally pinned torch
        tensors' numpy views).  ``out`` = optional dict of preallocated host arrays
        {"rp", "col", "val"} large enough for C.  Returns (rp, col, val, nnz)."""
        def host_csr(M):
            vb = IN_NP[sr]
            val = None if vb is None else np.ascontiguousarray(M.val, dtype=vb)
            rp = np.ascontiguousarray(M.rp, dtype=np.int64)
            col = np.ascontiguousarray(M.col, dtype=np.int32)
            return spg_csr(M.nrows, M.ncols, col.size, rp.ctypes.data,
                           col.ctypes.data if col.size else None,
                           None if val is None or val.size == 0 else val.ctypes.data), (rp, col, val)
        a, ka = host_csr(A)
        b, kb = (a, ka) if B is A else host_csr(B)
        rp = out["rp"] if out else np.empty(A.nrows + 1, dtype=np.int64)
        nnz = ctypes.c_int64()
        self._ok(self.lib.spgemm_host_symbolic(self._h, sr, ctypes.byref(a), ctypes.byref(b),
                                               rp.ctypes.data, ctypes.byref(nnz)))
        n = nnz.value
        if out:
            col, val = out["col"], out.get("val")
        else:
            col = np.empty(n, dtype=np.int32)
            val = None if OUT_BYTES[sr] == 0 else np.empty(n * OUT_BYTES[sr], dtype=np.uint8)
        self._ok(self.lib.spgemm_host_numeric(self._h, sr, col.ctypes.data if n else None,
                                              None if val is None or n == 0 else val.ctypes.data))
        return rp, col, val, n

    def workspace_size(self, sr: int, A: DeviceCSR, B: DeviceCSR) -> int:
        n = ctypes.c_size_t()
        a, b = A.c(), B.c()
        self._ok(self.lib.spgemm_workspace_size(self._h, sr, ctypes.byref(a), ctypes.byref(b),
                                                ctypes.byref(n)))
        return n.value

    def symbolic(self, sr, A: DeviceCSR, B: DeviceCSR, c_rp, ws, stream=None) -> int:
        nnz = ctypes.c_int64()
        a, b = A.c(), B.c()
        self._ok(self.lib.spgemm_symbolic(self._h, sr, ctypes.byref(a), ctypes.byref(b),
                                          c_rp.data_ptr(), ctypes.byref(nnz), ws.data_ptr(),
                                          ws.numel(), _stream_ptr(stream)))
        return nnz.value

    def numeric(self, sr, A: DeviceCSR, B: DeviceCSR, c_rp, c_col, c_val, ws, stream=None):
        a, b = A.c(), B.c()
        self._ok(self.lib.spgemm_numeric(
            self._h, sr, ctypes.byref(a), ctypes.byref(b), c_rp.data_ptr(),
            c_col.data_ptr() if c_col.numel() else None,
            None if c_val is None or c_val.numel() == 0 else c_val.data_ptr(),
            ws.data_ptr(), ws.numel(), _stream_ptr(stream)))

    def check(self, ws, stream=None):
        self._ok(self.lib.spgemm_check(self._h, ws.data_ptr(), _stream_ptr(stream)))

    def transpose(self, A: DeviceCSR, value_bytes: int, stream=None) -> DeviceCSR:
        """A^T on the GPU (values carried as raw bytes of the given width)."""
        import torch
        a = A.c()
        n = ctypes.c_size_t()
        self._ok(self.lib.spgemm_transpose_workspace_size(self._h, ctypes.byref(a),
                                                          ctypes.byref(n)))
        dev = A.rp.device
        ws = torch.empty(max(n.value, 1), dtype=torch.uint8, device=dev)
        t_rp = torch.empty(A.ncols + 1, dtype=torch.int64, device=dev)
        t_col = torch.empty(A.nnz, dtype=torch.int32, device=dev)
        t_val = None
        if value_bytes:
            t_val = torch.empty(A.nnz * value_bytes, dtype=torch.uint8, device=dev)
            if A.val is not None:
                t_val = t_val.view(A.val.dtype).reshape((-1,) + tuple(A.val.shape[1:]))
        self._ok(self.lib.spgemm_transpose(
            self._h, ctypes.byref(a), value_bytes, t_rp.data_ptr(),
            t_col.data_ptr() if A.nnz else None,
            t_val.data_ptr() if t_val is not None and A.nnz else None,
            ws.data_ptr(), ws.numel(), _stream_ptr(stream)))
        return DeviceCSR(A.ncols, A.nrows, t_rp, t_col, t_val)

    # ---- batched products, merges, splits -------------------------------------

    @staticmethod
    def _ptrs(tensors):
        arr = (ctypes.c_void_p * len(tensors))()
        for i, t in enumerate(tensors):
            arr[i] = None if t is None or t.numel() == 0 else t.data_ptr()
        return arr

    def workspace_size_batched(self, sr, As, Bs) -> int:
        a = (spg_csr * len(As))(*[x.c() for x in As])
        b = (spg_csr * len(Bs))(*[x.c() for x in Bs])
        n = ctypes.c_size_t()
        self._ok(self.lib.spgemm_workspace_size_batched(self._h, sr, len(As), a, b,
                                                        ctypes.byref(n)))
        return n.value

    def symbolic_batched(self, sr, As, Bs, c_rps, ws, stream=None, sync=True):
        """Batched symbolic phase; returns nnz(C_p) per product.  sync=False
        passes no host count array: nothing is copied back or synchronised
        (returns None), e.g. inside a CUDA-graph capture."""
        a = (spg_csr * len(As))(*[x.c() for x in As])
        b = (spg_csr * len(Bs))(*[x.c() for x in Bs])
        nnz = (ctypes.c_int64 * len(As))() if sync else None
        self._ok(self.lib.spgemm_symbolic_batched(self._h, sr, len(As), a, b, self._ptrs(c_rps),
                                                  nnz, ws.data_ptr(), ws.numel(),
                                                  _stream_ptr(stream)))
        return list(nnz) if sync else None

    def numeric_batched(self, sr, As, Bs, c_rps, c_cols, c_vals, ws, stream=None):
        a = (spg_csr * len(As))(*[x.c() for x in As])
        b = (spg_csr * len(Bs))(*[x.c() for x in Bs])
        self._ok(self.lib.spgemm_numeric_batched(
            self._h, sr, len(As), a, b, self._ptrs(c_rps), self._ptrs(c_cols),
            self._ptrs(c_vals) if c_vals is not None else None, ws.data_ptr(), ws.numel(),
            _stream_ptr(stream)))

    def merge_workspace_size(self, sr, groups) -> int:
        flat = [p for g in groups for p in g]
        parts = (spg_csr * len(flat))(*[p.c() for p in flat])
        npart = (ctypes.c_int * len(groups))(*[len(g) for g in groups])
        n = ctypes.c_size_t()
        self._ok(self.lib.spgemm_merge_workspace_size(self._h, sr, len(groups), npart, parts,
                                                      ctypes.byref(n)))
        return n.value

    def merge_count(self, sr, groups, c_rps, ws, stream=None, sync=True):
        """Row pointers of the merged C blocks; returns their nnz (None with
        sync=False: no host copy, no synchronisation)."""
        flat = [p for g in groups for p in g]
        parts = (spg_csr * len(flat))(*[p.c() for p in flat])
        npart = (ctypes.c_int * len(groups))(*[len(g) for g in groups])
        nnz = (ctypes.c_int64 * len(groups))() if sync else None
        self._ok(self.lib.spgemm_merge_stages_batched(
            self._h, sr, len(groups), npart, parts, self._ptrs(c_rps), nnz, None, None,
            ws.data_ptr(), ws.numel(), _stream_ptr(stream)))
        return list(nnz) if sync else None

    def merge_write(self, sr, groups, c_rps, c_cols, c_vals, ws, stream=None):
        flat = [p for g in groups for p in g]
        parts = (spg_csr * len(flat))(*[p.c() for p in flat])
        npart = (ctypes.c_int * len(groups))(*[len(g) for g in groups])
        self._ok(self.lib.spgemm_merge_stages_batched(
            self._h, sr, len(groups), npart, parts, self._ptrs(c_rps), None, self._ptrs(c_cols),
            self._ptrs(c_vals) if c_vals is not None else None, ws.data_ptr(), ws.numel(),
            _stream_ptr(stream)))

    def split_columns(self, M: DeviceCSR, cuts, value_bytes: int, stream=None):
        """Column parts of M (local column ids); returns a list of DeviceCSR."""
        import torch
        nparts = len(cuts) - 1
        m = M.c()
        n = ctypes.c_size_t()
        self._ok(self.lib.spgemm_split_workspace_size(self._h, ctypes.byref(m), nparts,
                                                      ctypes.byref(n)))
        dev = M.rp.device
        ws = torch.empty(max(n.value, 1), dtype=torch.uint8, device=dev)
        prp = torch.empty(nparts * (M.nrows + 1), dtype=torch.int64, device=dev)
        pcol = torch.empty(max(M.nnz, 1), dtype=torch.int32, device=dev)
        pval = None
        if value_bytes:
            pval = torch.empty(max(M.nnz, 1) * value_bytes, dtype=torch.uint8, device=dev)
        cuts_arr = (ctypes.c_int32 * len(cuts))(*[int(c) for c in cuts])
        pnnz = (ctypes.c_int64 * nparts)()
        self._ok(self.lib.spgemm_split_columns(
            self._h, ctypes.byref(m), nparts, cuts_arr, value_bytes, prp.data_ptr(),
            pcol.data_ptr(), None if pval is None else pval.data_ptr(), pnnz, ws.data_ptr(),
            ws.numel(), _stream_ptr(stream)))
        out, base = [], 0
        for p in range(nparts):
            k = int(pnnz[p])
            rp = prp[p * (M.nrows + 1):(p + 1) * (M.nrows + 1)]
            col = pcol[base:base + k]
            val = None
            if pval is not None:
                val = pval[base * value_bytes:(base + k) * value_bytes]
                if M.val is not None:
                    val = val.view(M.val.dtype)
                    if M.val.dim() > 1:
                        val = val.reshape((-1,) + tuple(M.val.shape[1:]))
            out.append(DeviceCSR(M.nrows, int(cuts[p + 1] - cuts[p]), rp, col, val))
            base += k
        return out

    # ---- learned output sizing ----------------------------------------------------

    def learned_workspace_size(self, sr, A: DeviceCSR, B: DeviceCSR) -> int:
        n = ctypes.c_size_t()
        a, b = A.c(), B.c()
        self._ok(self.lib.spgemm_learned_workspace_size(self._h, sr, ctypes.byref(a),
                                                        ctypes.byref(b), ctypes.byref(n)))
        return n.value

    def learned_plan(self, sr, A: DeviceCSR, B: DeviceCSR, ws, model=None, margin=0.0,
                     exact_max_ub=0, learned_max=0, stream=None) -> int:
        """Step 1 of the learned path; returns the staging bytes steps 2-3 need.
        model: device BF16 parameters (torch tensor of MLP_PARAMS) or None."""
        o = spg_learned_opts()
        o.model = None if model is None else model.data_ptr()
        o.margin = float(margin)
        o.exact_max_ub = int(exact_max_ub)
        o.learned_max = int(learned_max)
        n = ctypes.c_size_t()
        a, b = A.c(), B.c()
        self._ok(self.lib.spgemm_learned_plan(self._h, sr, ctypes.byref(a), ctypes.byref(b),
                                              ctypes.byref(o), ws.data_ptr(), ws.numel(),
                                              ctypes.byref(n), _stream_ptr(stream)))
        return n.value

    def learned_symbolic(self, sr, A, B, c_rp, ws, staging, stream=None) -> int:
        nnz = ctypes.c_int64()
        a, b = A.c(), B.c()
        self._ok(self.lib.spgemm_learned_symbolic(
            self._h, sr, ctypes.byref(a), ctypes.byref(b), c_rp.data_ptr(), ctypes.byref(nnz),
            ws.data_ptr(), ws.numel(), None if staging is None or staging.numel() == 0
            else staging.data_ptr(), 0 if staging is None else staging.numel(),
            _stream_ptr(stream)))
        return nnz.value

    def learned_numeric(self, sr, A, B, c_rp, c_col, c_val, ws, staging, stream=None):
        a, b = A.c(), B.c()
        self._ok(self.lib.spgemm_learned_numeric(
            self._h, sr, ctypes.byref(a), ctypes.byref(b), c_rp.data_ptr(),
            c_col.data_ptr() if c_col.numel() else None,
            None if c_val is None or c_val.numel() == 0 else c_val.data_ptr(),
            ws.data_ptr(), ws.numel(), None if staging is None or staging.numel() == 0
            else staging.data_ptr(), 0 if staging is None else staging.numel(),
            _stream_ptr(stream)))

    def row_features(self, A: DeviceCSR, B: DeviceCSR, ws, stream=None):
        """(feat [n, 4] float32, ub [n] int64) device tensors."""
        import torch
        dev = A.rp.device
        feat = torch.empty((A.nrows, 4), dtype=torch.float32, device=dev)
        ub = torch.empty(A.nrows, dtype=torch.int64, device=dev)
        a, b = A.c(), B.c()
        self._ok(self.lib.spgemm_row_features(self._h, ctypes.byref(a), ctypes.byref(b),
                                              feat.data_ptr() if A.nrows else None,
                                              ub.data_ptr() if A.nrows else None,
                                              ws.data_ptr(), ws.numel(), _stream_ptr(stream)))
        return feat, ub

    def mlp_forward(self, feat, params_bf16, stream=None):
        import torch
        n = int(feat.shape[0])
        z = torch.empty(n, dtype=torch.float32, device=feat.device)
        self._ok(self.lib.spgemm_mlp_forward(self._h, feat.data_ptr() if n else None, n,
                                             params_bf16.data_ptr(), z.data_ptr() if n else None,
                                             _stream_ptr(stream)))
        return z

    def mlp_grad(self, feat, log_target, tau, params_bf16, ws=None, stream=None):
        """(grad [MLP_PARAMS] float32, loss [1] float32) device tensors."""
        import torch
        n = int(feat.shape[0])
        need = self.lib.spgemm_mlp_train_workspace_size(n)
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=feat.device)
        grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=feat.device)
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        self._ok(self.lib.spgemm_mlp_grad(self._h, feat.data_ptr(), log_target.data_ptr(), n,
                                          float(tau), params_bf16.data_ptr(), grad.data_ptr(),
                                          loss.data_ptr(), ws.data_ptr(), ws.numel(),
                                          _stream_ptr(stream)))
        return grad, loss

    def mlp_train_workspace_size(self, n: int) -> int:
        return int(self.lib.spgemm_mlp_train_workspace_size(int(n)))

    def mlp_adam(self, master, m, v, grad, params_bf16, lr, step, stream=None):
        self._ok(self.lib.spgemm_mlp_adam(self._h, master.data_ptr(), m.data_ptr(), v.data_ptr(),
                                          grad.data_ptr(), params_bf16.data_ptr(), float(lr),
                                          int(step), _stream_ptr(stream)))

    def mlp_to_bf16(self, master, params_bf16, stream=None):
        self._ok(self.lib.spgemm_mlp_to_bf16(self._h, master.data_ptr(), params_bf16.data_ptr(),
                                             _stream_ptr(stream)))

    def validate(self, M: DeviceCSR, ws, stream=None):
        m = M.c()
        self._ok(self.lib.spgemm_validate_csr(self._h, ctypes.byref(m), ws.data_ptr(),
                                              ws.numel(), _stream_ptr(stream)))


def out_tensor(sr: int, nnz: int, device="cuda"):
    import torch
    if sr == BOOL_OR_AND:
        return None
    if sr == OVERLAP_I32:
        return torch.empty((nnz, 5), dtype=torch.int32, device=device)
    dt = {PLUS_TIMES_F64: torch.float64, MIN_PLUS_F32: torch.float32,
          PLUS_TIMES_I64: torch.int64, PLUS_TIMES_F32: torch.float32}[sr]
    return torch.empty(nnz, dtype=dt, device=device)


def spgemm(sr: int, A: DeviceCSR, B: DeviceCSR, handle: Optional[Handle] = None,
           ws=None, check: bool = True) -> DeviceCSR:
    """C = A (x).(+) B on the GPU (symbolic, allocation of C, numeric)."""
    import torch
    h = handle or Handle()
    dev = A.rp.device
    if ws is None:
        ws = torch.empty(h.workspace_size(sr, A, B), dtype=torch.uint8, device=dev)
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device=dev)
    nnz = h.symbolic(sr, A, B, c_rp, ws)
    c_col = torch.empty(nnz, dtype=torch.int32, device=dev)
    c_val = out_tensor(sr, nnz, dev)
    h.numeric(sr, A, B, c_rp, c_col, c_val, ws)
    if check:
        h.check(ws)
    return DeviceCSR(A.nrows, B.ncols, c_rp, c_col, c_val)


def learned_spgemm(sr: int, A: DeviceCSR, B: DeviceCSR, model=None, margin: float = 0.0,
                   handle: Optional[Handle] = None, check: bool = True, **opts) -> DeviceCSR:
    """C = A (x).(+) B through the learned-sizing path (plan, direct + exact
    symbolic, numeric).  model: device BF16 parameters or None (ub-sized)."""
    import torch
    h = handle or Handle()
    dev = A.rp.device
    ws = torch.empty(h.learned_workspace_size(sr, A, B), dtype=torch.uint8, device=dev)
    sb = h.learned_plan(sr, A, B, ws, model=model, margin=margin, **opts)
    staging = torch.empty(max(sb, 1), dtype=torch.uint8, device=dev)
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device=dev)
    nnz = h.learned_symbolic(sr, A, B, c_rp, ws, staging)
    c_col = torch.empty(nnz, dtype=torch.int32, device=dev)
    c_val = out_tensor(sr, nnz, dev)
    h.learned_numeric(sr, A, B, c_rp, c_col, c_val, ws, staging)
    if check:
        h.check(ws)
    return DeviceCSR(A.nrows, B.ncols, c_rp, c_col, c_val)


def masked_spgemm(sr: int, A: DeviceCSR, B: DeviceCSR, M: DeviceCSR,
                  handle: Optional[Handle] = None, check: bool = True) -> DeviceCSR:
    """C = (A (x).(+) B) on the pattern of M (masked product, on the GPU)."""
    import torch
    h = handle or Handle()
    dev = A.rp.device
    a, b, m = A.c(), B.c(), M.c()
    n = ctypes.c_size_t()
    h._ok(h.lib.spgemm_masked_workspace_size(h._h, sr, ctypes.byref(a), ctypes.byref(b),
                                             ctypes.byref(m), ctypes.byref(n)))
    ws = torch.empty(max(n.value, 1), dtype=torch.uint8, device=dev)
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device=dev)
    nnz = ctypes.c_int64()
    h._ok(h.lib.spgemm_masked_symbolic(h._h, sr, ctypes.byref(a), ctypes.byref(b),
                                       ctypes.byref(m), c_rp.data_ptr(), ctypes.byref(nnz),
                                       ws.data_ptr(), ws.numel(), _stream_ptr()))
    c_col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=dev)
    c_val = out_tensor(sr, max(nnz.value, 1), dev)
    h._ok(h.lib.spgemm_masked_numeric(
        h._h, sr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(m), c_rp.data_ptr(),
        c_col.data_ptr(), None if c_val is None else c_val.data_ptr(), ws.data_ptr(), ws.numel(),
        _stream_ptr()))
    if check:
        h.check(ws)
    k = nnz.value
    return DeviceCSR(A.nrows, B.ncols, c_rp, c_col[:k], None if c_val is None else c_val[:k])


def typed_out(sr: int, raw):
    """View a raw uint8 device buffer as the semiring's output values."""
    import torch
    if raw is None or sr == BOOL_OR_AND:
        return None
    if sr == OVERLAP_I32:
        return raw.view(torch.int32).reshape(-1, 5)
    dt = {PLUS_TIMES_F64: torch.float64, MIN_PLUS_F32: torch.float32,
          PLUS_TIMES_I64: torch.int64, PLUS_TIMES_F32: torch.float32}[sr]
    return raw.view(dt)


def panel_cuts(rp, nrows: int, cap_entries: int):
    """Row cuts [0, ..., nrows] of panels of at most cap_entries output
    entries each (a single row may exceed it)."""
    cuts, r0 = [0], 0
    while r0 < nrows:
        r1 = int(np.searchsorted(rp, rp[r0] + cap_entries, side="right")) - 1
        r1 = max(r1, r0 + 1)
        r1 = min(r1, nrows)
        cuts.append(r1)
        r0 = r1
    return cuts


def panel_product(sr: int, A: DeviceCSR, B: DeviceCSR, budget_bytes: int, on_panel,
                  handle: Optional[Handle] = None, learned: Optional[dict] = None,
                  stats: Optional[dict] = None):
    """C = A (x).(+) B in row panels whose output fits in budget_bytes of device
    memory (for products larger than HBM).  One symbolic call on all of A gives
    the row counts; each panel (a row view of A) then runs symbolic + numeric
    into a reused buffer and on_panel(r0, r1, C_panel) is called.

    learned: None for the plain form, else the options of the learned-sizing
    path ({} for ub-sized capacities, or model / margin / exact_max_ub /
    learned_max): each panel then runs learned plan, symbolic and numeric.
    stats: if given, filled with the device milliseconds of each panel's
    compute ("panel_ms", CUDA events around the library calls only) and the
    cuts.  Returns (nnz(C), number of panels)."""
    import torch
    h = handle or Handle()
    dev = A.rp.device
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device=dev)
    ws = torch.empty(h.workspace_size(sr, A, B), dtype=torch.uint8, device=dev)
    total = h.symbolic(sr, A, B, c_rp, ws)
    del ws
    per = 4 + OUT_BYTES[sr]
    cap = max(1, budget_bytes // per)
    rp = c_rp.cpu().numpy()
    cuts = panel_cuts(rp, A.nrows, cap)
    biggest = max(int(rp[b] - rp[a]) for a, b in zip(cuts[:-1], cuts[1:]))
    col = torch.empty(max(biggest, 1), dtype=torch.int32, device=dev)
    val = out_tensor(sr, max(biggest, 1), dev)
    times = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        Av = A.rows(a, b) if (a, b) != (0, A.nrows) else A
        prp = torch.empty(b - a + 1, dtype=torch.int64, device=dev)
        if learned is None:
            wsp = torch.empty(h.workspace_size(sr, Av, B), dtype=torch.uint8, device=dev)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            n = h.symbolic(sr, Av, B, prp, wsp)
            h.numeric(sr, Av, B, prp, col, val, wsp)
            e1.record()
        else:
            wsp = torch.empty(h.learned_workspace_size(sr, Av, B), dtype=torch.uint8, device=dev)
            sb = h.learned_plan(sr, Av, B, wsp, **learned)
            staging = torch.empty(max(sb, 1), dtype=torch.uint8, device=dev)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            h.learned_plan(sr, Av, B, wsp, **learned)
            n = h.learned_symbolic(sr, Av, B, prp, wsp, staging)
            h.learned_numeric(sr, Av, B, prp, col, val, wsp, staging)
            e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        h.check(wsp)
        on_panel(a, b, DeviceCSR(b - a, B.ncols, prp, col[:n], None if val is None else val[:n]))
        del wsp
        if learned is not None:
            del staging
    if stats is not None:
        stats["panel_ms"] = times
        stats["cuts"] = cuts
    return total, len(cuts) - 1


def to_host_rows(C: DeviceCSR, sr: int, rows):
    """Rows `rows` (ascending) of a device result copied to numpy as one CSR."""
    from types import SimpleNamespace
    rp = C.rp.cpu().numpy()
    rows = np.asarray(rows, dtype=np.int64)
    lens = rp[rows + 1] - rp[rows]
    orp = np.zeros(rows.size + 1, dtype=np.int64)
    np.cumsum(lens, out=orp[1:])
    cols, vals = [], []
    for r in rows:
        a, b = int(rp[r]), int(rp[r + 1])
        cols.append(C.col[a:b].cpu().numpy())
        if C.val is not None:
            v = C.val[a:b].cpu().numpy()
            vals.append(v.view(OVERLAP_NP).reshape(-1) if sr == OVERLAP_I32 else v)
    col = np.concatenate(cols) if cols else np.zeros(0, np.int32)
    val = (np.concatenate(vals) if vals else None) if C.val is not None else None
    return SimpleNamespace(nrows=rows.size, ncols=C.ncols, rp=orp, col=col, val=val,
                           nnz=int(orp[-1]))


def to_host(C: DeviceCSR, sr: int):
    """Copy a device result to numpy (rp, col, val) with the semiring's dtypes."""
    from types import SimpleNamespace
    rp = C.rp.cpu().numpy()
    col = C.col.cpu().numpy()
    val = None
    if C.val is not None:
        v = C.val.cpu().numpy()
        val = v.view(OVERLAP_NP).reshape(-1) if sr == OVERLAP_I32 else v
    return SimpleNamespace(nrows=C.nrows, ncols=C.ncols, rp=rp, col=col, val=val, nnz=col.size)
