"""Sparse SUMMA on one GPU: the block-grid emulation of the paper's distributed
multiply (Section 2.1, Fig. "2.5D" for the grid; merge of stage partials:
Section 3.4).

A q x q process grid owns block (I, J) of C.  At stage s, block A(I, s) is
broadcast along grid row I and B(s, J) along grid column J, and every grid
point multiplies them; C(I, J) is the (+)-merge of its q stage partials.
Here the q^3 block products of all stages are one batched call (one
persistent launch per kernel tier over every block's rows, heaviest first),
and the q^2 merges are one batched merge call.  The numeric phase and the
merge can be captured once into a CUDA graph and replayed.

Blocks are views: A's columns are split into the stage ranges and B's into
the q column ranges (spgemm_split_columns, on the GPU); block (I, s) is the
row range I of column part s (row views need no copy).

The 2.5D variant (Section 2.1's 2.5D grid: each stage split in halves, whose
partials are merged like stages) is the same driver with 2q stages
(`stages=2 * q`): q^2 x 2q block products and merges of 2q partials.

This module only orders library calls and allocates their buffers with
torch; every step runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import spgemm as api


def even_cuts(n: int, q: int) -> List[int]:
    return [(n * t) // q for t in range(q + 1)]


@dataclass
class Block:
    I: int
    J: int
    s: int


class Summa:
    """C = A (x).(+) B emulated on a q x q Sparse-SUMMA grid.

    row_cuts split A's rows (grid rows), inner_cuts split the inner dimension
    (stages; without inner_cuts, `stages` even ones, default q), col_cuts split
    B's columns (grid columns); defaults are even.
    batched=False runs one library call per block product and per merge (the
    plain form); batched=True one call for all of them.

    A symbolic call leaves state in its workspace that its numeric call reads,
    so the plain form gives every block product its own workspace, from a
    handle whose symbolic bitmap cache is split between the blocks
    (unbatched_cache_bytes in total; `tuning` = the other tier limits of that
    handle).
    """

    def __init__(self, handle: api.Handle, sr: int, A: api.DeviceCSR, B: api.DeviceCSR,
                 q: int = 4, row_cuts=None, inner_cuts=None, col_cuts=None, stages=None,
                 batched: bool = True, unbatched_cache_bytes: int = 4 << 30,
                 tuning: Optional[dict] = None):
        import torch
        self.h, self.sr, self.q, self.batched = handle, sr, q, batched
        self.A, self.B = A, B
        self.row_cuts = list(row_cuts or even_cuts(A.nrows, q))
        self.inner_cuts = list(inner_cuts or even_cuts(A.ncols, stages or q))
        self.stages = len(self.inner_cuts) - 1
        self.col_cuts = list(col_cuts or even_cuts(B.ncols, q))
        vb = api.IN_NP[sr] and np.dtype(api.IN_NP[sr]).itemsize or 0
        self.vb = vb
        self.Ap = handle.split_columns(A, self.inner_cuts, vb)   # stage parts of A
        self.Bp = handle.split_columns(B, self.col_cuts, vb)     # column parts of B
        self.blocks = [Block(I, J, s) for s in range(self.stages) for I in range(q)
                       for J in range(q)]
        self.As = [self.Ap[b.s].rows(self.row_cuts[b.I], self.row_cuts[b.I + 1]) for b in self.blocks]
        self.Bs = [self.Bp[b.J].rows(self.inner_cuts[b.s], self.inner_cuts[b.s + 1])
                   for b in self.blocks]
        self.dev = A.rp.device
        self._torch = torch
        self.graph = None
        if not batched:
            per = max(unbatched_cache_bytes // len(self.blocks), 1 << 20)
            self.hb = api.Handle(tuning=dict(tuning or {}, bitmap_cache_bytes=per))

    # ---- phase 1: block products -------------------------------------------------

    def symbolic(self):
        torch = self._torch
        self.p_rp = [torch.empty(a.nrows + 1, dtype=torch.int64, device=self.dev) for a in self.As]
        if self.batched:
            self.ws = torch.empty(self.h.workspace_size_batched(self.sr, self.As, self.Bs),
                                  dtype=torch.uint8, device=self.dev)
            self.p_nnz = self.h.symbolic_batched(self.sr, self.As, self.Bs, self.p_rp, self.ws)
        else:
            self.ws_list = [torch.empty(max(self.hb.workspace_size(self.sr, a, b), 1),
                                        dtype=torch.uint8, device=self.dev)
                            for a, b in zip(self.As, self.Bs)]
            self.ws = self.ws_list[0]
            self.p_nnz = [self.hb.symbolic(self.sr, a, b, rp, w)
                          for a, b, rp, w in zip(self.As, self.Bs, self.p_rp, self.ws_list)]
        self.products = self.h.stats()["products"] if self.batched else None
        # one buffer for all partials, sliced per block
        tot = int(sum(self.p_nnz))
        self._pcol = torch.empty(max(tot, 1), dtype=torch.int32, device=self.dev)
        ob = api.OUT_BYTES[self.sr]
        self._pval = torch.empty(max(tot, 1) * ob, dtype=torch.uint8, device=self.dev) if ob else None
        self.p_col, self.p_val, off = [], [], 0
        for n in self.p_nnz:
            self.p_col.append(self._pcol[off:off + n])
            self.p_val.append(None if ob == 0 else self._pval[off * ob:(off + n) * ob])
            off += n
        self.partials = [api.DeviceCSR(a.nrows, b.ncols, rp, c, v)
                         for a, b, rp, c, v in zip(self.As, self.Bs, self.p_rp, self.p_col,
                                                    self.p_val)]

    def numeric(self):
        if self.batched:
            self.h.numeric_batched(self.sr, self.As, self.Bs, self.p_rp, self.p_col,
                                   self.p_val if self._pval is not None else None, self.ws)
        else:
            for a, b, rp, c, v, w in zip(self.As, self.Bs, self.p_rp, self.p_col, self.p_val,
                                         self.ws_list):
                self.hb.numeric(self.sr, a, b, rp, c, v, w)

    # ---- phase 2: merge of the stage partials of every C block ------------------

    def _groups(self):
        q = self.q
        idx = {(b.I, b.J, b.s): k for k, b in enumerate(self.blocks)}
        return [[self.partials[idx[(I, J, s)]] for s in range(self.stages)]
                for I in range(q) for J in range(q)]

    def merge_count(self):
        torch = self._torch
        groups = self._groups()
        self.groups = groups
        self.c_rp = [torch.empty(g[0].nrows + 1, dtype=torch.int64, device=self.dev) for g in groups]
        if self.batched:
            self.mws = torch.empty(self.h.merge_workspace_size(self.sr, groups), dtype=torch.uint8,
                                   device=self.dev)
            self.c_nnz = self.h.merge_count(self.sr, groups, self.c_rp, self.mws)
            self._mws_per_group = None
        else:
            self._mws_per_group = [torch.empty(self.h.merge_workspace_size(self.sr, [g]),
                                               dtype=torch.uint8, device=self.dev) for g in groups]
            self.c_nnz = [self.h.merge_count(self.sr, [g], [rp], w)[0]
                          for g, rp, w in zip(groups, self.c_rp, self._mws_per_group)]
        ob = api.OUT_BYTES[self.sr]
        self.c_col = [torch.empty(max(n, 1), dtype=torch.int32, device=self.dev) for n in self.c_nnz]
        self.c_val = [torch.empty(max(n, 1) * ob, dtype=torch.uint8, device=self.dev) if ob else None
                      for n in self.c_nnz]

    def merge_write(self):
        if self.batched:
            self.h.merge_write(self.sr, self.groups, self.c_rp, self.c_col,
                               self.c_val if api.OUT_BYTES[self.sr] else None, self.mws)
        else:
            for g, rp, c, v, w in zip(self.groups, self.c_rp, self.c_col, self.c_val,
                                      self._mws_per_group):
                self.h.merge_write(self.sr, [g], [rp], [c], [v] if v is not None else None, w)

    # ---- whole product ---------------------------------------------------------

    def plan(self):
        """Symbolic phase of the blocks and of the merges (sizes every buffer)."""
        self.symbolic()
        self.numeric()          # partial values are needed by nothing in the count,
        self.merge_count()      # but running them once warms the kernels up

    def run(self):
        """Numeric phase of every block product and the merges (replays the
        CUDA graph if one was captured)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self.numeric()
            self.merge_write()

    def capture(self, full: bool = False):
        """Capture numeric + merge write into one CUDA graph; with full=True
        (batched form) the whole product: row analysis, symbolic phase and
        scan of every block product, numeric phase, merge count and merge
        write, with no host synchronisation inside (every buffer was sized
        by plan())."""
        torch = self._torch
        if full and not self.batched:
            raise ValueError("the full graph needs the batched form")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())

        def body():
            if full:
                self.h.symbolic_batched(self.sr, self.As, self.Bs, self.p_rp, self.ws, sync=False)
            self.numeric()
            if full:
                self.h.merge_count(self.sr, self.groups, self.c_rp, self.mws, sync=False)
            self.merge_write()

        with torch.cuda.stream(s):
            body()                # warm-up outside the graph
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            body()
        self.graph = g
        self.graph_full = full
        return g

    def check(self):
        """Kernel-detected errors of every call (raises SpgemmError)."""
        if self.batched:
            self.h.check(self.ws)
            self.h.check(self.mws)
        else:
            for w in self.ws_list:
                self.hb.check(w)
            for w in self._mws_per_group:
                self.h.check(w)

    def block(self, I: int, J: int) -> api.DeviceCSR:
        k = I * self.q + J
        ob = api.OUT_BYTES[self.sr]
        val = self.c_val[k]
        if val is not None:
            val = api.typed_out(self.sr, val[:self.c_nnz[k] * ob])
        return api.DeviceCSR(self.row_cuts[I + 1] - self.row_cuts[I],
                             self.col_cuts[J + 1] - self.col_cuts[J], self.c_rp[k],
                             self.c_col[k][:self.c_nnz[k]], val)


def summa_panels(handle: api.Handle, sr: int, A: api.DeviceCSR, B: api.DeviceCSR,
                 budget_bytes: int, on_panel, q: int = 4, batched: bool = True,
                 stats: Optional[dict] = None):
    """The q x q Sparse-SUMMA emulation of C = A (x).(+) B in row panels whose
    output fits in budget_bytes (for products larger than HBM): every panel (a
    row view of A) is a full q x q grid of its own (block products of all
    stages and the merge of their partials); on_panel(r0, r1, summa) is called
    with the panel's finished Summa (blocks via summa.block(I, J)).
    stats: if given, filled with each panel's device milliseconds ("panel_ms",
    CUDA events around the phases; the host synchronisations of the symbolic
    and merge-count calls included) and the cuts.  Returns the panel count."""
    import torch
    h = handle
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device=A.rp.device)
    ws = torch.empty(h.workspace_size(sr, A, B), dtype=torch.uint8, device=A.rp.device)
    h.symbolic(sr, A, B, c_rp, ws)
    del ws
    per = 4 + api.OUT_BYTES[sr]
    cuts = api.panel_cuts(c_rp.cpu().numpy(), A.nrows, max(1, budget_bytes // per))
    times = []
    for r0, r1 in zip(cuts[:-1], cuts[1:]):
        Av = A.rows(r0, r1) if (r0, r1) != (0, A.nrows) else A
        sm = Summa(h, sr, Av, B, q=q, batched=batched)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sm.symbolic()
        sm.numeric()
        sm.merge_count()
        sm.merge_write()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        sm.check()
        on_panel(r0, r1, sm)
        del sm
        torch.cuda.empty_cache()
    if stats is not None:
        stats["panel_ms"] = times
        stats["cuts"] = cuts
    return len(cuts) - 1
