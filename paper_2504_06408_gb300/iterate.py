"""Iterated semiring products on the GPU: W^k and k-hop path semirings
(Section 2.2: with the min-plus semiring, entry (i, j) of W^k is the length of
the shortest walk of exactly k edges from i to j).

* `power(sr, W, k)`: W^k by repeated squaring (about log2 k squarings and as
  many multiplies by an accumulated power).  The pattern never depends on the
  association; values of float semirings do (min-plus sums and plus-times
  sums round differently along a different tree), integer and boolean ones
  do not.
* `hops(sr, W, k)`: D_k = D_{k-1} (+) (D_{k-1} (x) W), D_1 = W, i.e. the (+)
  over walks of 1..k edges (k-hop shortest distances for min-plus, k-hop
  reachability for boolean).  The elementwise (+) is the library's stage
  merge of two partials.

Only library calls and torch buffer handling happen here.
"""
from __future__ import annotations

from typing import Optional

from . import spgemm as api


def multiply(sr: int, A: api.DeviceCSR, B: api.DeviceCSR,
             handle: Optional[api.Handle] = None) -> api.DeviceCSR:
    return api.spgemm(sr, A, B, handle=handle)


def add(sr: int, X: api.DeviceCSR, Y: api.DeviceCSR,
        handle: Optional[api.Handle] = None) -> api.DeviceCSR:
    """Elementwise X (+) Y over the union of the patterns (the merge of two
    partials, X first)."""
    import torch
    h = handle or api.Handle()
    dev = X.rp.device
    ob = api.OUT_BYTES[sr]
    groups = [[X, Y]]
    ws = torch.empty(h.merge_workspace_size(sr, groups), dtype=torch.uint8, device=dev)
    c_rp = torch.empty(X.nrows + 1, dtype=torch.int64, device=dev)
    n = h.merge_count(sr, groups, [c_rp], ws)[0]
    c_col = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    c_val = torch.empty(max(n, 1) * ob, dtype=torch.uint8, device=dev) if ob else None
    h.merge_write(sr, groups, [c_rp], [c_col], [c_val] if ob else None, ws)
    h.check(ws)
    val = api.typed_out(sr, c_val[:n * ob]) if ob else None
    return api.DeviceCSR(X.nrows, X.ncols, c_rp, c_col[:n], val)


def as_input(sr: int, M: api.DeviceCSR) -> api.DeviceCSR:
    """A product's output used as the next product's input (same value type
    for every semiring but the overlap one, which is not iterable)."""
    if sr == api.OVERLAP_I32:
        raise ValueError("overlap records are not inputs of the overlap semiring")
    return M


def power(sr: int, W: api.DeviceCSR, k: int, handle: Optional[api.Handle] = None) -> api.DeviceCSR:
    if k < 1:
        raise ValueError("k >= 1")
    h = handle or api.Handle()
    result = None
    base = W
    e = k
    while True:
        if e & 1:
            result = base if result is None else as_input(sr, multiply(sr, result, base, h))
        e >>= 1
        if not e:
            return result
        base = as_input(sr, multiply(sr, base, base, h))


def hops(sr: int, W: api.DeviceCSR, k: int, handle: Optional[api.Handle] = None) -> api.DeviceCSR:
    if k < 1:
        raise ValueError("k >= 1")
    h = handle or api.Handle()
    D = W
    for _ in range(k - 1):
        D = as_input(sr, add(sr, D, multiply(sr, D, W, h), h))
    return D
