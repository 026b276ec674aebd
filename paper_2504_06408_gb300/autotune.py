"""Autotuner of the kernel tier limits (the counterpart of the paper's GALATIC
configuration knobs, Section 3.3: threads, threads per nonzero and chunk
limits were set by hand there).

Coordinate descent over the spg_tuning fields on a calibration product: each
field in turn is tried at a few values around the current one, the whole
symbolic + numeric call is timed with CUDA events (median of a few runs),
and the best value is kept; sweeps repeat until no field improves.  The
tuning changes only which kernel tier handles a row and how wide the
shared-memory slabs are, never C.  Results are cached in a JSON file keyed
by GPU name, semiring and workload tag.
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Callable, Dict, Optional

from . import spgemm as api

# candidate values per field (0 = library default)
SPACE = {
    "sym_warp_max_ub": [128, 256, 512, 1024, 2048],
    "sym_block_max_ub": [2048, 4096, 8192, 16384],
    "num_warp_max_nnz": [32, 64, 128, 256, 512],
    "num_block_max_nnz": [512, 1024, 2048, 4096],
    "dense_slab_cols": [8192, 16384, 32768],
    "rank_light_ub": [-1, 4096, 8192, 16384, 65536],
}

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "spgemm_gb300_tuning.json")
# tunings measured on this project's target GPU, shipped with the package
# (written by `python -m paper_2504_06408_gb300.autotune --out <this file> ...`)
SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


def _time_call(h: api.Handle, sr, dA, dB, ws, c_rp, c_col, c_val, reps: int) -> float:
    import torch
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        h.symbolic(sr, dA, dB, c_rp, ws)
        h.numeric(sr, dA, dB, c_rp, c_col, c_val, ws)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def tune(sr: int, dA: api.DeviceCSR, dB: api.DeviceCSR, reps: int = 3, sweeps: int = 2,
         start: Optional[Dict[str, int]] = None, log=None) -> Dict[str, int]:
    """Coordinate descent; returns the best tuning found (dict of spg_tuning fields)."""
    import torch
    best = dict(start or {})
    h = api.Handle(tuning=best or None)
    c_rp = torch.empty(dA.nrows + 1, dtype=torch.int64, device=dA.rp.device)
    # buffers sized once (nnz(C) does not depend on the tuning)
    ws_size = max(h.workspace_size(sr, dA, dB), 1)
    ws = torch.empty(ws_size, dtype=torch.uint8, device=dA.rp.device)
    nnz = h.symbolic(sr, dA, dB, c_rp, ws)
    c_col = torch.empty(max(nnz, 1), dtype=torch.int32, device=dA.rp.device)
    c_val = api.out_tensor(sr, max(nnz, 1), dA.rp.device)

    def measure(cfg):
        hh = api.Handle(tuning=cfg or None)
        need = hh.workspace_size(sr, dA, dB)
        nonlocal ws
        if need > ws.numel():
            ws = torch.empty(need, dtype=torch.uint8, device=dA.rp.device)
        _time_call(hh, sr, dA, dB, ws, c_rp, c_col, c_val, 1)   # warm-up
        return _time_call(hh, sr, dA, dB, ws, c_rp, c_col, c_val, reps)

    return descend(measure, SPACE, best, sweeps, log)


def tune_summa(sr: int, dA: api.DeviceCSR, dB: api.DeviceCSR, q: int = 4, reps: int = 3,
               sweeps: int = 1, start: Optional[Dict[str, int]] = None, log=None,
               space: Optional[Dict[str, list]] = None) -> Dict[str, int]:
    """Coordinate descent for the batched Sparse-SUMMA form: each candidate
    tuning times the CUDA-graph replay of the whole batched product (block
    symbolic and numeric phases and the merge of the stage partials)."""
    import torch
    from .summa import Summa

    def measure(cfg):
        h = api.Handle(tuning=cfg or None)
        sm = Summa(h, sr, dA, dB, q=q, batched=True)
        sm.plan()
        sm.capture(full=True)
        sm.run()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sm.run()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        sm.check()
        del sm
        torch.cuda.empty_cache()
        return statistics.median(ts)

    return descend(measure, space or SPACE, dict(start or {}), sweeps, log)


def descend(measure: Callable[[Dict[str, int]], float], space: Dict[str, list],
            start: Dict[str, int], sweeps: int = 2, log=None) -> Dict[str, int]:
    """Coordinate descent: every field of ``space`` in turn is tried at each
    candidate value with the others fixed; a value is kept when it beats the
    best time by more than 1%.  Sweeps repeat until one improves nothing."""
    best = dict(start)
    best_t = measure(best)
    if log:
        log(f"start {best} {best_t:.3f} ms")
    for _ in range(sweeps):
        improved = False
        for field, cands in space.items():
            for v in cands:
                if best.get(field) == v:
                    continue
                cfg = dict(best, **{field: v})
                t = measure(cfg)
                if log:
                    log(f"  {field}={v}: {t:.3f} ms")
                if t < best_t * 0.99:
                    best, best_t, improved = cfg, t, True
        if not improved:
            break
    if log:
        log(f"best {best} {best_t:.3f} ms")
    return best


def cache_key(sr: int, tag: str, device: Optional[str] = None) -> str:
    if device is None:
        import torch
        device = torch.cuda.get_device_name()
    return f"{device}|{api.SEMIRING_NAMES[sr]}|{tag}"


def load(sr: int, tag: str, path: str = DEFAULT_CACHE,
         device: Optional[str] = None) -> Optional[Dict[str, int]]:
    try:
        with open(path) as f:
            return json.load(f).get(cache_key(sr, tag, device))
    except (OSError, ValueError):
        return None


def save(sr: int, tag: str, tuning: Dict[str, int], path: str = DEFAULT_CACHE,
         device: Optional[str] = None) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    data = {}
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        pass
    data[cache_key(sr, tag, device)] = tuning
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned_handle(sr: int, dA, dB, tag: str, path: str = DEFAULT_CACHE, **kw) -> api.Handle:
    """Handle with the cached tuning for (GPU, semiring, tag), tuning first if absent."""
    t = load(sr, tag, path)
    if t is None:
        t = tune(sr, dA, dB, **kw)
        save(sr, tag, t, path)
    return api.Handle(tuning=t or None)


def main(argv=None):
    """Tune a workload on the current GPU and store the result in a JSON file."""
    import argparse

    import numpy as np
    import torch

    from . import inputs as I
    ap = argparse.ArgumentParser(description="tune the kernel tier limits on this GPU")
    ap.add_argument("form", choices=["plain", "summa"])
    ap.add_argument("--scale", type=int, default=18, help="R-MAT scale of A (A^2 is tuned)")
    ap.add_argument("--semiring", default="plus_times_f64", choices=sorted(
        api.SEMIRING_NAMES.values()))
    ap.add_argument("--sweeps", type=int, default=1)
    ap.add_argument("--out", default=DEFAULT_CACHE)
    args = ap.parse_args(argv)
    sr = {v: k for k, v in api.SEMIRING_NAMES.items()}[args.semiring]
    dt = api.IN_NP[sr]
    kw = {"lo": 0.0, "hi": 1.0} if dt == np.float64 else {}
    A = I.rmat(args.scale, dtype=dt, seed=1, **kw)
    dA = api.DeviceCSR.from_host(A, val_dtype=dt)
    if args.form == "plain":
        t = tune(sr, dA, dA, reps=3, sweeps=args.sweeps, log=print)
        tag = f"rmat{args.scale}"
    else:
        t = tune_summa(sr, dA, dA, reps=3, sweeps=args.sweeps, log=print)
        tag = f"summa4x4_rmat{args.scale}"
    save(sr, tag, t, args.out)
    torch.cuda.synchronize()
    print(json.dumps({"tag": tag, "tuning": t}))


if __name__ == "__main__":
    main()
