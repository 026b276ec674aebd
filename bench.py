#!/usr/bin/env python3
"""Benchmark of the semiring SpGEMM hot path on GB300.

Workload: C = A * A over the min-plus FP32 semiring for a symmetric R-MAT
graph of scale 18 (262,144 vertices, edge factor 16, a, b, c, d = .57, .19,
.19, .05, self loops and duplicates removed, weights U[1, 100), seed 1): a
synthetic stand-in of the paper's graph workloads (Table 2 "rmat").

One step = the whole path on resident device inputs: row analysis and
binning, symbolic phase, scan into C's row pointers, numeric phase with sorted
compacted output (spgemm_symbolic + spgemm_numeric).  value = 2 * products /
time (GFLOPS).  The inputs (61 MB) fit in L2, so a 256 MiB buffer is written
before every timed step to flush it.

Also reported: e2e (the same metric through the host-memory C ABI call,
host->device copies of A and the device->host copy of C inside the timed
region), the roofline of the dominant kernel, the CPU oracle on a bounded row
sample (cpu_baseline), clocks sampled during the timed steps, and the number
of library kernel launches.

--impl reference runs the CPU oracle (the plain sorted-map definition) as the
reference arm on a bounded row sample per step.

Multi-GPU: one process per GPU (torchrun); every rank runs the full product
(independent replicas, no data-path collective), value = total products of
all ranks / max time over ranks ("scaling": "weak").
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the comparison forms allocate and free tens of GB in turn (both names: the
# variable was renamed between PyTorch releases)
if "PYTORCH_CUDA_ALLOC_CONF" not in os.environ and "PYTORCH_ALLOC_CONF" not in os.environ:
    os.environ["PYTORCH_CUDA_ALLOC_CONF"] = "expandable_segments:True"
    os.environ["PYTORCH_ALLOC_CONF"] = "expandable_segments:True"

METRIC = "semiring SpGEMM GFLOPS (2*products/s), R-MAT scale 18 A^2 over min-plus FP32"
METRIC_SCALED = "semiring SpGEMM GFLOPS (2*products/s), R-MAT scale %d A^2 over min-plus FP32"
UNIT = "GFLOPS"
SCALE = 18
L2_FLUSH_BYTES = 256 << 20


def workload_config(P=None, nnz_c=None, nnz_a=None, scale=SCALE):
    cfg = {"workload": "R-MAT scale %d (%s vertices, edge factor 16, a=.57 b=.19 c=.19 "
                       "d=.05), symmetrised, self-loops and duplicates removed, FP32 weights "
                       "U[1,100), seed 1; C = A*A over min-plus FP32" % (scale, f"{1 << scale:,}"),
           "semiring": "min_plus_f32", "n": 1 << scale,
           "l2": "256 MiB buffer written before every timed step"}
    if nnz_a is not None:
        cfg["nnz_A"] = int(nnz_a)
    if P is not None:
        cfg["products"] = int(P)
    if nnz_c is not None:
        cfg["nnz_C"] = int(nnz_c)
    return cfg


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest value of x over the ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_mem_available():
    """MemAvailable of this node in bytes (None where /proc/meminfo is missing)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except (OSError, ValueError, IndexError):
        pass
    return None


def job_throughput(total_ms: float, steps: int, products_per_rank: int, world: int, dist=None,
                   device="cuda"):
    """(ms per step, GFLOPS) of the whole job: every rank runs the same product
    (replicas, weak scaling), the job takes as long as the slowest rank, and
    value = all ranks' 2 x products / that time."""
    ms = max_over_ranks(total_ms, dist, device) / steps
    return ms, world * 2.0 * products_per_rank / (ms * 1e-3) / 1e9


def host_placement():
    """CPU affinity of this process and the NUMA node of the current GPU (the
    host memory the e2e copies land in is placed by first touch)."""
    info = {}
    try:
        info["cpus"] = len(os.sched_getaffinity(0))
    except Exception:
        pass
    try:
        import torch
        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        bus = "%04x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        info["gpu_pci"] = bus
        with open(f"/sys/bus/pci/devices/{bus}/numa_node") as f:
            info["gpu_numa_node"] = int(f.read().strip())
    except Exception:
        pass
    return info


def _cpulist(text):
    out = set()
    for part in text.strip().split(","):
        if not part:
            continue
        if "-" in part:
            a, b = part.split("-")
            out.update(range(int(a), int(b) + 1))
        else:
            out.add(int(part))
    return out


def bind_host_to_gpu_node():
    """Keep this process's CPUs and new host pages on the current GPU's NUMA
    node (best effort, this process only): the e2e leg's pinned buffers are
    placed where they are first allocated, and device-host copies to a
    remote node cross the CPU-CPU link.  Returns what was applied."""
    info = host_placement()
    node = info.get("gpu_numa_node")
    bus = info.get("gpu_pci")
    if node is None or node < 0 or not bus:
        return info
    try:
        local = _cpulist(open(f"/sys/bus/pci/devices/{bus}/local_cpulist").read())
        allowed = os.sched_getaffinity(0)
        both = allowed & local
        info["cpus_local_to_gpu"] = len(both)
        if both and both != allowed:
            os.sched_setaffinity(0, both)
            info["affinity_set"] = True
    except (OSError, ValueError):
        pass
    try:   # set_mempolicy(MPOL_PREFERRED, {node}): new pages from the GPU's node
        import ctypes
        import platform
        nr = {"aarch64": 237, "x86_64": 238}.get(platform.machine())
        if nr is not None and node < 64:
            mask = ctypes.c_ulong(1 << node)
            rc = ctypes.CDLL(None, use_errno=True).syscall(nr, 1, ctypes.byref(mask), 65)
            info["mempolicy_preferred_node"] = node if rc == 0 else None
    except OSError:
        pass
    return info


def reset_mempolicy():
    try:
        import ctypes
        import platform
        nr = {"aarch64": 237, "x86_64": 238}.get(platform.machine())
        if nr is not None:
            ctypes.CDLL(None, use_errno=True).syscall(nr, 0, None, 0)
    except OSError:
        pass


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def row_stats(A, c_rp):
    """Per-row products (ub), nnz(A_i) and nnz(C_i) on the host (metrics only)."""
    deg = np.diff(A.rp)
    blen = deg  # B = A
    per_entry = blen[A.col.astype(np.int64)]
    ub = np.add.reduceat(np.r_[per_entry, 0], np.minimum(A.rp[:-1], A.col.size)) * (deg > 0)
    cnt = np.diff(c_rp)
    return ub.astype(np.int64), deg.astype(np.int64), cnt.astype(np.int64)


def traffic_from_profiles(kernel_src_hash):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "num_rank_minplus_rmat18_traffic.txt")
    try:
        kv = {}
        for line in open(path):
            if "=" in line and not line.startswith("#"):
                k, v = line.strip().split("=", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_sha256") == kernel_src_hash:
            return int(kv["traffic_bytes_per_launch"])
    except Exception:
        pass
    return None


# the sources the dominant kernel (k_num_rank, numeric.cu) is compiled from
RANK_KERNEL_SOURCES = ("common.cuh", "numeric.cu", "plan.h", "rowwork.cuh", "semiring.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2504_06408_gb300", "csrc")
    for name in RANK_KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()


def cpu_oracle_sample(A, target_s=12.0, seed=7):
    """Time the CPU oracle on a random row sample sized for ~target_s seconds."""
    import oracle
    ub, deg, _ = row_stats(A, np.zeros(A.nrows + 1, np.int64))
    rng = np.random.default_rng(seed)
    order = rng.permutation(np.nonzero(ub > 0)[0])
    threads = oracle.default_threads()
    # calibrate on a small sample
    csum = np.cumsum(ub[order])
    k = int(np.searchsorted(csum, 2e7)) + 1
    t0 = time.perf_counter()
    oracle.spgemm(oracle.SR_MP_F32, A, A, rows=order[:k], threads=threads)
    dt = time.perf_counter() - t0
    rate = csum[k - 1] / max(dt, 1e-3)
    want = rate * target_s
    k2 = int(np.searchsorted(csum, want)) + 1
    k2 = min(k2, order.size)
    rows = np.sort(order[:k2])
    P = int(ub[rows].sum())
    t0 = time.perf_counter()
    oracle.spgemm(oracle.SR_MP_F32, A, A, rows=rows, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": 2.0 * P / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{rows.size} random non-empty rows of the same product "
                      f"({P} of {int(ub.sum())} products), {dt:.1f} s wall"}, dt, P


def _time_ms(fn, reps, flush):
    """Median CUDA-event time of fn() (one warm-up call; L2 flushed before each)."""
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def same_result(ref_col, ref_val, col, val):
    """(same pattern, same values) of two device results with the same row
    pointers: columns bit-exact; values bit-exact (every semiring but the
    floating plus-times ones, whose atomic summation order is free) or, for
    those, max |got - ref| / |ref| (the inputs here are non-negative, so
    |ref| = sum |a b| and the parity bound is 1e-12)."""
    import torch
    same_col = bool(torch.equal(ref_col, col))
    if ref_val is None:
        return same_col, True, 0.0
    if ref_val.dtype in (torch.float64, torch.float32):
        exact = bool(torch.equal(ref_val.view(torch.uint8), val.view(torch.uint8)))
        if exact:
            return same_col, True, 0.0
        den = ref_val.abs().clamp_min(torch.finfo(ref_val.dtype).tiny)
        rel = float(((val - ref_val).abs() / den).max().item())
        return same_col, rel <= 1e-12, rel
    return same_col, bool(torch.equal(ref_val, val)), 0.0


def learned_forms(api, h, sr, dA, dB, flush, reps, plain_ms, params, meta):
    """plain vs learned (ub-sized capacities) vs learned (trained network) on
    one product; every form's C is compared with the plain C on the device,
    column by column and value by value (same_result)."""
    import torch
    out = {"plain_ms": plain_ms}
    ref_rp = torch.empty(dA.nrows + 1, dtype=torch.int64, device="cuda")
    ws0 = torch.empty(h.workspace_size(sr, dA, dB), dtype=torch.uint8, device="cuda")
    nnz = h.symbolic(sr, dA, dB, ref_rp, ws0)
    ref_col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    ref_val = api.out_tensor(sr, max(nnz, 1))
    h.numeric(sr, dA, dB, ref_rp, ref_col, ref_val, ws0)
    h.check(ws0)
    del ws0
    c_col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    c_val = api.out_tensor(sr, max(nnz, 1))
    lws = torch.empty(h.learned_workspace_size(sr, dA, dB), dtype=torch.uint8, device="cuda")
    c_rp = torch.empty_like(ref_rp)
    for name, model in (("learned_ub_sized", None), ("learned_network", params)):
        kw = {} if model is None else {"model": model, "margin": meta["margin"],
                                       "exact_max_ub": meta["exact_max_ub"]}
        sb = h.learned_plan(sr, dA, dB, lws, **kw)
        staging = torch.empty(max(sb, 1), dtype=torch.uint8, device="cuda")

        def step():
            h.learned_plan(sr, dA, dB, lws, **kw)
            h.learned_symbolic(sr, dA, dB, c_rp, lws, staging)
            h.learned_numeric(sr, dA, dB, c_rp, c_col, c_val, lws, staging)

        ms = _time_ms(step, reps, flush)
        st = h.stats()
        h.check(lws)
        same = bool(torch.equal(c_rp, ref_rp)) and st["nnz_c"] == nnz
        same_col, same_val, rel = same_result(ref_col, ref_val, c_col, c_val)
        out[name] = {"ms": ms, "speedup_vs_plain": plain_ms / ms, "same_row_ptr": same,
                     "same_columns": same_col, "same_values": same_val, "max_rel_diff": rel,
                     "learned_rows": st["learned_rows"], "overflow_rows": st["overflow_rows"],
                     "staging_entries": st["staging_entries"],
                     "staging_per_entry": st["staging_entries"] / max(st["learned_nnz"], 1)}
        del staging
    out["rows"] = dA.nrows
    del ref_col, ref_val, c_col, c_val
    return out


def plain_ms_of(api, h, sr, dA, dB, flush, reps, keep=False):
    """Median ms of symbolic + numeric, nnz(C) and (keep) C = (rp, col, val)."""
    import torch
    ws = torch.empty(h.workspace_size(sr, dA, dB), dtype=torch.uint8, device="cuda")
    c_rp = torch.empty(dA.nrows + 1, dtype=torch.int64, device="cuda")
    nnz = h.symbolic(sr, dA, dB, c_rp, ws)
    c_col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    c_val = api.out_tensor(sr, max(nnz, 1))

    def step():
        h.symbolic(sr, dA, dB, c_rp, ws)
        h.numeric(sr, dA, dB, c_rp, c_col, c_val, ws)

    ms = _time_ms(step, reps, flush)
    h.check(ws)
    if keep:
        return ms, nnz, (c_rp, c_col[:nnz], None if c_val is None else c_val[:nnz])
    return ms, nnz


def block_matches(ref, r0, r1, c0, c1, blk, chunk=1 << 27):
    """(same pattern, max rel value diff) of C block [r0, r1) x [c0, c1) (local
    column ids) against the same block cut out of the unblocked C, on the
    device, a chunk of rows at a time."""
    import torch
    rp, col, val = ref
    brp, bcol, bval = blk.rp, blk.col, blk.val
    rph = rp[r0:r1 + 1].cpu()
    ok, worst, x0 = True, 0.0, r0
    while x0 < r1:
        x1 = int(torch.searchsorted(rph, rph[x0 - r0] + chunk, right=True).item()) - 1 + r0
        x1 = min(max(x1, x0 + 1), r1)
        a, b = int(rph[x0 - r0]), int(rph[x1 - r0])
        cc = col[a:b]
        m = (cc >= c0) & (cc < c1)
        rows = torch.repeat_interleave(torch.arange(x1 - x0, device=cc.device, dtype=torch.int32),
                                       (rp[x0 + 1:x1 + 1] - rp[x0:x1]))
        cnt = torch.bincount(rows[m], minlength=x1 - x0)
        ba, bb = int(brp[x0 - r0].item()), int(brp[x1 - r0].item())
        ok &= bool(torch.equal(brp[x0 - r0 + 1:x1 - r0 + 1] - brp[x0 - r0:x1 - r0], cnt))
        ok &= bb - ba == int(m.sum().item()) and bool(torch.equal(bcol[ba:bb], cc[m] - c0))
        if ok and val is not None:
            ev = val[a:b][m]
            gv = bval[ba:bb]
            den = ev.abs().clamp_min(torch.finfo(ev.dtype).tiny)
            if ev.numel():
                worst = max(worst, float(((gv - ev).abs() / den).max().item()))
        x0 = x1
    return ok, worst


def summa_forms(api, Summa, h, sr, dA, flush, reps, ref=None, tuning=None):
    """4 x 4 Sparse-SUMMA block grid.  Batched: one launch per kernel tier over
    all 64 block products and one merge call, timed eagerly (host
    synchronisations between the phases) and as one CUDA graph of the whole
    product (analysis, symbolic, numeric and merge of every block, no host
    synchronisation); also with autotuned tier limits.  Unbatched: one call per
    block product and per merge.  With ref (the unblocked C), every C block of
    every form is compared with the same block of the unblocked product."""
    import torch
    out = {}
    forms = [("batched", True, None), ("unbatched", False, None)]
    if tuning:
        forms.insert(1, ("batched_tuned", True, tuning))
        out["tuning"] = tuning
    for key, batched, tun in forms:
        hh = api.Handle(tuning=tun) if tun else h
        sm = Summa(hh, sr, dA, dA, q=4, batched=batched)
        sm.plan()

        def full():
            sm.symbolic()
            sm.numeric()
            sm.merge_count()
            sm.merge_write()

        out[f"{key}_full_ms"] = _time_ms(full, reps, flush)
        if batched:
            sm.capture(full=True)
            out[f"{key}_graph_full_ms"] = _time_ms(sm.run, reps, flush)
        else:
            out["unbatched_numeric_merge_ms"] = _time_ms(sm.run, reps, flush)
        out[f"{key}_nnz_c"] = int(sum(sm.c_nnz))
        out["partial_entries"] = int(sum(sm.p_nnz))
        if ref is not None:
            sm.check()
            same, worst = True, 0.0
            for I_ in range(sm.q):
                for J_ in range(sm.q):
                    ok, w = block_matches(ref, sm.row_cuts[I_], sm.row_cuts[I_ + 1],
                                          sm.col_cuts[J_], sm.col_cuts[J_ + 1], sm.block(I_, J_))
                    same &= ok
                    worst = max(worst, w)
            out[f"{key}_same_pattern_as_unblocked"] = same
            out[f"{key}_max_rel_diff_vs_unblocked"] = worst
            out[f"{key}_within_1e-12"] = same and worst <= 1e-12
        del sm
        torch.cuda.empty_cache()
    out["speedup_full"] = out["unbatched_full_ms"] / out["batched_full_ms"]
    best = min(out.get("batched_tuned_graph_full_ms", float("inf")), out["batched_graph_full_ms"])
    out["speedup_graph_full_vs_unbatched"] = out["unbatched_full_ms"] / best
    return out


def summa_tuning(api, scale):
    """Tier limits of the batched SUMMA form on this workload: the autotuner's
    result shipped with the package for this GPU, else the per-user cache,
    else None (the library defaults)."""
    from paper_2504_06408_gb300 import autotune
    tag = f"summa4x4_rmat{scale}"
    t = autotune.load(api.PLUS_TIMES_F64, tag, autotune.SHIPPED)
    if t is None:
        t = autotune.load(api.PLUS_TIMES_F64, tag)
    return t


def t_alg_bytes(n, nnz_a, P, nnz_c, s_in, s_out):
    """Gustavson traffic model: row pointers of A and C, A's entries and the
    B row-pointer gathers, every product's B entry, C's entries."""
    return 8 * (n + 1) + nnz_a * (4 + s_in) + 8 * nnz_a + P * (4 + s_in) + 8 * (n + 1) + \
        nnz_c * (4 + s_out)


def bool_form(api, h, A, flush, reps, peak):
    """C = A A over the boolean semiring (pattern only) on the headline graph."""
    import torch
    dAb = api.DeviceCSR.from_host(A.with_values(None))
    ms, nnz = plain_ms_of(api, h, api.BOOL_OR_AND, dAb, dAb, flush, reps)
    P = h.stats()["products"]
    t = t_alg_bytes(A.nrows, A.nnz, P, nnz, 0, 0)
    del dAb
    torch.cuda.empty_cache()
    return {"ms": ms, "gflops": 2.0 * P / (ms * 1e-3) / 1e9, "products": P, "nnz_c": nnz,
            "algorithmic_bytes": t, "hbm_roofline_frac_step": t / (ms * 1e-3) / 1e9 / peak}


def er_forms(api, h, flush, reps=21):
    """Erdos-Renyi 4096 x 4096, 8 entries per row, A A over plus-times FP64 and
    boolean: latency-bound, reported in microseconds (median of 21)."""
    from paper_2504_06408_gb300 import inputs as I
    E = I.er(4096, 8, seed=1)
    out = {}
    for name, sr, dt in (("plus_times_f64", api.PLUS_TIMES_F64, np.float64),
                         ("bool", api.BOOL_OR_AND, None)):
        dE = api.DeviceCSR.from_host(E if dt else E.with_values(None), val_dtype=dt)
        ms, nnz = plain_ms_of(api, h, sr, dE, dE, flush, reps)
        P = h.stats()["products"]
        out[name] = {"us": 1e3 * ms, "gflops": 2.0 * P / (ms * 1e-3) / 1e9, "products": P,
                     "nnz_c": nnz}
    return out


def kmer_form(api, h, flush, reps, peak, reads=200_000):
    """k-mer overlap product C = A A^T (200,000 reads x 2^24 k-mers, overlap
    semiring, int32 positions; fewer reads for profiling captures); A^T by the
    library's transpose (untimed)."""
    import torch
    from paper_2504_06408_gb300 import inputs as I
    A = I.kmer(nrows=reads, seed=1)
    dA = api.DeviceCSR.from_host(A, val_dtype=np.int32)
    dAt = h.transpose(dA, 4)
    ms, nnz = plain_ms_of(api, h, api.OVERLAP_I32, dA, dAt, flush, reps)
    P = h.stats()["products"]
    t = t_alg_bytes(A.nrows, A.nnz, P, nnz, 4, 20)
    del dA, dAt
    torch.cuda.empty_cache()
    return {"ms": ms, "gflops": 2.0 * P / (ms * 1e-3) / 1e9, "products": P, "nnz_c": nnz,
            "algorithmic_bytes": t, "hbm_roofline_frac": t / (ms * 1e-3) / 1e9 / peak}


def panel_budget(frac=0.12, cap=32 << 30):
    """Output bytes per row panel: a fraction of the free device memory (the
    panel's C, its partials and workspaces must fit at once)."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    return int(min(cap, free * frac))


def config4_form(api, peak):
    """R-MAT 20 A^2 over plus-times FP64 (1,048,576 vertices, FP64 weights
    U[0,1)) as a 4 x 4 Sparse-SUMMA emulation: C is about 294 GB, so the
    product runs in row panels, each a full 4 x 4 grid (batched: one launch
    per tier over its 64 block products; unbatched: one call per block and
    merge), against the unblocked product in the same panels."""
    import torch
    from paper_2504_06408_gb300 import inputs as I
    from paper_2504_06408_gb300.summa import summa_panels
    sr = api.PLUS_TIMES_F64
    A = I.rmat(20, dtype=np.float64, seed=1, lo=0.0, hi=1.0)
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float64)
    h = api.Handle()
    budget = panel_budget()
    out = {"workload": "R-MAT scale 20 A^2, plus-times FP64, 4 x 4 grid, row panels",
           "panel_output_bytes": budget}
    nnz = {}
    st = {}
    nnz["plain"], out["plain_panels"] = api.panel_product(
        sr, dA, dA, budget, lambda a, b, C: None, handle=h, stats=st)
    out["plain_ms"] = sum(st["panel_ms"])
    for key, batched in (("summa_batched", True), ("summa_unbatched", False)):
        st = {}
        tot = [0]

        def on_panel(r0, r1, sm, tot=tot):
            tot[0] += int(sum(sm.c_nnz))

        out[f"{key}_panels"] = summa_panels(h, sr, dA, dA, budget, on_panel, q=4,
                                            batched=batched, stats=st)
        out[f"{key}_ms"] = sum(st["panel_ms"])
        nnz[key] = tot[0]
        torch.cuda.empty_cache()
    ws = torch.empty(h.workspace_size(sr, dA, dA), dtype=torch.uint8, device="cuda")
    rp = torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda")
    h.symbolic(sr, dA, dA, rp, ws)
    P = h.stats()["products"]
    del ws
    out["products"] = P
    out["nnz_c"] = nnz["plain"]
    out["same_nnz_all_forms"] = len(set(nnz.values())) == 1
    t = t_alg_bytes(A.nrows, A.nnz, P, nnz["plain"], 8, 8)
    for key in ("plain", "summa_batched", "summa_unbatched"):
        ms = out[f"{key}_ms"]
        out[f"{key}_gflops"] = 2.0 * P / (ms * 1e-3) / 1e9
        out[f"{key}_hbm_roofline_frac"] = t / (ms * 1e-3) / 1e9 / peak
    out["summa_batched_vs_unbatched"] = out["summa_unbatched_ms"] / out["summa_batched_ms"]
    out["summa_batched_vs_unblocked"] = out["summa_batched_ms"] / out["plain_ms"]
    del dA
    torch.cuda.empty_cache()
    return out


def config5_form(api, params, meta, peak):
    """R-MAT 21 A^2 over plus-times FP64 (2,097,152 vertices, FP64 weights
    U[0,1)): C is about 757 GB, so every form runs in row panels: plain,
    learned sizing with ub-sized capacities, learned sizing with the trained
    network."""
    import torch
    from paper_2504_06408_gb300 import inputs as I
    sr = api.PLUS_TIMES_F64
    A = I.rmat(21, dtype=np.float64, seed=1, lo=0.0, hi=1.0)
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float64)
    h = api.Handle()
    budget = panel_budget()
    out = {"workload": "R-MAT scale 21 A^2, plus-times FP64, row panels",
           "panel_output_bytes": budget}
    nnz = {}
    forms = (("plain", None), ("learned_ub_sized", {}),
             ("learned_network", {"model": params, "margin": meta["margin"],
                                  "exact_max_ub": meta["exact_max_ub"]}))
    for key, learned in forms:
        st = {}
        nnz[key], out[f"{key}_panels"] = api.panel_product(
            sr, dA, dA, budget, lambda a, b, C: None, handle=h, learned=learned, stats=st)
        out[f"{key}_ms"] = sum(st["panel_ms"])
        torch.cuda.empty_cache()
    ws = torch.empty(h.workspace_size(sr, dA, dA), dtype=torch.uint8, device="cuda")
    rp = torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda")
    h.symbolic(sr, dA, dA, rp, ws)
    P = h.stats()["products"]
    del ws
    out["products"] = P
    out["nnz_c"] = nnz["plain"]
    out["same_nnz_all_forms"] = len(set(nnz.values())) == 1
    t = t_alg_bytes(A.nrows, A.nnz, P, nnz["plain"], 8, 8)
    for key, _ in forms:
        ms = out[f"{key}_ms"]
        out[f"{key}_gflops"] = 2.0 * P / (ms * 1e-3) / 1e9
        out[f"{key}_hbm_roofline_frac"] = t / (ms * 1e-3) / 1e9 / peak
        if key != "plain":
            out[f"{key}_speedup_vs_plain"] = out["plain_ms"] / ms
    del dA
    torch.cuda.empty_cache()
    return out


# Stand-ins shaped like the paper's Table 2 matrices, multiplied over the
# plus-times "float" semiring as in its experiments
FLOAT_STANDINS = {
    "rmat_16_ef4": "R-MAT scale 16, edge factor 4 (65,536 rows, 494,224 entries; Table 2 rmat: "
                   "65,536 rows, 490,228)",
    "stencil7_108": "3D 7-point stencil on 108^3 (1,259,712 rows, 8,748,000 entries; atmosmodd: "
                    "1,270,432 rows, 8,814,880)",
    "trigrid_2048": "triangular lattice 2048^2, 6 neighbours (4,194,304 rows, 25,149,442 "
                    "entries; delaunay_n22: 4,194,304 rows, 25,165,738)",
    "stencil27_114": "3D 27-point stencil on 114^3 (1,481,544 rows; Long_dt_Coup0: 1,470,152 "
                     "rows, 70,219,816 entries, denser rows)",
}


def float_standin(name):
    from paper_2504_06408_gb300 import inputs as I
    if name == "rmat_16_ef4":
        return I.rmat(16, edge_factor=4, seed=1, dtype=np.float32)
    if name == "stencil7_108":
        return I.stencil3d(108, 7)
    if name == "trigrid_2048":
        return I.trigrid(2048)
    return I.stencil3d(114, 27)


def cold_warm_one(name):
    """First multiplication in a fresh process (lazy kernel loading, workspace
    and output allocation included: the paper's first-iteration time) against
    the median of 5 warm ones on preallocated buffers; plus-times FP32."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_06408_gb300 import spgemm as api
    A = float_standin(name)
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float32)
    torch.cuda.synchronize()
    sr = api.PLUS_TIMES_F32
    t0 = time.perf_counter()
    h = api.Handle()
    C = api.spgemm(sr, dA, dA, handle=h)
    torch.cuda.synchronize()
    cold = 1e3 * (time.perf_counter() - t0)
    P = h.stats()["products"]
    ws = torch.empty(h.workspace_size(sr, dA, dA), dtype=torch.uint8, device="cuda")
    ts = []
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.symbolic(sr, dA, dA, C.rp, ws)
        h.numeric(sr, dA, dA, C.rp, C.col, C.val, ws)
        torch.cuda.synchronize()
        ts.append(1e3 * (time.perf_counter() - t0))
    return {"cold_ms": cold, "warm_ms": statistics.median(ts), "nrows": A.nrows, "nnz": A.nnz,
            "products": P, "nnz_c": C.nnz}


def cold_warm_forms():
    """cold_warm_one for every stand-in, each in its own process."""
    out = {"note": "plus-times FP32; cold = first call in a fresh process (host wall clock, "
                   "kernel loading and allocations included), warm = median of 5 later "
                   "calls (host wall clock)"}
    for name, what in FLOAT_STANDINS.items():
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cold-warm", name],
                           capture_output=True, text=True)
        try:
            res = json.loads(r.stdout.strip().splitlines()[-1])
        except Exception:
            res = {"error": (r.stderr or r.stdout)[-300:]}
        res["matrix"] = what
        out[name] = res
    return out


def run_reference(args, rank):
    """Reference arm: the CPU oracle on a bounded row sample per step.  Only
    the oracle is built and loaded here, never the CUDA library."""
    if rank != 0:
        return 0
    import oracle.build as _ob
    _ob.build()
    import oracle
    from paper_2504_06408_gb300 import inputs as I
    A = I.rmat(SCALE, dtype=np.float32, seed=1)
    ub, _, _ = row_stats(A, np.zeros(A.nrows + 1, np.int64))
    threads = oracle.default_threads()
    rng = np.random.default_rng(11)
    nz = np.nonzero(ub > 0)[0]
    # per-step sample sized for ~6 s of oracle work
    probe = np.sort(rng.choice(nz, 2000, replace=False))
    t0 = time.perf_counter()
    oracle.spgemm(oracle.SR_MP_F32, A, A, rows=probe, threads=threads)
    rate = ub[probe].sum() / max(time.perf_counter() - t0, 1e-3)
    times, prods = [], []
    for step in range(args.warmup + args.steps):
        order = rng.permutation(nz)
        csum = np.cumsum(ub[order])
        k = int(np.searchsorted(csum, rate * 6.0)) + 1
        rows = np.sort(order[:k])
        t0 = time.perf_counter()
        oracle.spgemm(oracle.SR_MP_F32, A, A, rows=rows, threads=threads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            prods.append(int(ub[rows].sum()))
    value = 2.0 * sum(prods) / sum(times) / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": workload_config(P=int(ub.sum()), nnz_a=A.nnz),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": f"per step a random row sample of ~6 s "
                                      f"({int(np.mean(prods))} products on average)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cold-warm", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the learned / batched vs plain comparisons")
    ap.add_argument("--form-reps", type=int, default=3)
    ap.add_argument("--forms", default="",
                    help="comma-separated subset of the comparison forms to run (names as in "
                         "the output, without the scale prefix: min_plus, bool, er4096, "
                         "kmer_overlap, laplacian, summa, float_cold_warm, rmat20, rmat21); "
                         "default all")
    ap.add_argument("--kmer-reads", type=int, default=200_000,
                    help="reads of the k-mer overlap form (200,000 = the workload; fewer for "
                         "profiling captures)")
    ap.add_argument("--no-big-forms", action="store_true",
                    help="skip the R-MAT 20 / 21 forms whose C exceeds device memory")
    ap.add_argument("--scale", type=int, default=SCALE,
                    help="R-MAT scale of the product (18 = the headline workload; smaller "
                         "scales are for profiling captures)")
    args = ap.parse_args()
    world, rank, local = dist_info()
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.cold_warm:
        print(json.dumps(cold_warm_one(args.cold_warm)), flush=True)
        return 0

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_06408_gb300 import inputs as I
    from paper_2504_06408_gb300 import spgemm as api

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    sr = api.MIN_PLUS_F32
    A = I.rmat(args.scale, dtype=np.float32, seed=1)
    # the kernel tier limits the autotuner found for this workload on this GPU
    # (shipped with the package), else the library defaults
    from paper_2504_06408_gb300 import autotune
    tuning = autotune.load(sr, f"rmat{args.scale}", autotune.SHIPPED)
    h = api.Handle(tuning=tuning or None)
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float32)
    ws = torch.empty(h.workspace_size(sr, dA, dA), dtype=torch.uint8, device="cuda")
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda")
    nnz = h.symbolic(sr, dA, dA, c_rp, ws)
    stats = h.stats()
    P = stats["products"]
    c_col = torch.empty(nnz, dtype=torch.int32, device="cuda")
    c_val = torch.empty(nnz, dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        h.symbolic(sr, dA, dA, c_rp, ws)
        h.numeric(sr, dA, dA, c_rp, c_col, c_val, ws)

    # the clock sampler (an nvidia-smi process) starts before the warm-up steps,
    # so that its start-up does not fall inside the timed region
    sampler = ClockSampler(torch.cuda.current_device())
    times, dense_ms, launches, stages = [], [], 0, []
    with sampler:
        for _ in range(args.warmup):
            step()
        h.check(ws)
        torch.cuda.synchronize()
        h.set_timing(True)
        barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.symbolic(sr, dA, dA, c_rp, ws)
            launches += h.stats()["launches"]
            sym_st = h.stage_times()
            h.numeric(sr, dA, dA, c_rp, c_col, c_val, ws)
            e1.record(stream)
            torch.cuda.synchronize()
            launches += h.stats()["launches"]
            num_st = h.stage_times()
            dense_ms.append(num_st["num_dense"])
            stages.append({k: v for st_ in (sym_st, num_st) for k, v in st_.items() if v > 0})
            times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        barrier()
    h.set_timing(False)
    h.check(ws)
    ms_per_step, value = job_throughput(sum(times), args.steps, P, world, dist)

    # roofline of the dominant kernel (numeric dense tier) by the Gustavson
    # traffic model restricted to the rows it processes
    hc_rp = c_rp.cpu().numpy()
    ub, deg, cnt = row_stats(A, hc_rp)
    # numeric dense tier: nnz(C_i) above the block-tier limit in effect (the
    # library's default 2048 unless the tuning sets it)
    dense = cnt > int((tuning or {}).get("num_block_max_nnz") or 2048)
    s_in, s_out = 4, 4
    t_alg = (16 * int(dense.sum()) + int(deg[dense].sum()) * (4 + s_in) + 8 * int(deg[dense].sum())
             + int(ub[dense].sum()) * (4 + s_in) + int(cnt[dense].sum()) * (4 + s_out))
    d_ms = statistics.mean(dense_ms)
    achieved = t_alg / (d_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = traffic_from_profiles(kernel_source_hash()) if args.scale == SCALE else None
    roofline = {"bound": "hbm",
                "kernel": "k_num_rank<SrMpF32> (numeric dense tier: the 1024-thread launch for "
                          "dense rows and the 512-thread one for light rows)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind, "traffic": traffic, "kernel_ms": d_ms,
                "algorithmic_bytes": t_alg}

    # whole-step fraction of the HBM roofline by the same model
    t_alg_all = (16 * A.nrows + A.nnz * (8 + 8) + P * 8 + nnz * 8)
    # compulsory bytes: A and B read once, C written once (B = A, counted twice)
    t_min = 2 * (8 * (A.nrows + 1) + A.nnz * 8) + 8 * (A.nrows + 1) + nnz * 8

    # e2e through the host-memory C ABI call: H2D of A, D2H of C every step
    e2e = None
    run_e2e = args.e2e_steps > 0
    if run_e2e:
        # with several ranks, every rank of the node pins A and all of C on the
        # host at once; with too little host memory for that the e2e leg is
        # left out on every rank
        need = world * (A.nnz * 16 + nnz * 8 + (A.nrows + 1) * 16)
        avail = host_mem_available()
        short = 1.0 if (world > 1 and avail is not None and need > 0.9 * avail) else 0.0
        run_e2e = max_over_ranks(short, dist) == 0.0
        if not run_e2e and rank == 0:
            print(f"e2e left out: {world} ranks need {need / 1e9:.0f} GB of pinned host memory, "
                  f"{(avail or 0) / 1e9:.0f} GB available", file=sys.stderr, flush=True)
    if run_e2e:
        saved_affinity = os.sched_getaffinity(0)
        placement = bind_host_to_gpu_node()
        pinned = []

        def pin(n, dt):
            t = torch.empty(n, dtype=dt, pin_memory=True)
            pinned.append(t)
            return t.numpy()
        hA = I.CSR(A.nrows, A.ncols, pin(A.nrows + 1, torch.int64), pin(A.nnz, torch.int32),
                   pin(A.nnz, torch.float32))
        hA.rp[:] = A.rp
        hA.col[:] = A.col
        hA.val[:] = A.val
        out = {"rp": pin(A.nrows + 1, torch.int64), "col": pin(nnz, torch.int32),
               "val": pin(nnz * 4, torch.uint8)}
        # first touch of the output pages outside the timed region
        out["col"][::1024] = 0
        out["val"][::4096] = 0
        h2 = api.Handle()
        h2.host_multiply(sr, hA, hA, out=out)         # warm-up (device buffers allocated)
        et = []
        for _ in range(args.e2e_steps):
            barrier()
            t0 = time.perf_counter()
            _, _, _, n2 = h2.host_multiply(sr, hA, hA, out=out)
            et.append(time.perf_counter() - t0)
        assert n2 == nnz
        e_s = max_over_ranks(statistics.mean(et), dist)
        h2d = (A.nrows + 1) * 8 + A.nnz * 8
        d2h = (A.nrows + 1) * 8 + nnz * 8
        # the same run's device-to-host bandwidth into the same pinned buffers
        # (C's columns and values from the device step): the e2e floor
        t_col, t_val = pinned[-2], pinned[-1]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t_col.copy_(c_col, non_blocking=True)
        t_val.copy_(c_val.view(torch.uint8), non_blocking=True)
        torch.cuda.synchronize()
        d2h_s = time.perf_counter() - t0
        d2h_gbs = nnz * 8 / d2h_s / 1e9
        e2e = {"value": world * 2.0 * P / e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e_s, "steps": len(et),
               "step_ms": [1e3 * x for x in et],
               "d2h_gbs_same_run": d2h_gbs, "d2h_floor_ms": 1e3 * d2h / (d2h_gbs * 1e9),
               "host": placement}
        del h2, pinned, hA, out
        os.sched_setaffinity(0, saved_affinity)   # the CPU baseline uses every core
        reset_mempolicy()

    forms = None
    if not args.no_forms:
        from paper_2504_06408_gb300 import learned as L
        from paper_2504_06408_gb300.summa import Summa
        params, meta = L.load()
        reps = args.form_reps
        forms = {"note": "median of %d CUDA-event timings per form, L2 flushed before each; "
                         "each form's C is compared with the plain C on the device "
                         "(same_* keys); plain_ms of the headline workload = the median of "
                         "its timed steps"
                         % reps}
        del c_col, c_val, step
        torch.cuda.empty_cache()

        wanted = [w for w in args.forms.split(",") if w]

        def form(name, fn, key):
            """one comparison form (selected by `key` with --forms); a failure is
            recorded, not fatal to the bench line"""
            if wanted and key not in wanted:
                return
            try:
                forms[name] = fn()
            except Exception as ex:   # noqa: BLE001
                forms[name] = {"error": f"{type(ex).__name__}: {str(ex)[:300]}"}
            torch.cuda.empty_cache()

        form(f"rmat{args.scale}_min_plus",
             lambda: learned_forms(api, h, sr, dA, dA, flush, reps, statistics.median(times),
                                  params, meta),
             "min_plus")
        form(f"rmat{args.scale}_bool", lambda: bool_form(api, h, A, flush, reps, peak), "bool")
        del dA
        torch.cuda.empty_cache()
        form("er4096", lambda: er_forms(api, h, flush), "er4096")
        form("kmer_overlap", lambda: kmer_form(api, h, flush, reps, peak, args.kmer_reads),
             "kmer_overlap")

        def laplacian_form():
            lap = I.laplacian(2048)
            dL = api.DeviceCSR.from_host(lap, val_dtype=np.float64)
            pms, _ = plain_ms_of(api, h, api.PLUS_TIMES_F64, dL, dL, flush, reps)
            return learned_forms(api, h, api.PLUS_TIMES_F64, dL, dL, flush, reps, pms, params,
                                 meta)

        form("laplacian2048_plus_times_f64", laplacian_form, "laplacian")

        def summa_form():
            A64 = I.rmat(args.scale, dtype=np.float64, seed=1, lo=0.0, hi=1.0)
            dA64 = api.DeviceCSR.from_host(A64, val_dtype=np.float64)
            pms, _, ref = plain_ms_of(api, h, api.PLUS_TIMES_F64, dA64, dA64, flush, reps,
                                      keep=True)
            torch.cuda.empty_cache()
            tuning = summa_tuning(api, args.scale)
            sf = summa_forms(api, Summa, h, api.PLUS_TIMES_F64, dA64, flush, reps, ref=ref,
                             tuning=tuning)
            sf["plain_unblocked_ms"] = pms
            best = min(sf.get("batched_tuned_graph_full_ms", float("inf")),
                       sf["batched_graph_full_ms"])
            sf["batched_graph_full_vs_unblocked"] = best / pms
            return sf

        form(f"rmat{args.scale}_plus_times_f64_summa4x4", summa_form, "summa")
        form("float_cold_warm", cold_warm_forms, "float_cold_warm")
        if not args.no_big_forms:
            form("rmat20_plus_times_f64_summa4x4_panels", lambda: config4_form(api, peak),
                 "rmat20")
            form("rmat21_plus_times_f64_learned_panels",
                 lambda: config5_form(api, params, meta, peak), "rmat21")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, _, _ = cpu_oracle_sample(A)

    if rank == 0:
        res = {"metric": METRIC if args.scale == SCALE else METRIC_SCALED % args.scale,
               "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": dict(workload_config(P=P, nnz_c=nnz, nnz_a=A.nnz, scale=args.scale),
                              parallelism=f"replicas x{world}", tuning=tuning or "defaults"),
               "hbm_roofline_frac_step": (t_alg_all / (ms_per_step * 1e-3) / 1e9) / peak,
               "hbm_compulsory_frac_step": (t_min / (ms_per_step * 1e-3) / 1e9) / peak,
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "clocks": sampler.summary(), "gpu_launches": launches,
               "step_ms": times,
               "stage_ms": {k: statistics.median([st.get(k, 0.0) for st in stages])
                            for k in sorted({k for st in stages for k in st})},
               "forms": forms}
        print(json.dumps(res), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
