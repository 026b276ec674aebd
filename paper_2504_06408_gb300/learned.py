"""Output-size network: training data, GPU training, margin calibration,
weights file, and loading for the learned-sizing path of the library.

The paper sizes every output row with an exact symbolic pass (Section 2.1,
Gustavson).  The library's learned path (spgemm_learned_*) lets a small
network predict r_i = nnz(C_i) / ub_i instead, so that most rows skip that
pass; rows that overflow their predicted capacity are redone exactly.

Training data is what the method itself produces: for products drawn by the
three workload generators (Erdos-Renyi, R-MAT, k-mer reads x k-mers with
B = A^T) at seeds the tests and the benchmark never use, the library's row
features (spgemm_row_features) and exact row counts (spgemm_symbolic) give
(f_i, log r_i) for every row with ub_i above the exact-bound threshold.  The
network is trained on the GPU by the library's own kernels
(spgemm_mlp_grad: forward + backward of the pinball loss; spgemm_mlp_adam),
then the capacity margin m is chosen on held-out rows so that at most a
target fraction of rows overflow cap_i = ceil(ub_i * r_i * m).

Weights file: ``<stem>.json`` (format, layout, training record, margin,
sha256 of the binary) + ``<stem>.bin`` (SPGEMM_MLP_PARAMS float32
little-endian FP32 master weights).  Loading converts them to the BF16 copy
used for inference with the library's kernel.

Only library calls and torch buffer handling happen here: every arithmetic
step of the network runs in the CUDA library.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import time
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import inputs as I
from . import spgemm as api

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_STEM = os.path.join(HERE, "weights", "row_nnz_mlp")
EXACT_MAX_UB = 32          # rows with ub <= this are sized by ub (no prediction): they
                           # take the library's register path, whose capacity is ub
TRAIN_SEEDS = (1001, 1002, 1003, 1004, 1005, 1006)
VALID_SEEDS = (1007,)


def workload_products(seed: int, small: bool = False):
    """Host products (name, A, B) of the three workload generators at one seed.
    B = A for ER and R-MAT (C = A A), B = A^T for the k-mer matrix (C = A A^T,
    transposed on the GPU by the caller).  The R-MAT scale cycles through
    14..18 with the seed (and scale 18 is added for the validation seed and
    the first and last training seeds), so the data spans graph sizes."""
    out = [("er4096", I.er(4096, 8, seed=seed, dtype=None), None)]
    if small:
        out.append(("rmat14", I.rmat(14, seed=seed, dtype=None), None))
        out.append(("kmer", I.kmer(nrows=5000, seed=seed), "T"))
        return out
    scale = 14 + (seed - TRAIN_SEEDS[0]) % 5
    out.append((f"rmat{scale}", I.rmat(scale, seed=seed, dtype=None), None))
    if scale != 18 and seed in (TRAIN_SEEDS[0], TRAIN_SEEDS[-1]) + VALID_SEEDS:
        out.append(("rmat18", I.rmat(18, seed=seed, dtype=None), None))
    out.append(("kmer", I.kmer(nrows=20000, seed=seed), "T"))
    return out


def _names(seed: int, small: bool):
    """Names of workload_products(seed) without drawing the matrices."""
    if small:
        return [("er4096", None, None), ("rmat14", None, None), ("kmer", None, None)]
    scale = 14 + (seed - TRAIN_SEEDS[0]) % 5
    out = [("er4096", None, None), (f"rmat{scale}", None, None)]
    if scale != 18 and seed in (TRAIN_SEEDS[0], TRAIN_SEEDS[-1]) + VALID_SEEDS:
        out.append(("rmat18", None, None))
    return out + [("kmer", None, None)]


def row_dataset(h: api.Handle, A: api.DeviceCSR, B: api.DeviceCSR,
                exact_max: int = EXACT_MAX_UB):
    """(features [m, 4], log r [m], ub [m], nnz [m]) device tensors for the rows
    of C = A B with ub > exact_max."""
    import torch
    ws = torch.empty(max(h.workspace_size(api.BOOL_OR_AND, A, B), 1), dtype=torch.uint8,
                     device=A.rp.device)
    feat, ub = h.row_features(A, B, ws)
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device=A.rp.device)
    h.symbolic(api.BOOL_OR_AND, A, B, c_rp, ws)
    nnz = c_rp[1:] - c_rp[:-1]
    keep = ub > exact_max
    feat, ub, nnz = feat[keep].contiguous(), ub[keep], nnz[keep]
    logt = torch.log(nnz.double() / ub.double()).float().contiguous()
    return feat, logt, ub, nnz


def collect(seeds, small: bool = False, log=None):
    import torch
    h = api.Handle()
    feats, logts, ubs, nnzs = [], [], [], []
    for seed in seeds:
        for name, A, how in workload_products(seed, small):
            dA = api.DeviceCSR.from_host(A)
            dB = h.transpose(dA, 0) if how == "T" else dA
            f, lt, ub, nz = row_dataset(h, dA, dB)
            feats.append(f)
            logts.append(lt)
            ubs.append(ub)
            nnzs.append(nz)
            if log:
                log(f"seed {seed} {name}: {A.nrows} rows, {f.shape[0]} with ub > {EXACT_MAX_UB}")
            del dA, dB
    return torch.cat(feats), torch.cat(logts), torch.cat(ubs), torch.cat(nnzs)


def init_master(seed: int = 0) -> np.ndarray:
    """Uniform fan-in initialisation, zero hidden biases.  The features reach
    ~15 (log1p of counts up to millions), so W1 is scaled down 8x; W3 starts
    100x smaller and b3 = 2, so that every row starts at r = sigmoid(2) = 0.88,
    near the typical ratio.  Starting far below it (r = 1/2) made the first
    steps push every row to r -> 1, where the gradient of log sigmoid(z)
    vanishes and training stalls."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, fan_in, scale, shape in (("W1", 4, 1 / 8, (64, 4)), ("b1", 0, 0, (64,)),
                                       ("W2", 64, 1.0, (64, 64)), ("b2", 0, 0, (64,)),
                                       ("W3", 64, 1e-2, (64,)), ("b3", 0, 0, (1,))):
        if fan_in:
            lim = scale * np.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-lim, lim, shape).ravel())
        else:
            parts.append(np.zeros(int(np.prod(shape))))
    out = np.concatenate(parts).astype(np.float32)
    out[-1] = 2.0
    return out


def train(feat, logt, tau: float = 0.9, steps: int = 20000, batch: int = 8192,
          lr: float = 1e-3, seed: int = 0, r_max: float = 0.98, log=None):
    """GPU training with the library's kernels; returns (master FP32 tensor,
    BF16 tensor, loss history).  Targets are clipped at r_max < 1: rows
    with r = 1 would otherwise pull z to +infinity; the calibrated margin
    restores their capacity (cap is clamped to ub anyway)."""
    import torch
    dev = feat.device
    logt = torch.clamp(logt, max=float(np.log(r_max))).contiguous()
    h = api.Handle()
    master = torch.from_numpy(init_master(seed)).to(dev)
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    params = torch.empty(api.MLP_PARAMS, dtype=torch.bfloat16, device=dev)
    h.mlp_to_bf16(master, params)
    n = int(feat.shape[0])
    batch = min(batch, n)
    ws = torch.empty(h.mlp_train_workspace_size(batch), dtype=torch.uint8, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    hist = []
    perm, pos = torch.randperm(n, device=dev, generator=g), 0
    for step in range(1, steps + 1):
        if pos + batch > n:
            perm, pos = torch.randperm(n, device=dev, generator=g), 0
        idx = perm[pos:pos + batch]
        pos += batch
        grad, loss = h.mlp_grad(feat[idx].contiguous(), logt[idx].contiguous(), tau, params, ws)
        # cosine decay to lr / 20
        lr_t = lr * (0.05 + 0.95 * 0.5 * (1 + np.cos(np.pi * (step - 1) / steps)))
        h.mlp_adam(master, m, v, grad, params, lr_t, step)
        if step % 1000 == 0 or step == steps:
            hist.append((step, float(loss.item())))
            if log:
                log(f"step {step} loss {hist[-1][1]:.5f}")
    return master, params, hist


def predict_r(h: api.Handle, feat, params):
    import torch
    return torch.sigmoid(h.mlp_forward(feat, params).double())


def calibrate_margin(h, feat, ub, nnz, params, overflow: float = 0.02,
                     learned_max: int = 2048) -> float:
    """Smallest margin m (to 1e-3) with at most `overflow` of the rows whose
    capacity fits learned_max overflowing cap = ceil(ub r m)."""
    import torch
    r = predict_r(h, feat, params)
    ubd, nzd = ub.double(), nnz.double()
    lo, hi = 0.5, 8.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        cap = torch.clamp(torch.ceil(ubd * r * mid), min=1.0)
        cap = torch.minimum(cap, ubd)
        sel = cap <= learned_max
        frac = float(((nzd > cap) & sel).sum().item()) / max(int(sel.sum().item()), 1)
        if frac <= overflow:
            hi = mid
        else:
            lo = mid
    return float(np.ceil(hi * 1000) / 1000)


def save(stem: str, master, meta: Dict) -> None:
    os.makedirs(os.path.dirname(stem) or ".", exist_ok=True)
    raw = master.detach().cpu().numpy().astype("<f4").tobytes()
    meta = dict(meta)
    meta.update({"format": "spgemm-row-nnz-mlp/1", "n_params": api.MLP_PARAMS,
                 "layout": "W1[64][4] b1[64] W2[64][64] b2[64] W3[64] b3, float32 LE",
                 "features": "log1p(nnz(A_i), ub_i, max_k nnz(B_k), mean_k nnz(B_k))",
                 "sha256": hashlib.sha256(raw).hexdigest()})
    with open(stem + ".bin", "wb") as f:
        f.write(raw)
    with open(stem + ".json", "w") as f:
        json.dump(meta, f, indent=1, sort_keys=True)


def load(stem: str = DEFAULT_STEM, device="cuda", handle: Optional[api.Handle] = None):
    """(BF16 parameter tensor on `device`, metadata dict); checks the hash."""
    import torch
    with open(stem + ".json") as f:
        meta = json.load(f)
    with open(stem + ".bin", "rb") as f:
        raw = f.read()
    if hashlib.sha256(raw).hexdigest() != meta["sha256"]:
        raise ValueError(f"{stem}.bin does not match the hash in its header")
    master = torch.from_numpy(np.frombuffer(raw, dtype="<f4").copy()).to(device)
    if master.numel() != api.MLP_PARAMS:
        raise ValueError("parameter count mismatch")
    params = torch.empty(api.MLP_PARAMS, dtype=torch.bfloat16, device=device)
    (handle or api.Handle()).mlp_to_bf16(master, params)
    torch.cuda.synchronize()
    return params, meta


def main(argv=None):
    ap = argparse.ArgumentParser(description="train the output-size network on the GPU")
    ap.add_argument("--out", default=DEFAULT_STEM)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--tau", type=float, default=0.9)
    ap.add_argument("--overflow", type=float, default=0.02)
    ap.add_argument("--small", action="store_true", help="small generator sizes (quick check)")
    args = ap.parse_args(argv)
    import torch
    t0 = time.time()
    log = lambda s: print(f"[{time.time() - t0:7.1f}s] {s}", flush=True)   # noqa: E731
    feat, logt, ub, nnz = collect(TRAIN_SEEDS if not args.small else TRAIN_SEEDS[:2],
                                  args.small, log)
    vf, vl, vub, vnnz = collect(VALID_SEEDS, args.small, log)
    log(f"train rows {feat.shape[0]}, valid rows {vf.shape[0]}")
    master, params, hist = train(feat, logt, tau=args.tau, steps=args.steps, log=log)
    h = api.Handle()
    margin = calibrate_margin(h, vf, vub, vnnz, params, overflow=args.overflow)
    r = predict_r(h, vf, params)
    ubd, nzd = vub.double(), vnnz.double()
    cap = torch.minimum(torch.clamp(torch.ceil(ubd * r * margin), min=1.0), ubd)
    lm = 2048
    sel_ub, sel_nn = ubd <= lm, cap <= lm
    stats = {"valid_rows": int(vf.shape[0]),
             "learned_rows_ub_sized": int(sel_ub.sum().item()),
             "learned_rows_network": int(sel_nn.sum().item()),
             "overflow_frac_network": float(((nzd > cap) & sel_nn).sum().item()
                                            / max(int(sel_nn.sum().item()), 1)),
             "staging_over_nnz_ub_sized": float(ubd[sel_ub].sum().item()
                                                / max(nzd[sel_ub].sum().item(), 1.0)),
             "staging_over_nnz_network": float(cap[sel_nn].sum().item()
                                               / max(nzd[sel_nn].sum().item(), 1.0))}
    gens = sorted({name for seed in TRAIN_SEEDS[:2 if args.small else None]
                   for name, _, _ in _names(seed, args.small)})
    meta = {"tau": args.tau, "margin": margin, "exact_max_ub": EXACT_MAX_UB,
            "overflow_target": args.overflow, "steps": args.steps,
            "train_seeds": list(TRAIN_SEEDS), "valid_seeds": list(VALID_SEEDS),
            "train_rows": int(feat.shape[0]), "loss_history": hist[-5:],
            "generators": gens, "small": bool(args.small), "validation": stats,
            "gpu": torch.cuda.get_device_name()}
    save(args.out, master, meta)
    log(json.dumps({"margin": margin, **stats}))


if __name__ == "__main__":
    main()
