"""CPU reference of the learned output-size predictor -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module.  It shares no code with the CUDA library.

The paper sizes every output row with a symbolic pass (Section 2.1,
Gustavson row-wise SpGEMM); it has no learned component.  What is written out
here is the network the library uses to predict a row's output size, in the
plainest form: float64 numpy, whole-batch matrix products, no fusion.

Quantities, per output row i of C = A B:

* ub_i = sum_{k in cols(A_i)} nnz(B_k), the row's intermediate products;
* features f_i = log1p of (nnz(A_i), ub_i, max_k nnz(B_k), mean_k nnz(B_k))
  (max / mean over k in cols(A_i); 0 for an empty row);
* target r_i = nnz(C_i) / ub_i in (0, 1];
* network 4 -> 64 -> 64 -> 1 with ReLU, output z_i, prediction sigmoid(z_i);
* loss: mean over rows of the pinball (quantile tau) loss of u_i =
  log r_i - log sigmoid(z_i):  rho(u) = tau u for u > 0, (tau - 1) u else.

"BF16 mode" rounds what the GPU rounds: weights, features and both hidden
activations (after ReLU) to bfloat16, nearest-even; every sum stays float64
here (float32 on the GPU).  Gradients treat the rounding as the identity
(the GPU's convention).  Parameters are one flat vector in the order
W1[64][4] b1[64] W2[64][64] b2[64] W3[64] b3 (W[out][in]).

Pins (tests/test_oracle_mlp.py): central finite differences of the loss for
every gradient formula (float64 mode), a network whose output has a closed
form, pinball loss special cases, bfloat16 rounding of hand-picked values,
and features against per-row Python loops.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 4, 64
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)   # 4545


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even), returned as float64.  The
    value is first rounded to float32 (the GPU rounds float32 values)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def unpack(params) -> dict:
    p = np.asarray(params, dtype=np.float64).ravel()
    assert p.size == N_PARAMS
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def features(A, B):
    """(f [n, 4] float64, ub [n] int64) of C = A B from CSR arrays."""
    blen = np.diff(np.asarray(B.rp, dtype=np.int64))
    n = A.nrows
    f = np.zeros((n, 4))
    ub = np.zeros(n, dtype=np.int64)
    rp = np.asarray(A.rp, dtype=np.int64)
    col = np.asarray(A.col)
    for i in range(n):
        ks = col[rp[i]:rp[i + 1]]
        lens = blen[ks]
        na = ks.size
        s = int(lens.sum())
        mx = int(lens.max()) if na else 0
        f[i] = np.log1p([na, s, mx, s / na if na else 0.0])
        ub[i] = s
    return f, ub


def forward(params, feat, bf16_mode: bool = True):
    """z [n] and the activations (f, a1, h1, a2, h2) of the network."""
    W = unpack(params)
    r = bf16 if bf16_mode else (lambda x: np.asarray(x, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = (r(W[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    f = r(feat)
    a1 = f @ W1.T + b1
    h1 = r(np.maximum(a1, 0.0))
    a2 = h1 @ W2.T + b2
    h2 = r(np.maximum(a2, 0.0))
    z = h2 @ W3 + b3[0]
    return z, (f, a1, h1, a2, h2)


def log_sigmoid(z):
    z = np.asarray(z, dtype=np.float64)
    return -(np.maximum(-z, 0.0) + np.log1p(np.exp(-np.abs(z))))


def pinball(u, tau):
    u = np.asarray(u, dtype=np.float64)
    return np.where(u > 0, tau * u, (tau - 1.0) * u)


def loss(params, feat, log_target, tau, bf16_mode: bool = True) -> float:
    z, _ = forward(params, feat, bf16_mode)
    return float(np.mean(pinball(np.asarray(log_target, np.float64) - log_sigmoid(z), tau)))


def loss_and_grad(params, feat, log_target, tau, bf16_mode: bool = True):
    """(loss, grad [N_PARAMS], bound [N_PARAMS]).  bound is the same sum over
    rows with every term replaced by its absolute value: the scale against
    which a float32 evaluation of grad is compared."""
    W = unpack(params)
    r = bf16 if bf16_mode else (lambda x: np.asarray(x, dtype=np.float64))
    W2, W3 = r(W["W2"]), r(W["W3"])
    z, (f, a1, h1, a2, h2) = forward(params, feat, bf16_mode)
    n = z.shape[0]
    u = np.asarray(log_target, np.float64) - log_sigmoid(z)
    L = float(np.mean(pinball(u, tau)))
    drho = np.where(u > 0, tau, tau - 1.0)
    sig = 1.0 / (1.0 + np.exp(-z))
    dz = -drho * (1.0 - sig) / n                 # dL/dz (d log sigmoid / dz = 1 - sigmoid)
    g, b = {}, {}
    g["W3"], b["W3"] = dz @ h2, np.abs(dz) @ np.abs(h2)
    g["b3"], b["b3"] = np.array([dz.sum()]), np.array([np.abs(dz).sum()])
    da2 = np.outer(dz, W3) * (a2 > 0)
    g["W2"], b["W2"] = da2.T @ h1, np.abs(da2).T @ np.abs(h1)
    g["b2"], b["b2"] = da2.sum(0), np.abs(da2).sum(0)
    dh1 = da2 @ W2
    da1 = dh1 * (a1 > 0)
    g["W1"], b["W1"] = da1.T @ f, (np.abs(da2) @ np.abs(W2) * (a1 > 0)).T @ np.abs(f)
    g["b1"], b["b1"] = da1.sum(0), (np.abs(da2) @ np.abs(W2) * (a1 > 0)).sum(0)
    return L, pack(g), pack(b)


def adam_step(master, m, v, grad, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, bias-corrected): new (master, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return master - lr * mh / (np.sqrt(vh) + eps), m, v
