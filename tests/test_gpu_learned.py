"""GPU tests of learned output sizing.

* the network's kernels against the CPU reference (oracle/mlp.py): row
  features, forward, gradient of the pinball loss, Adam step;
* the learned path's C against the plain path's C and the oracle, for every
  semiring, with no model (ub-sized capacities), a random model, capacities
  forced to 1 (every predicted row overflows and is redone exactly), and
  small learned limits (most rows exact);
* the trained network's gain over the ub-sized path on held-out inputs.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from _util import abs_csr, assert_pattern_equal, assert_values
from paper_2504_06408_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2504_06408_gb300 import spgemm as api  # noqa: E402
from paper_2504_06408_gb300 import learned  # noqa: E402

from test_gpu_spgemm import SR, values_for  # noqa: E402


def dev(sr, M):
    return api.DeviceCSR.from_host(M, val_dtype=api.IN_NP[sr])


def random_params(h, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    master_np = (rng.normal(0, scale, api.MLP_PARAMS)).astype(np.float32)
    master = torch.from_numpy(master_np).cuda()
    params = torch.empty(api.MLP_PARAMS, dtype=torch.bfloat16, device="cuda")
    h.mlp_to_bf16(master, params)
    torch.cuda.synchronize()
    return master_np, params


def gpu_features(h, A, B):
    dA, dB = api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(B)
    ws = torch.empty(h.workspace_size(api.BOOL_OR_AND, dA, dB), dtype=torch.uint8, device="cuda")
    feat, ub = h.row_features(dA, dB, ws)
    torch.cuda.synchronize()
    return feat.cpu().numpy(), ub.cpu().numpy()


# ---- network kernels vs the CPU reference -------------------------------------------

@pytest.mark.parametrize("case", ["rmat11", "er", "kmer_t", "ragged"])
def test_row_features_match_oracle(case):
    if case == "rmat11":
        A = B = I.rmat(11, seed=3, dtype=None)
    elif case == "er":
        A = B = I.er(1000, 8, seed=2, dtype=None)
    elif case == "kmer_t":
        A = I.kmer(800, 1 << 14, len_lo=10, len_hi=40, col_cap=16, seed=4)
        B = oracle.transpose(A, None)
    else:
        A = I.random_csr(333, 97, 0.05, 7, dtype=None, empty_row_frac=0.3)
        B = I.random_csr(97, 500, 0.02, 8, dtype=None, empty_row_frac=0.3)
    h = api.Handle()
    f, ub = gpu_features(h, A, B)
    ef, eub = omlp.features(A, B)
    assert np.array_equal(ub, eub)
    assert np.allclose(f, ef, rtol=1e-6, atol=1e-6)


def test_bf16_copy_rounds_like_reference():
    h = api.Handle()
    master_np, params = random_params(h, 1)
    got = params.float().cpu().numpy().astype(np.float64)
    assert np.array_equal(got, omlp.bf16(master_np))


def _real_features(n_rows_min=2000):
    A = I.rmat(12, seed=9, dtype=None)
    h = api.Handle()
    f, ub = gpu_features(h, A, A)
    keep = ub > 0
    return f[keep][:max(n_rows_min, 1)]


@pytest.mark.parametrize("seed", [1, 2])
def test_forward_matches_reference(seed):
    h = api.Handle()
    master_np, params = random_params(h, seed)
    feat = _real_features()
    z = h.mlp_forward(torch.from_numpy(feat).cuda(), params).cpu().numpy()
    ez, (f, a1, h1, a2, h2) = omlp.forward(master_np, feat, bf16_mode=True)
    W = omlp.unpack(master_np)
    scale = np.abs(h2) @ np.abs(omlp.bf16(W["W3"])) + abs(omlp.bf16(W["b3"])[0])
    assert np.all(np.abs(z - ez) <= 1e-3 * scale + 1e-6)


@pytest.mark.parametrize("tau", [0.5, 0.9])
def test_gradient_matches_reference(tau):
    h = api.Handle()
    master_np, params = random_params(h, 3, scale=0.2)
    feat = _real_features()
    rng = np.random.default_rng(4)
    logt = np.log(rng.uniform(0.02, 1.0, feat.shape[0])).astype(np.float32)
    grad, loss = h.mlp_grad(torch.from_numpy(feat).cuda(), torch.from_numpy(logt).cuda(), tau,
                            params)
    g = grad.cpu().numpy().astype(np.float64)
    eL, eg, bound = omlp.loss_and_grad(master_np, feat, logt, tau, bf16_mode=True)
    assert abs(float(loss.item()) - eL) <= 1e-3 * abs(eL) + 1e-6
    assert np.all(np.abs(g - eg) <= 1e-3 * bound + 1e-7 * bound.max())
    assert np.abs(eg).max() > 0


def test_adam_matches_reference():
    h = api.Handle()
    rng = np.random.default_rng(5)
    master = rng.normal(0, 0.5, api.MLP_PARAMS).astype(np.float32)
    m = np.zeros_like(master)
    v = np.zeros_like(master)
    dm, dmm, dv = (torch.from_numpy(x.copy()).cuda() for x in (master, m, v))
    params = torch.empty(api.MLP_PARAMS, dtype=torch.bfloat16, device="cuda")
    w64, m64, v64 = master.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step in range(1, 4):
        g = rng.normal(0, 1e-2, api.MLP_PARAMS).astype(np.float32)
        h.mlp_adam(dm, dmm, dv, torch.from_numpy(g).cuda(), params, 1e-3, step)
        w64, m64, v64 = omlp.adam_step(w64, m64, v64, g.astype(np.float64), 1e-3, step)
    torch.cuda.synchronize()
    assert np.allclose(dm.cpu().numpy(), w64, rtol=1e-6, atol=1e-6)
    assert np.allclose(dmm.cpu().numpy(), m64, rtol=1e-5, atol=1e-9)
    assert np.array_equal(params.float().cpu().numpy().astype(np.float64),
                          omlp.bf16(dm.cpu().numpy()))


# ---- learned path == plain path ------------------------------------------------------

def assert_matches_oracle(sr, got, A, B, what=""):
    exp = oracle.spgemm(sr, A, B)
    assert_pattern_equal(got.rp, got.col, exp.rp, exp.col, what)
    if sr == api.PLUS_TIMES_F64:
        bound = oracle.spgemm(sr, abs_csr(A), abs_csr(B))
        assert_values(sr, got.val, exp.val, bound=bound.val, what=what)
    elif sr == api.PLUS_TIMES_F32:
        a64 = A.with_values(np.abs(A.val).astype(np.float64))
        b64 = B.with_values(np.abs(B.val).astype(np.float64))
        bound = oracle.spgemm(oracle.SR_PT_F64, a64, b64)
        terms = oracle.spgemm(oracle.SR_OVERLAP, I.positions_csr(A, 1), I.positions_csr(B, 2))
        assert_values(sr, got.val, exp.val, bound=bound.val,
                      terms=terms.val["count"].astype(np.float64), what=what)
    elif sr != api.BOOL_OR_AND:
        assert_values(sr, got.val, exp.val, what=what)


def assert_same_c(sr, got, plain):
    assert np.array_equal(got.rp, plain.rp)
    assert np.array_equal(got.col, plain.col)
    if sr in (api.MIN_PLUS_F32, api.OVERLAP_I32, api.PLUS_TIMES_I64):
        assert np.array_equal(np.ascontiguousarray(got.val).view(np.uint8),
                              np.ascontiguousarray(plain.val).view(np.uint8))


MODES = {
    "ub_sized": dict(),
    "random_model": dict(model="random", margin=1.0, exact_max_ub=8),
    "capacity_one": dict(model="random", margin=1e-7, exact_max_ub=1),
    "mostly_exact": dict(learned_max=4),
    "small_limit": dict(learned_max=100, exact_max_ub=8, model="random", margin=2.0),
}


def run_learned(sr, dA, dB, h, mode):
    opts = dict(MODES[mode])
    if opts.get("model") == "random":
        opts["model"] = random_params(h, 11)[1]
    C = api.learned_spgemm(sr, dA, dB, handle=h, **opts)
    torch.cuda.synchronize()
    return api.to_host(C, sr), h.stats()


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("sr", SR)
def test_learned_equals_plain_rmat(sr, mode):
    pat = I.rmat(11, seed=3, dtype=None)
    A = values_for(sr, pat, 5)
    B = values_for(sr, pat, 6) if sr != api.OVERLAP_I32 else I.positions_csr(pat, 6)
    h = api.Handle()
    dA, dB = dev(sr, A), dev(sr, B)
    got, st = run_learned(sr, dA, dB, h, mode)
    plain = api.to_host(api.spgemm(sr, dA, dB, handle=h), sr)
    assert_same_c(sr, got, plain)
    assert_matches_oracle(sr, got, A, B, mode)
    nonempty = int(np.count_nonzero(np.diff(got.rp)))
    assert 0 <= st["learned_rows"] <= A.nrows
    if mode == "capacity_one":
        assert st["overflow_rows"] > nonempty // 2
    if mode == "ub_sized":
        assert st["overflow_rows"] == 0
        assert st["learned_rows"] >= nonempty      # ncols = 2048: every row fits the limit
    if mode == "mostly_exact":
        assert st["learned_rows"] < nonempty // 4


@pytest.mark.parametrize("sr", [api.MIN_PLUS_F32, api.BOOL_OR_AND, api.PLUS_TIMES_F64])
def test_learned_with_dense_exact_rows(sr):
    # 8192 columns: hub rows exceed the learned limit and go to the exact
    # path's dense tier (with the symbolic bitmap cache)
    pat = I.rmat(13, seed=4, dtype=None)
    A = values_for(sr, pat, 1)
    h = api.Handle()
    dA = dev(sr, A)
    got, st = run_learned(sr, dA, dA, h, "ub_sized")
    plain = api.to_host(api.spgemm(sr, dA, dA, handle=h), sr)
    assert_same_c(sr, got, plain)
    assert_matches_oracle(sr, got, A, A)
    assert st["learned_rows"] < int(np.count_nonzero(np.diff(got.rp)))


@pytest.mark.parametrize("mode", ["ub_sized", "capacity_one", "small_limit"])
def test_learned_kmer_overlap(mode):
    A = I.kmer(3000, 1 << 16, len_lo=20, len_hi=80, col_cap=16, seed=4)
    h = api.Handle()
    dA = api.DeviceCSR.from_host(A, val_dtype=np.int32)
    dAt = h.transpose(dA, 4)
    got, _ = run_learned(api.OVERLAP_I32, dA, dAt, h, mode)
    plain = api.to_host(api.spgemm(api.OVERLAP_I32, dA, dAt, handle=h), api.OVERLAP_I32)
    assert_same_c(api.OVERLAP_I32, got, plain)
    assert_matches_oracle(api.OVERLAP_I32, got, A, oracle.transpose(A, np.int32))


@pytest.mark.parametrize("shape", ["no_rows", "empty_rows", "one_row", "empty_b"])
def test_learned_edge_cases(shape):
    sr = api.MIN_PLUS_F32
    if shape == "no_rows":
        A, B = I.random_csr(0, 50, 0.1, 1, dtype=np.float32), I.random_csr(50, 40, 0.1, 2,
                                                                           dtype=np.float32)
    elif shape == "empty_rows":
        A = I.random_csr(100, 50, 0.0, 1, dtype=np.float32)
        B = I.random_csr(50, 40, 0.2, 2, dtype=np.float32)
    elif shape == "one_row":
        A = I.random_csr(1, 50, 0.5, 1, dtype=np.float32)
        B = I.random_csr(50, 4000, 0.3, 2, dtype=np.float32)
    else:
        A = I.random_csr(100, 50, 0.1, 1, dtype=np.float32)
        B = I.random_csr(50, 40, 0.0, 2, dtype=np.float32)
    h = api.Handle()
    for mode in ("ub_sized", "capacity_one"):
        got, _ = run_learned(sr, dev(sr, A), dev(sr, B), h, mode)
        assert_matches_oracle(sr, got, A, B, f"{shape} {mode}")


def test_learned_calls_need_a_plan():
    sr = api.MIN_PLUS_F32
    A = values_for(sr, I.rmat(8, seed=1, dtype=None), 1)
    dA = dev(sr, A)
    h = api.Handle()
    ws = torch.empty(h.learned_workspace_size(sr, dA, dA), dtype=torch.uint8, device="cuda")
    c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(api.SpgemmError) as e:
        h.learned_symbolic(sr, dA, dA, c_rp, ws, None)
    assert e.value.status == 1
    sb = h.learned_plan(sr, dA, dA, ws)
    assert sb > 0
    small = torch.empty(sb // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(api.SpgemmError) as e:
        h.learned_symbolic(sr, dA, dA, c_rp, ws, small)
    assert e.value.status == 8


@pytest.mark.parametrize("mode", ["ub_sized", "capacity_one"])
def test_learned_calls_repeat_after_one_plan(mode):
    """symbolic + numeric may run again on the same plan (e.g. new values of
    the same patterns): same C, same statistics."""
    sr = api.MIN_PLUS_F32
    pat = I.rmat(12, seed=5, dtype=None)
    A = values_for(sr, pat, 2)
    dA = dev(sr, A)
    h = api.Handle()
    opts = dict(MODES[mode])
    if opts.get("model") == "random":
        opts["model"] = random_params(h, 11)[1]
    ws = torch.empty(h.learned_workspace_size(sr, dA, dA), dtype=torch.uint8, device="cuda")
    sb = h.learned_plan(sr, dA, dA, ws, **opts)
    staging = torch.empty(max(sb, 1), dtype=torch.uint8, device="cuda")
    exp = oracle.spgemm(sr, A, A)
    seen = []
    for _ in range(3):
        c_rp = torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda")
        nnz = h.learned_symbolic(sr, dA, dA, c_rp, ws, staging)
        assert nnz == exp.nnz
        c_col = torch.empty(nnz, dtype=torch.int32, device="cuda")
        c_val = api.out_tensor(sr, nnz)
        h.learned_numeric(sr, dA, dA, c_rp, c_col, c_val, ws, staging)
        h.check(ws)
        got = api.to_host(api.DeviceCSR(A.nrows, A.ncols, c_rp, c_col, c_val), sr)
        assert_pattern_equal(got.rp, got.col, exp.rp, exp.col)
        assert_values(sr, got.val, exp.val)
        st = h.stats()
        seen.append((st["learned_rows"], st["overflow_rows"], st["learned_nnz"]))
    assert seen[0] == seen[1] == seen[2]


# ---- what the trained network gains ----------------------------------------------------

def _weights_or_skip():
    if not os.path.exists(learned.DEFAULT_STEM + ".json"):
        pytest.skip("no trained weights file in the package")
    return learned.load()


@pytest.mark.parametrize("case", ["rmat16_plus_times", "kmer_overlap", "laplacian_plus_times"])
def test_trained_network_gain(case):
    """Held-out inputs (the training generators and sizes at seeds outside
    the training set).  Both learned forms
    give the plain C.  With the trained network, at least as many rows skip
    the symbolic pass as with ub-sized capacities, its staging area holds at
    most as many unused slots per entry written, and few of its rows
    overflow."""
    params, meta = _weights_or_skip()
    if case == "rmat16_plus_times":
        sr = api.PLUS_TIMES_F64
        A = I.rmat(16, seed=1, dtype=np.float64)
        dA = dev(sr, A)
        dB = dA
    elif case == "kmer_overlap":
        sr = api.OVERLAP_I32
        A = I.kmer(20000, seed=1)
        dA = api.DeviceCSR.from_host(A, val_dtype=np.int32)
        dB = api.Handle().transpose(dA, 4)
    else:
        sr = api.PLUS_TIMES_F64
        A = I.laplacian(256)
        dA = dev(sr, A)
        dB = dA
    h = api.Handle()
    base = api.to_host(api.spgemm(sr, dA, dB, handle=h), sr)
    ub_c = api.to_host(api.learned_spgemm(sr, dA, dB, handle=h), sr)
    st_ub = h.stats()
    nn_c = api.to_host(api.learned_spgemm(sr, dA, dB, model=params, margin=meta["margin"],
                                          exact_max_ub=meta["exact_max_ub"], handle=h), sr)
    st_nn = h.stats()
    for got in (ub_c, nn_c):
        assert np.array_equal(got.rp, base.rp) and np.array_equal(got.col, base.col)
        if sr == api.OVERLAP_I32:
            assert np.array_equal(got.val.view(np.uint8), base.val.view(np.uint8))
        else:
            assert np.allclose(got.val, base.val, rtol=1e-12, atol=1e-12)
    predicted = st_nn["learned_rows"] + st_nn["overflow_rows"]
    assert st_nn["overflow_rows"] <= max(0.05 * predicted, 5)
    assert st_nn["learned_rows"] >= st_ub["learned_rows"] - st_nn["overflow_rows"]
    slack_ub = st_ub["staging_entries"] / max(st_ub["learned_nnz"], 1)
    slack_nn = st_nn["staging_entries"] / max(st_nn["learned_nnz"], 1)
    print(f"{case}: learned rows ub-sized {st_ub['learned_rows']} network {st_nn['learned_rows']}"
          f" (overflow {st_nn['overflow_rows']}); staging per entry {slack_ub:.3f} vs "
          f"{slack_nn:.3f}")
    if case == "kmer_overlap":
        assert st_nn["learned_rows"] > st_ub["learned_rows"]
        assert slack_nn < slack_ub
