"""Deterministic plus-times mode (spg_tuning.deterministic): values summed in
the order of A's entries from -0, i.e. the sequential left fold the oracle
computes, so FP64 and FP32 results are bit-identical to the oracle's --
plain, batched, learned and host-API calls, every tier."""
import numpy as np
import pytest

import oracle
from _util import assert_pattern_equal
from paper_2504_06408_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2504_06408_gb300 import spgemm as api  # noqa: E402

from test_gpu_spgemm import TIERS, values_for  # noqa: E402

DET = {"deterministic": 1}


def bits(x):
    return np.ascontiguousarray(x).view(np.uint8)


def inputs(case, sr):
    if case == "rmat11":
        pat = I.rmat(11, seed=3, dtype=None)
        return values_for(sr, pat, 5), values_for(sr, pat, 6)
    if case == "er":
        pat = I.er(4096, 8, seed=2, dtype=None)
        return values_for(sr, pat, 1), values_for(sr, pat, 2)
    if case == "signed_zeros":
        # values 0 and -0 and cancelling pairs: signed zeros must come out as
        # the left fold gives them
        A = I.random_csr(300, 200, 0.05, 4, dtype=None, empty_row_frac=0.1)
        B = I.random_csr(200, 250, 0.05, 5, dtype=None)
        rng = np.random.default_rng(9)
        dt = api.IN_NP[sr]
        pick = np.array([0.0, -0.0, 1.5, -1.5, 2.0**-30], dtype=dt)
        return (A.with_values(pick[rng.integers(0, 5, A.nnz)]),
                B.with_values(pick[rng.integers(0, 5, B.nnz)]))
    lap = I.laplacian(64)
    if sr == api.PLUS_TIMES_F32:
        lap = lap.with_values(lap.val.astype(np.float32))
    return lap, lap


@pytest.mark.parametrize("tier", ["default", "all_warp", "all_block", "all_dense"])
@pytest.mark.parametrize("case", ["rmat11", "er", "signed_zeros", "laplacian"])
@pytest.mark.parametrize("sr", [api.PLUS_TIMES_F64, api.PLUS_TIMES_F32])
def test_deterministic_equals_oracle_bits(sr, case, tier):
    A, B = inputs(case, sr)
    h = api.Handle(tuning=dict(TIERS[tier], **DET))
    dA = api.DeviceCSR.from_host(A, val_dtype=api.IN_NP[sr])
    dB = api.DeviceCSR.from_host(B, val_dtype=api.IN_NP[sr])
    got = api.to_host(api.spgemm(sr, dA, dB, handle=h), sr)
    exp = oracle.spgemm(sr, A, B)
    assert_pattern_equal(got.rp, got.col, exp.rp, exp.col)
    assert np.array_equal(bits(got.val), bits(exp.val))


@pytest.mark.parametrize("form", ["batched", "learned", "host"])
def test_deterministic_other_forms(form):
    sr = api.PLUS_TIMES_F64
    A, B = inputs("rmat11", sr)
    exp = oracle.spgemm(sr, A, B)
    h = api.Handle(tuning=dict(DET, host_panel_bytes=64 << 10))
    if form == "host":
        rp, col, val, n = h.host_multiply(sr, A, B)
        assert np.array_equal(rp, exp.rp) and np.array_equal(col[:n], exp.col)
        assert np.array_equal(val[:n * 8], bits(exp.val))
        return
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float64)
    dB = api.DeviceCSR.from_host(B, val_dtype=np.float64)
    if form == "learned":
        got = api.to_host(api.learned_spgemm(sr, dA, dB, handle=h), sr)
        assert np.array_equal(got.col, exp.col)
        assert np.array_equal(bits(got.val), bits(exp.val))
        return
    As = [dA.rows(0, 700), dA.rows(700, 2048)]
    ws = torch.empty(h.workspace_size_batched(sr, As, [dB, dB]), dtype=torch.uint8, device="cuda")
    rps = [torch.empty(a.nrows + 1, dtype=torch.int64, device="cuda") for a in As]
    nnz = h.symbolic_batched(sr, As, [dB, dB], rps, ws)
    cols = [torch.empty(max(n, 1), dtype=torch.int32, device="cuda") for n in nnz]
    vals = [api.out_tensor(sr, max(n, 1)) for n in nnz]
    h.numeric_batched(sr, As, [dB, dB], rps, cols, vals, ws)
    h.check(ws)
    got = np.concatenate([v[:n].cpu().numpy() for v, n in zip(vals, nnz)])
    assert np.array_equal(bits(got), bits(exp.val))
