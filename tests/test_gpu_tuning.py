"""Autotuner: tuning changes only speed, never C; the cache round-trips.

The tuned product is compared with the oracle element by element (not only
with the untuned CUDA product), for the tuning the descent picks and for
every corner of the search space."""
import itertools

import numpy as np
import pytest

import oracle
from _util import abs_csr, assert_pattern_equal, assert_values
from paper_2504_06408_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2504_06408_gb300 import autotune  # noqa: E402
from paper_2504_06408_gb300 import spgemm as api  # noqa: E402


def test_tuned_result_identical_and_cached(tmp_path):
    sr = api.MIN_PLUS_F32
    A = I.rmat(12, seed=3, dtype=np.float32)
    dA = api.DeviceCSR.from_host(A, val_dtype=np.float32)
    best = autotune.tune(sr, dA, dA, reps=1, sweeps=1)
    assert set(best) <= set(autotune.SPACE)
    ref = api.to_host(api.spgemm(sr, dA, dA, handle=api.Handle()), sr)
    got = api.to_host(api.spgemm(sr, dA, dA, handle=api.Handle(tuning=best or None)), sr)
    exp = oracle.spgemm(sr, A, A)
    assert_pattern_equal(got.rp, got.col, exp.rp, exp.col, f"tuned {best}")
    assert_values(sr, got.val, exp.val, what=f"tuned {best}")
    assert np.array_equal(ref.rp, got.rp) and np.array_equal(ref.col, got.col)
    assert np.array_equal(ref.val.view(np.uint32), got.val.view(np.uint32))
    path = str(tmp_path / "t.json")
    autotune.save(sr, "rmat12", best, path)
    assert autotune.load(sr, "rmat12", path) == best
    h = autotune.tuned_handle(sr, dA, dA, "rmat12", path)
    got2 = api.to_host(api.spgemm(sr, dA, dA, handle=h), sr)
    assert np.array_equal(ref.col, got2.col)


@pytest.mark.parametrize("sr", [api.PLUS_TIMES_F64, api.MIN_PLUS_F32, api.BOOL_OR_AND,
                                api.OVERLAP_I32])
def test_search_space_corners_match_oracle(sr):
    """Every combination of the smallest and largest candidate of each tuning
    field gives the oracle's C."""
    from test_gpu_spgemm import values_for
    pat = I.rmat(11, seed=31, dtype=None)
    A = values_for(sr, pat, 1)
    B = values_for(sr, pat, 2)
    exp = oracle.spgemm(sr, A, B)
    bound = oracle.spgemm(sr, abs_csr(A), abs_csr(B)).val if sr == api.PLUS_TIMES_F64 else None
    dA = api.DeviceCSR.from_host(A, val_dtype=api.IN_NP[sr])
    dB = api.DeviceCSR.from_host(B, val_dtype=api.IN_NP[sr])
    fields = sorted(autotune.SPACE)
    for corner in itertools.product(*[(autotune.SPACE[f][0], autotune.SPACE[f][-1])
                                      for f in fields]):
        tuning = dict(zip(fields, corner))
        got = api.to_host(api.spgemm(sr, dA, dB, handle=api.Handle(tuning=tuning)), sr)
        assert_pattern_equal(got.rp, got.col, exp.rp, exp.col, str(tuning))
        if sr == api.PLUS_TIMES_F64:
            assert_values(sr, got.val, exp.val, bound=bound, what=str(tuning))
        elif sr != api.BOOL_OR_AND:
            assert_values(sr, got.val, exp.val, what=str(tuning))
