"""Autotuner: tuning changes only speed, never C; the cache round-trips."""
import numpy as np
import pytest

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
    assert np.array_equal(ref.rp, got.rp) and np.array_equal(ref.col, got.col)
    assert np.array_equal(ref.val.view(np.uint32), got.val.view(np.uint32))
    path = str(tmp_path / "t.json")
    autotune.save(sr, "rmat12", best, path)
    assert autotune.load(sr, "rmat12", path) == best
    h = autotune.tuned_handle(sr, dA, dA, "rmat12", path)
    got2 = api.to_host(api.spgemm(sr, dA, dA, handle=h), sr)
    assert np.array_equal(ref.col, got2.col)
