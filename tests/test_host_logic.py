"""Host-side logic that needs no GPU: the autotuner's coordinate descent and
cache, the SUMMA grid cuts, the association of iterated products, the
sizing network's weight-file format, and the binding's tuning fields."""
import hashlib
import json

import numpy as np
import pytest

from paper_2504_06408_gb300 import autotune, iterate, summa
from paper_2504_06408_gb300 import spgemm as api


# ---- autotuner -------------------------------------------------------------------

SPACE = {"a": [1, 2, 3, 4], "b": [10, 20, 30], "c": [5, 6]}
DEFAULT = {"a": 1, "b": 10, "c": 5}


def separable_cost(opt):
    def cost(cfg):
        full = dict(DEFAULT, **cfg)
        return 10.0 + sum((full[f] - opt[f]) ** 2 for f in opt)
    return cost


def test_descent_finds_the_minimum_of_a_separable_cost():
    opt = {"a": 3, "b": 20, "c": 6}
    best = autotune.descend(separable_cost(opt), SPACE, {})
    assert dict(DEFAULT, **best) == opt


def test_descent_keeps_the_start_when_nothing_improves():
    calls = []

    def flat(cfg):
        calls.append(dict(cfg))
        return 5.0
    start = {"a": 2}
    assert autotune.descend(flat, SPACE, start, sweeps=3) == start
    # one timing of the start, then every other candidate once; no second sweep
    assert len(calls) == 1 + (len(SPACE["a"]) - 1) + len(SPACE["b"]) + len(SPACE["c"])


def test_descent_ignores_gains_below_one_percent():
    def cost(cfg):
        return 99.6 if cfg.get("b") == 20 else 100.0   # 0.4% better: noise
    assert autotune.descend(cost, SPACE, {}) == {}


def test_tuning_cache_round_trip_and_keys(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    t1, t2 = {"num_block_max_nnz": 4096}, {"dense_slab_cols": 8192}
    autotune.save(api.MIN_PLUS_F32, "rmat18", t1, path, device="GPU-X")
    autotune.save(api.BOOL_OR_AND, "rmat18", t2, path, device="GPU-X")
    assert autotune.load(api.MIN_PLUS_F32, "rmat18", path, device="GPU-X") == t1
    assert autotune.load(api.BOOL_OR_AND, "rmat18", path, device="GPU-X") == t2
    assert autotune.load(api.MIN_PLUS_F32, "rmat18", path, device="GPU-Y") is None
    assert autotune.load(api.MIN_PLUS_F32, "kmer", path, device="GPU-X") is None
    with open(path) as f:
        assert len(json.load(f)) == 2


def test_tuning_cache_survives_a_corrupt_file(tmp_path):
    path = str(tmp_path / "tuning.json")
    with open(path, "w") as f:
        f.write("{ not json")
    assert autotune.load(api.MIN_PLUS_F32, "x", path, device="G") is None
    autotune.save(api.MIN_PLUS_F32, "x", {"a": 1}, path, device="G")
    assert autotune.load(api.MIN_PLUS_F32, "x", path, device="G") == {"a": 1}


# ---- SUMMA grid ---------------------------------------------------------------------

@pytest.mark.parametrize("n,q", [(262144, 4), (10, 4), (3, 4), (0, 2), (7, 1)])
def test_even_cuts(n, q):
    c = summa.even_cuts(n, q)
    assert len(c) == q + 1 and c[0] == 0 and c[-1] == n
    sizes = np.diff(c)
    assert np.all(sizes >= 0) and sizes.max() - sizes.min() <= 1


# ---- iterated products --------------------------------------------------------------

class Expr:
    """Stand-in matrix that records how products were associated."""
    def __init__(self, s, w):
        self.s, self.w = s, w      # w = number of factors W

    def __repr__(self):
        return self.s


@pytest.fixture
def symbolic_ops(monkeypatch):
    calls = {"mul": 0, "add": 0}

    def mul(sr, x, y, handle=None):
        calls["mul"] += 1
        return Expr(f"({x}*{y})", x.w + y.w)

    def add(sr, x, y, handle=None):
        calls["add"] += 1
        return Expr(f"({x}+{y})", max(x.w, y.w))
    monkeypatch.setattr(iterate, "multiply", mul)
    monkeypatch.setattr(iterate, "add", add)
    monkeypatch.setattr(iterate.api, "Handle", lambda *a, **k: None)
    return calls


@pytest.mark.parametrize("k", list(range(1, 21)) + [64, 100])
def test_power_by_squaring(symbolic_ops, k):
    W = Expr("W", 1)
    R = iterate.power(api.MIN_PLUS_F32, W, k)
    assert R.w == k
    # floor(log2 k) squarings plus one product per further set bit
    assert symbolic_ops["mul"] == (k.bit_length() - 1) + (bin(k).count("1") - 1)


def test_power_association_is_fixed(symbolic_ops):
    W = Expr("W", 1)
    assert repr(iterate.power(api.MIN_PLUS_F32, W, 5)) == "(W*((W*W)*(W*W)))"
    assert repr(iterate.power(api.MIN_PLUS_F32, W, 6)) == "((W*W)*((W*W)*(W*W)))"


def test_hops_recurrence(symbolic_ops):
    W = Expr("W", 1)
    assert repr(iterate.hops(api.BOOL_OR_AND, W, 1)) == "W"
    assert repr(iterate.hops(api.BOOL_OR_AND, W, 3)) == "((W+(W*W))+((W+(W*W))*W))"
    assert symbolic_ops == {"mul": 2, "add": 2}


def test_iterate_rejects_bad_arguments():
    with pytest.raises(ValueError):
        iterate.power(api.MIN_PLUS_F32, None, 0)
    with pytest.raises(ValueError):
        iterate.hops(api.MIN_PLUS_F32, None, 0)
    with pytest.raises(ValueError):
        iterate.as_input(api.OVERLAP_I32, None)


# ---- sizing network weight file -----------------------------------------------------

def test_weight_file_header_and_hash_check(tmp_path):
    torch = pytest.importorskip("torch")
    from paper_2504_06408_gb300 import learned
    stem = str(tmp_path / "net")
    master = torch.arange(api.MLP_PARAMS, dtype=torch.float32) / 7.0
    learned.save(stem, master, {"margin": 1.02})
    with open(stem + ".json") as f:
        meta = json.load(f)
    raw = open(stem + ".bin", "rb").read()
    assert len(raw) == 4 * api.MLP_PARAMS and meta["n_params"] == api.MLP_PARAMS
    assert meta["sha256"] == hashlib.sha256(raw).hexdigest() and meta["margin"] == 1.02
    assert np.array_equal(np.frombuffer(raw, "<f4"), master.numpy())
    # a changed byte is caught before anything touches a device
    bad = bytearray(raw)
    bad[100] ^= 1
    open(stem + ".bin", "wb").write(bytes(bad))
    with pytest.raises(ValueError):
        learned.load(stem, device="cpu")


# ---- binding ------------------------------------------------------------------------

def test_set_tuning_rejects_unknown_fields():
    import ctypes

    class FakeLib:
        def spgemm_set_tuning(self, h, t):
            self.t = t._obj
            return 0

    h = api.Handle.__new__(api.Handle)
    h.lib, h._h = FakeLib(), ctypes.c_void_p()
    h.set_tuning(num_block_max_nnz=4096, deterministic=1)
    assert h.lib.t.num_block_max_nnz == 4096 and h.lib.t.deterministic == 1
    with pytest.raises(ValueError):
        h.set_tuning(num_block_max=4096)      # a misspelt field is not ignored
    with pytest.raises(ValueError):
        h.set_tuning(reserved=1)


def test_shipped_tuning_names_only_known_fields():
    """Every entry of the shipped GB300 tuning loads by its key and names only
    spg_tuning fields with positive values (Handle.set_tuning raises on an
    unknown name, which would stop the benchmark on the GPU)."""
    known = {name for name, _ in api.spg_tuning._fields_} - {"reserved"}
    with open(autotune.SHIPPED) as f:
        data = json.load(f)
    assert data
    for key, tuning in data.items():
        device, sr_name, tag = key.split("|")
        sr = next(k for k, v in api.SEMIRING_NAMES.items() if v == sr_name)
        assert autotune.load(sr, tag, autotune.SHIPPED, device=device) == tuning
        assert set(tuning) <= known, key
        assert all(isinstance(v, int) and v > 0 for v in tuning.values()), key
