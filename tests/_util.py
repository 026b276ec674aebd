"""Shared test helpers: comparison of CSR results under the parity rules.

Parity rules: identical patterns always; bit-exact values for boolean,
min-plus, integer and overlap semirings; plus-times FP64 within
|g - o| <= 1e-12 * sum_k |a_ik * b_kj| per entry; plus-times FP32 within
2 * 2^-24 * (terms) * sum_k |a_ik * b_kj| (the first-order bound of a
recursive sum of that many float terms in any order).
"""
import numpy as np

import oracle

PT_F64_RTOL = 1e-12


def abs_csr(M):
    from types import SimpleNamespace
    return SimpleNamespace(nrows=M.nrows, ncols=M.ncols, rp=M.rp, col=M.col,
                           val=None if M.val is None else np.abs(M.val))


def assert_pattern_equal(got_rp, got_col, exp_rp, exp_col, what=""):
    got_rp = np.asarray(got_rp)
    exp_rp = np.asarray(exp_rp)
    if not np.array_equal(got_rp, exp_rp):
        bad = np.nonzero(got_rp != exp_rp)[0]
        raise AssertionError(f"{what}: row pointers differ at {bad[:10]} "
                             f"(got {got_rp[bad[:3]]}, expected {exp_rp[bad[:3]]})")
    got_col = np.asarray(got_col)
    exp_col = np.asarray(exp_col)
    if not np.array_equal(got_col, exp_col):
        bad = np.nonzero(got_col != exp_col)[0]
        raise AssertionError(f"{what}: column ids differ at {bad[:10]}")


def assert_values(sr, got, exp, bound=None, terms=None, what=""):
    """Compare value arrays under the semiring's parity rule.

    ``bound`` = sum_k |a_ik b_kj| per entry (plus-times only); ``terms`` = number
    of products per entry (plus-times FP32 only).
    """
    if sr == oracle.SR_BOOL:
        return
    got = np.asarray(got)
    exp = np.asarray(exp)
    assert got.shape == exp.shape, f"{what}: {got.shape} values, expected {exp.shape}"
    if got.size == 0:
        return
    if sr == oracle.SR_PT_F64:
        assert bound is not None
        err = np.abs(got - exp)
        lim = PT_F64_RTOL * bound
        bad = np.nonzero(~(err <= lim))[0]
        if bad.size:
            raise AssertionError(f"{what}: {bad.size} plus-times values beyond 1e-12 "
                                 f"(first {bad[:5]}, got {got[bad[:3]]}, exp {exp[bad[:3]]})")
    elif sr == oracle.SR_PT_F32:
        assert bound is not None and terms is not None
        err = np.abs(got.astype(np.float64) - exp.astype(np.float64))
        lim = 2.0 * 2.0**-24 * np.maximum(terms, 1) * bound.astype(np.float64)
        bad = np.nonzero(~(err <= lim))[0]
        if bad.size:
            raise AssertionError(f"{what}: {bad.size} fp32 plus-times values out of bound")
    else:
        if got.dtype.fields:
            same = np.ones(got.shape, bool)
            for f in got.dtype.names:
                same &= got[f] == exp[f]
        else:
            same = got.view(np.uint8).reshape(got.size, -1) == exp.view(np.uint8).reshape(exp.size, -1)
            same = same.all(axis=1)
        bad = np.nonzero(~same)[0]
        if bad.size:
            raise AssertionError(f"{what}: {bad.size} values not bit-identical "
                                 f"(first {bad[:5]}: got {got[bad[:3]]}, exp {exp[bad[:3]]})")
