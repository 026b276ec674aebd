"""Pins of the CPU reference of the output-size network (oracle/mlp.py):
bfloat16 rounding of hand-picked values, a network with a closed-form output,
pinball-loss special cases, central finite differences of every gradient,
Adam's first step, and row features of a hand-made product."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2504_06408_gb300 import inputs as I


def test_bf16_rounding_hand_values():
    u = 2.0 ** -7                       # bf16 spacing at 1
    cases = {
        1.0: 1.0,
        1 + u / 2: 1.0,                 # tie -> even (1.0)
        1 + u + u / 2: 1 + 2 * u,       # tie -> even (1 + 2u)
        1 + u / 2 + 2.0 ** -20: 1 + u,  # above the tie -> up
        -(1 + u / 2): -1.0,
        np.pi: 3.140625,                # 1.1001001b x 2
        0.0: 0.0,
        2.0 ** -130: 2.0 ** -130,       # subnormal, exact
    }
    got = mlp.bf16(np.array(list(cases)))
    assert np.array_equal(got, np.array(list(cases.values())))


def _identity_net(w3=(1.0, 2.0, 3.0, 4.0), b3=0.5):
    d = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    d["W1"][:4, :4] = np.eye(4)
    d["W2"][:4, :4] = np.eye(4)
    d["W3"][:4] = w3
    d["b3"][0] = b3
    return mlp.pack(d)


def test_forward_closed_form():
    p = _identity_net()
    feat = np.array([[0.3, 1.7, 2.2, 0.1], [-1.0, 0.5, -2.0, 3.0], [0.0, 0.0, 0.0, 0.0]])
    z64, _ = mlp.forward(p, feat, bf16_mode=False)
    exp64 = np.maximum(feat, 0) @ np.array([1.0, 2.0, 3.0, 4.0]) + 0.5
    assert np.allclose(z64, exp64, rtol=0, atol=1e-15)
    zbf, _ = mlp.forward(p, feat, bf16_mode=True)
    expbf = mlp.bf16(np.maximum(feat, 0)) @ np.array([1.0, 2.0, 3.0, 4.0]) + 0.5
    assert np.allclose(zbf, expbf, rtol=0, atol=1e-15)
    assert mlp.N_PARAMS == 4545


def test_pinball_special_cases():
    u = np.array([2.0, -2.0, 0.0])
    assert np.allclose(mlp.pinball(u, 0.5), 0.5 * np.abs(u))
    assert np.allclose(mlp.pinball(u, 0.9), [1.8, 0.2, 0.0])
    # log sigmoid: closed values and no overflow at large |z|
    assert np.isclose(mlp.log_sigmoid(0.0), -np.log(2.0))
    assert np.isclose(mlp.log_sigmoid(-800.0), -800.0)
    assert mlp.log_sigmoid(800.0) == 0.0


def _random_problem(seed, n=50):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, mlp.N_PARAMS)
    feat = rng.uniform(0, 4, (n, 4))
    logt = np.log(rng.uniform(0.05, 1.0, n))
    return p, feat, logt


def test_gradient_matches_central_differences():
    p, feat, logt = _random_problem(11)
    tau = 0.8
    L, g, bound = mlp.loss_and_grad(p, feat, logt, tau, bf16_mode=False)
    assert np.isclose(L, mlp.loss(p, feat, logt, tau, bf16_mode=False))
    eps = 1e-6
    fd = np.empty_like(p)
    for j in range(p.size):
        q = p.copy()
        q[j] += eps
        lp = mlp.loss(q, feat, logt, tau, bf16_mode=False)
        q[j] -= 2 * eps
        lm = mlp.loss(q, feat, logt, tau, bf16_mode=False)
        fd[j] = (lp - lm) / (2 * eps)
    assert np.all(np.abs(g - fd) <= 1e-7 + 1e-5 * np.abs(g))
    assert np.all(np.abs(g) <= bound * (1 + 1e-12) + 1e-300)
    # every parameter group has a non-trivial gradient in this problem
    o = 0
    for name, shape in mlp.SHAPES:
        n = int(np.prod(shape))
        assert np.abs(g[o:o + n]).max() > 0, name
        o += n


def test_bf16_mode_equals_fp64_on_representable_values():
    # weights in multiples of 1/8 and integer features keep every activation an
    # integer multiple of 1/64 below 256: exact in bfloat16, so both modes agree
    rng = np.random.default_rng(5)
    p = rng.integers(-3, 4, mlp.N_PARAMS) / 8.0
    d = mlp.unpack(p)
    d["W2"] = rng.integers(-1, 2, d["W2"].shape) / 8.0
    p = mlp.pack(d)
    feat = rng.integers(0, 4, (20, 4)).astype(np.float64)
    z1, acts = mlp.forward(p, feat, bf16_mode=True)
    z2, _ = mlp.forward(p, feat, bf16_mode=False)
    for a in acts:
        assert np.array_equal(mlp.bf16(a), a)
    assert np.array_equal(z1, z2)
    logt = np.log(np.full(20, 0.5))
    _, g1, _ = mlp.loss_and_grad(p, feat, logt, 0.9, bf16_mode=True)
    _, g2, _ = mlp.loss_and_grad(p, feat, logt, 0.9, bf16_mode=False)
    assert np.array_equal(g1, g2)


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    w, m, v = mlp.adam_step(np.ones(4), np.zeros(4), np.zeros(4), g, lr=0.01, step=1)
    assert np.allclose(w[:3], 1 - 0.01 * np.sign(g[:3]), rtol=0, atol=1e-7)
    assert w[3] == 1.0
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_features_hand_example():
    # A = [[1 1], [0 0], [0 1]] (pattern), B rows of lengths 3 and 1
    A = I.CSR(3, 2, np.array([0, 2, 2, 3]), np.array([0, 1, 1], np.int32), None)
    B = I.CSR(2, 5, np.array([0, 3, 4]), np.array([0, 2, 4, 1], np.int32), None)
    f, ub = mlp.features(A, B)
    assert ub.tolist() == [4, 0, 1]
    assert np.allclose(f, np.log1p([[2, 4, 3, 2.0], [0, 0, 0, 0], [1, 1, 1, 1]]))


def test_features_ub_matches_row_upper_bounds():
    A = I.rmat(9, seed=3, dtype=None)
    f, ub = mlp.features(A, A)
    assert np.array_equal(ub, oracle.row_upper_bounds(A, A))
    assert np.allclose(np.expm1(f[:, 1]), ub)
    assert np.all(f[:, 2] >= f[:, 3] - 1e-12)      # max >= mean
