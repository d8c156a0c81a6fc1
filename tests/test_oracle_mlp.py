"""Pins of the FP64 MLP oracle (oracle/mlp.py) against things other than
itself: exact bf16 codes and torch's own bf16 cast, brute-force loops,
central finite differences, the closed-form gradient of one linear layer, Adam
under a constant gradient, and exact polynomial coefficient histories."""
import numpy as np
import pytest
import torch

from oracle import mlp


# ---------------------------------------------------------------------------
# bf16 rounding
# ---------------------------------------------------------------------------
def test_bf16_exact_codes():
    one = 1.0
    cases = {
        1.0: 0x3F80,
        -2.5: 0xC020,
        one + 2.0 ** -8: 0x3F80,          # tie between 0x3F80 and 0x3F81 -> even
        one + 3 * 2.0 ** -8: 0x3F82,      # tie between 0x3F81 and 0x3F82 -> even
        one + 2.0 ** -7: 0x3F81,          # exact
        one + 2.0 ** -8 + 2.0 ** -20: 0x3F81,   # just above the tie
        0.0: 0x0000,
        2.0 ** -130: 0x0000 | (1 << 3),   # subnormal float32 kept exactly (bits 0x00080000)
        65280.0: 0x477F,                  # largest bf16 below 2^16
    }
    for v, code in cases.items():
        assert int(mlp.bf16_bits(np.array([v]))[0]) == code, (v, hex(int(mlp.bf16_bits(np.array([v]))[0])))


def test_bf16_matches_torch_cast():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-30, 30, 20000),
                        rng.normal(size=1000)]).astype(np.float32)
    ours = mlp.bf16_bits(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)
    np.testing.assert_array_equal(mlp.bf16_value(ours),
                                  torch.from_numpy(ref.view(np.int16)).view(torch.bfloat16)
                                  .to(torch.float64).numpy())


# ---------------------------------------------------------------------------
# forward / gradient
# ---------------------------------------------------------------------------
def test_forward_matches_loops():
    dims = [3, 4, 2]
    p = mlp.init_params(dims, seed=3)
    p[mlp.param_count(dims) - 2:] = [0.25, -0.5]          # nonzero output bias
    x = np.array([[0.5, -1.0, 2.0], [0.0, 0.25, -0.75]])
    (w1, b1), (w2, b2) = mlp.unpack(p, dims)
    y, _ = mlp.forward(p, dims, x)
    for b in range(2):
        h = [np.tanh(sum(x[b, i] * w1[i, j] for i in range(3)) + b1[j]) for j in range(4)]
        for k in range(2):
            yk = sum(h[j] * w2[j, k] for j in range(4)) + b2[k]
            assert abs(y[b, k] - yk) < 1e-15


def test_gradient_finite_differences():
    dims = [5, 4, 3, 2]
    rng = np.random.default_rng(0)
    p = mlp.init_params(dims, seed=1) * 3.0
    p += rng.normal(size=p.size) * 0.1                   # nonzero biases too
    x = rng.normal(size=(3, 5))
    t = rng.normal(size=(3, 2))
    _, g = mlp.loss_grad(p, dims, x, t)
    for i in range(p.size):
        h = 1e-5
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_grad(pp, dims, x, t)[0] - mlp.loss_grad(pm, dims, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-8 * max(1.0, abs(g[i])), i


def test_gradient_linear_layer_closed_form():
    dims = [6, 3]
    rng = np.random.default_rng(2)
    p = rng.normal(size=mlp.param_count(dims))
    x = rng.normal(size=(7, 6))
    t = rng.normal(size=(7, 3))
    w, b = p[:18].reshape(6, 3), p[18:]
    r = x @ w + b - t
    loss, g = mlp.loss_grad(p, dims, x, t)
    assert abs(loss - np.mean(r * r)) < 1e-13
    np.testing.assert_allclose(g[:18].reshape(6, 3), 2.0 / 21.0 * x.T @ r, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(g[18:], 2.0 / 21.0 * r.sum(axis=0), rtol=1e-12, atol=1e-14)


def test_quantized_equals_exact_on_bf16_representable_data():
    # one linear layer, dyadic operands and a residual whose scaled values
    # 2 r / (B D) are bf16-exact: the rounding points change nothing
    dims = [4, 2]
    w = np.array([[0.5, -0.25], [1.0, 0.125], [-2.0, 0.75], [0.0, 1.5]])
    p = np.concatenate([w.ravel(), [0.25, -0.5]])
    x = np.array([[1.0, 0.5, -0.25, 2.0], [0.0, -1.0, 0.5, 0.125]])
    y, _ = mlp.forward(p, dims, x)
    t = y - np.array([[0.5, -1.0], [2.0, 0.25]])
    l0, g0 = mlp.loss_grad(p, dims, x, t)
    l1, g1 = mlp.loss_grad(p, dims, x, t, quantize=True)
    assert l0 == l1 and np.array_equal(g0, g1)


def test_quantized_within_bf16_bound():
    dims = [16, 8, 4]
    rng = np.random.default_rng(4)
    p = mlp.init_params(dims, seed=4)
    x = mlp.bf16_round(rng.normal(size=(5, 16)))
    t = rng.normal(size=(5, 4))
    _, g0 = mlp.loss_grad(p, dims, x, t)
    _, g1 = mlp.loss_grad(p, dims, x, t, quantize=True)
    # each product operand carries a relative error <= 2^-9
    assert np.linalg.norm(g1 - g0) <= 8 * 2.0 ** -9 * np.linalg.norm(g0)
    assert not np.array_equal(g0, g1)


def test_adam_constant_gradient_closed_form():
    # with a constant gradient the bias-corrected moments are exactly g and
    # g^2, so every step moves by -lr g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    p = np.array([1.0, 2.0, 3.0])
    m = np.zeros(3)
    v = np.zeros(3)
    lr, eps = 0.01, 1e-8
    for t in range(1, 6):
        p, m, v = mlp.adam(p, g, m, v, t, lr, eps=eps)
    np.testing.assert_allclose(p, np.array([1.0, 2.0, 3.0]) - 5 * lr * g / (np.abs(g) + eps),
                               rtol=1e-13)


# ---------------------------------------------------------------------------
# forecast features and update
# ---------------------------------------------------------------------------
def _poly_store(t0, nvec, a, b, c):
    ts = np.arange(t0, t0 + nvec, dtype=np.float64)[:, None]
    return a[None, :] + b[None, :] * ts + c[None, :] * ts * ts


def test_stats_closed_form():
    # c_t = a + b t (t = 0..T-1): mean a + b (T-1)/2, population variance
    # b^2 (T^2 - 1)/12, RMS first difference |b|, second difference 0
    T = 9
    a = np.array([1.0, -2.0, 0.5])
    b = np.array([0.25, 0.0, -3.0])
    mu, inv_sigma, inv_s1, inv_s2, s2 = mlp.stats(_poly_store(0, T, a, b, np.zeros(3)))
    np.testing.assert_allclose(mu, a + b * (T - 1) / 2, rtol=1e-15)
    sig = np.abs(b) * np.sqrt((T * T - 1) / 12.0)
    np.testing.assert_allclose(inv_sigma, np.where(sig > 0, 1 / np.where(sig > 0, sig, 1), 0), rtol=1e-14)
    np.testing.assert_allclose(inv_s1, np.where(b != 0, 1 / np.where(b != 0, np.abs(b), 1), 0), rtol=1e-14)
    assert np.all(inv_s2 == 0) and np.all(s2 == 0)


def test_features_of_quadratic_history():
    # c_t = a + b t + c t^2: first difference b + c (2t - 1), every second
    # difference 2c (exact in binary for these dyadic values)
    a = np.array([1.0, -0.5])
    b = np.array([0.25, 0.125])
    c = np.array([0.0625, -0.03125])
    store = _poly_store(3, 9, a, b, c)          # t = 3..11
    mu = np.array([0.5, 0.25])
    inv_sigma = np.array([2.0, 0.5])
    inv_s1 = np.array([4.0, 8.0])
    inv_s2 = np.array([16.0, 2.0])
    rows = np.array([[0, 1, 2, 3, 4, 5, 6, 7]])
    x, tgt = mlp.features(store, rows, mu, inv_sigma, inv_s1, inv_s2, next_rows=np.array([8]))
    v = mlp.bf16_value(x[0]).reshape(8, 2)
    t7 = 10.0
    np.testing.assert_array_equal(v[0], mlp.bf16_round((a + b * t7 + c * t7 * t7 - mu) * inv_sigma))
    np.testing.assert_array_equal(v[1], mlp.bf16_round((b + c * (2 * t7 - 1)) * inv_s1))
    for k in range(2, 8):
        np.testing.assert_array_equal(v[k], 2 * c * inv_s2)
    np.testing.assert_array_equal(tgt[0], (2 * c * inv_s2).astype(np.float32))


def test_features_row_order_matters():
    rng = np.random.default_rng(8)
    store = rng.normal(size=(12, 5))
    st = mlp.stats(store)
    x1, _ = mlp.features(store, np.array([[0, 1, 2, 3, 4, 5, 6, 7]]), *st[:4])
    x2, _ = mlp.features(store, np.array([[1, 0, 2, 3, 4, 5, 6, 7]]), *st[:4])
    # swapping the two oldest vectors changes only the two oldest second
    # differences (blocks 6 and 7: c_3-2c_2+c_1 and c_2-2c_1+c_0)
    d = (x1[0] != x2[0]).reshape(8, 5).any(axis=1)
    assert list(d) == [False] * 6 + [True, True]


def test_advance_inverts_target():
    # forecasting with the exact target reproduces the next quadratic vector;
    # s2 and inv_s2 are powers of two so that s2 * y undoes the scaling exactly
    a = np.array([1.0, -0.5, 0.0])
    b = np.array([0.25, 0.125, -1.0])
    c = np.array([0.0625, -0.03125, 0.5])
    store = _poly_store(0, 9, a, b, c)
    inv_s2 = np.array([4.0, 0.5, 1.0])
    s2 = 1.0 / inv_s2
    _, tgt = mlp.features(store, np.arange(8)[None, :], np.zeros(3), np.ones(3), np.ones(3),
                          inv_s2, next_rows=np.array([8]))
    ring = store[:8].copy()
    order = list(range(8))
    ring2, order2, new = mlp.advance(ring, order, s2, y=tgt[0])
    np.testing.assert_array_equal(new, store[8])
    assert order2 == [1, 2, 3, 4, 5, 6, 7, 0] and np.array_equal(ring2[0], store[8])
    # pushing a given vector writes it into the oldest slot
    ring3, order3, _ = mlp.advance(ring2, order2, s2, coeffs=np.array([7.0, 8.0, 9.0]))
    assert order3 == [2, 3, 4, 5, 6, 7, 0, 1] and np.array_equal(ring3[1], [7.0, 8.0, 9.0])
