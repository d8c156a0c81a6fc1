"""Pins of the FP64 MLP oracle (oracle/mlp.py) against things other than
itself: exact bf16 codes and torch's own bf16 cast, brute-force loops,
central finite differences, the closed-form gradient of one linear layer, Adam
under a constant gradient, and exact polynomial coefficient histories."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_1406_4254_gb300 import inputs


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
    p = inputs.mlp_params(dims, seed=3)
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
    p = inputs.mlp_params(dims, seed=1) * 3.0
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
    p = inputs.mlp_params(dims, seed=4)
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
def _poly_store(t0, nvec, coef):
    """c_t = sum_k coef[k] t^k for t = t0 .. t0+nvec-1 (rows), exact in binary
    for the dyadic coefficients and small t used here."""
    ts = np.arange(t0, t0 + nvec, dtype=np.float64)[:, None]
    return sum(coef[k][None, :] * ts ** k for k in range(len(coef)))


def test_stats_closed_form():
    # c_t = a + b t (t = 0..T-1): mean a + b (T-1)/2, population variance
    # b^2 (T^2 - 1)/12, RMS first difference |b|, higher differences 0
    T = 9
    a = np.array([1.0, -2.0, 0.5])
    b = np.array([0.25, 0.0, -3.0])
    norm = mlp.stats(_poly_store(0, T, [a, b]))
    assert norm.shape == (mlp.norm_rows(1), 3)
    np.testing.assert_allclose(norm[0], a + b * (T - 1) / 2, rtol=1e-15)
    sig = np.abs(b) * np.sqrt((T * T - 1) / 12.0)
    np.testing.assert_allclose(norm[1], np.where(sig > 0, 1 / np.where(sig > 0, sig, 1), 0), rtol=1e-14)
    np.testing.assert_allclose(norm[2], np.where(b != 0, 1 / np.where(b != 0, np.abs(b), 1), 0), rtol=1e-14)
    assert np.all(norm[3:] == 0)


def test_stats_of_a_cubic():
    # c_t = d t^3: third difference 6d everywhere, fourth difference 0
    d = np.array([0.5, -0.125])
    norm = mlp.stats(_poly_store(0, 12, [0 * d, 0 * d, 0 * d, d]))
    np.testing.assert_allclose(norm[4], 1.0 / (6 * np.abs(d)), rtol=1e-15)
    assert np.all(norm[5] == 0) and np.all(norm[6] == 0)


def _norm(d, mu=0.5, isg=2.0, is1=4.0, is2=16.0, is3=0.5, is4=8.0, s4=0.125,
          beta=(0.0,) * 7, q=1.0):
    """Normaliser rows by hand; beta = 0 and q = 1 leave the cubic base and the
    plain next-fourth-difference target."""
    vals = (mu, isg, is1, is2, is3, is4, s4) + tuple(beta) + (q, 1.0 / q if q else 0.0)
    return np.array([[v] * d for v in vals], dtype=np.float64)


def test_features_of_cubic_history():
    # c_t = a + b t + c t^2 + e t^3: d1_t = b + c (2t-1) + e (3t^2-3t+1),
    # d2_t = 2c + 6e (t-1), d3 = 6e, d4 = 0
    a = np.array([1.0, -0.5])
    b = np.array([0.25, 0.125])
    c = np.array([0.0625, -0.03125])
    e = np.array([0.0078125, 0.015625])
    store = _poly_store(3, 9, [a, b, c, e])     # t = 3..11
    norm = _norm(2)
    rows = np.array([[0, 1, 2, 3, 4, 5, 6, 7]])
    x, tgt = mlp.features(store, rows, norm, next_rows=np.array([8]))
    v = mlp.bf16_value(x[0]).reshape(8, 2)
    t7 = 10.0
    c7 = a + b * t7 + c * t7 ** 2 + e * t7 ** 3
    np.testing.assert_array_equal(v[0], mlp.bf16_round((c7 - 0.5) * 2.0))
    np.testing.assert_array_equal(v[1], mlp.bf16_round((b + c * (2 * t7 - 1) + e * (3 * t7 ** 2 - 3 * t7 + 1)) * 4.0))
    np.testing.assert_array_equal(v[2], mlp.bf16_round((2 * c + 6 * e * (t7 - 1)) * 16.0))
    np.testing.assert_array_equal(v[3], mlp.bf16_round(6 * e * 0.5))
    assert np.all(v[4:] == 0) and np.all(tgt[0] == 0)
    # one row of eight per coefficient: the same values, coefficient-major
    xp, _ = mlp.features(store, rows, norm, per_coeff=True)
    vp = mlp.bf16_value(xp)
    assert vp.shape == (2, 8)
    for j in range(2):
        np.testing.assert_array_equal(vp[j], v[:, j])


def test_features_fourth_differences_and_target():
    # c_t = t^4 / 16: fourth difference 24/16 = 1.5 everywhere
    q = np.array([1.0 / 16.0])
    z = 0 * q
    store = _poly_store(0, 9, [z, z, z, z, q])
    x, tgt = mlp.features(store, np.arange(8)[None, :], _norm(1, is4=2.0),
                          next_rows=np.array([8]))
    v = mlp.bf16_value(x[0])
    np.testing.assert_array_equal(v[4:], [3.0] * 4)
    assert tgt[0, 0] == np.float32(3.0)


def test_features_row_order_matters():
    rng = np.random.default_rng(8)
    store = rng.normal(size=(12, 5))
    norm = mlp.stats(store)
    x1, _ = mlp.features(store, np.array([[0, 1, 2, 3, 4, 5, 6, 7]]), norm)
    x2, _ = mlp.features(store, np.array([[1, 0, 2, 3, 4, 5, 6, 7]]), norm)
    # swapping the two oldest vectors changes only the fourth differences
    # that reach back to c_1: d4_5 (block 6) and d4_4 (block 7)
    d = (x1[0] != x2[0]).reshape(8, 5).any(axis=1)
    assert list(d) == [False] * 6 + [True, True]


def test_advance_inverts_target():
    # forecasting with the exact target reproduces the next vector of a
    # quartic history (the cubic base misses exactly d4 = 24 q); s4 and
    # inv_s4 are powers of two so that s4 * y undoes the scaling exactly
    coef = [np.array([1.0, -0.5, 0.0]), np.array([0.25, 0.125, -1.0]),
            np.array([0.0625, -0.03125, 0.5]), np.array([0.0, 0.5, -0.25]),
            np.array([0.125, 0.0, 0.0625])]
    store = _poly_store(0, 9, coef)
    norm = _norm(3, is4=4.0, s4=0.25)
    _, tgt = mlp.features(store, np.arange(8)[None, :], norm, next_rows=np.array([8]))
    ring = store[:8].copy()
    order = list(range(8))
    ring2, order2, new = mlp.advance(ring, order, norm, y=tgt[0])
    np.testing.assert_array_equal(new, store[8])
    assert order2 == [1, 2, 3, 4, 5, 6, 7, 0] and np.array_equal(ring2[0], store[8])
    # with y = 0 the forecast is the cubic extrapolation 4c7 - 6c6 + 4c5 - c4
    _, _, base = mlp.advance(ring, order, norm, y=np.zeros(3))
    np.testing.assert_array_equal(base, 4 * store[7] - 6 * store[6] + 4 * store[5] - store[4])
    # pushing a given vector writes it into the oldest slot
    ring3, order3, _ = mlp.advance(ring2, order2, norm, coeffs=np.array([7.0, 8.0, 9.0]))
    assert order3 == [2, 3, 4, 5, 6, 7, 0, 1] and np.array_equal(ring3[1], [7.0, 8.0, 9.0])


def _windows(traj, norm):
    """Regressors and targets of every 9-vector window, from numpy's
    difference operator (independent of the oracle's difference lists)."""
    U, t = [], []
    for w in range(traj.shape[0] - 8):
        c = traj[w:w + 9]
        d1, d2, d3, d4 = (np.diff(c, n=k, axis=0) for k in (1, 2, 3, 4))
        # the history ends at c[7]: its k-th difference is the second-to-last
        u = [d1[-2] * norm[2], d2[-2] * norm[3], d3[-2] * norm[4],
             d4[-2] * norm[5], d4[-3] * norm[5], d4[-4] * norm[5], d4[-5] * norm[5]]
        U.append(np.stack(u))
        t.append(d4[-1] * norm[5])
    return np.stack(U), np.stack(t)


def test_linear_fit_is_the_least_squares_solution():
    # a smooth trajectory with noise: the fitted beta satisfies the ridged
    # normal equations of the windows' regressors, and moving beta in any
    # direction raises the residual sum of squares
    rng = np.random.default_rng(21)
    T, D = 70, 4
    ts = np.arange(T)[:, None]
    traj = (np.cos(0.3 * ts * rng.uniform(0.5, 1.5, size=(1, D))) + 1e-3 * ts
            + 1e-4 * rng.normal(size=(T, D)))
    norm = mlp.stats(traj)
    assert norm.shape == (mlp.norm_rows(1), D)
    U, t = _windows(traj, norm)
    for j in range(D):
        A, b, beta = U[:, :, j], t[:, j], norm[7:14, j]
        G = A.T @ A
        lhs = (G + mlp.RIDGE * np.trace(G) / 7 * np.eye(7)) @ beta
        np.testing.assert_allclose(lhs, A.T @ b, rtol=1e-7, atol=1e-9 * np.abs(A.T @ b).max())
        rss = np.sum((b - A @ beta) ** 2)
        assert norm[14, j] == pytest.approx(np.sqrt(rss / len(b)), rel=1e-9)
        for k in range(7):
            step = np.zeros(7)
            step[k] = 1e-3 * max(1.0, abs(beta[k]))
            assert np.sum((b - A @ (beta + step)) ** 2) > rss
            assert np.sum((b - A @ (beta - step)) ** 2) > rss


def test_linear_fit_predicts_a_sinusoid_exactly():
    # the fourth differences of cos(w t) obey d4_{t+1} = 2 cos(w) d4_t - d4_{t-1}:
    # a linear function of the regressors, so the fitted predictor's residual
    # vanishes and the forecast with y = 0 is the next value (which the cubic
    # base alone misses)
    w = np.array([0.7, 1.3, 2.1])
    T = 40
    traj = np.cos(np.arange(T)[:, None] * w[None, :])
    norm = mlp.stats(traj)
    assert np.all(norm[14] < 1e-6)
    ring = traj[20:28].copy()
    _, _, new = mlp.advance(ring, list(range(8)), norm, y=np.zeros(3))
    np.testing.assert_allclose(new, traj[28], atol=1e-9)
    cubic = 4 * traj[27] - 6 * traj[26] + 4 * traj[25] - traj[24]
    assert np.all(np.abs(cubic - traj[28]) > 1e-3)


def test_linear_fit_degenerate_cases():
    # a constant coefficient and a trajectory too short for a window
    traj = np.stack([np.full(12, 1.5), np.arange(12, dtype=np.float64) ** 2], axis=1)
    norm = mlp.stats(traj)
    assert np.all(norm[7:14, 0] == 0) and norm[14, 0] == 0 and norm[15, 0] == 0
    short = mlp.stats(traj[:8])
    assert np.all(short[7:14] == 0) and np.all(short[14] == 1) and np.all(short[15] == 1)


def test_cubic_base_interpolates_a_cubic_at_every_horizon():
    # a cubic trajectory sampled at stride 3: the base at s = k/3 is the
    # polynomial's value k steps after the newest sample
    coef = [np.array([0.5, -1.0]), np.array([0.25, 0.125]), np.array([-0.0625, 0.03125]),
            np.array([0.0078125, -0.00390625])]
    store = _poly_store(0, 40, coef)
    hist = [store[5 + 3 * i] for i in range(8)]        # t = 5, 8, ..., 26
    dd = mlp._differences(hist)
    for k in (1, 2, 3):
        p = mlp.cubic_base(hist[7], dd[1][7], dd[2][7], dd[3][7], k, 3)
        np.testing.assert_allclose(p, store[26 + k], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("stride", [2, 3, 4])
def test_strided_fit_predicts_a_sinusoid_at_every_horizon(stride):
    # cos(w t) sampled at any stride spans two dimensions, so every horizon's
    # next value is a linear function of the history: the fitted predictors
    # are exact, and the forecast with y = 0 reproduces the trajectory
    w = np.array([0.31, 0.57, 0.83])
    T = 12 * stride + 40
    traj = np.cos(np.arange(T)[:, None] * w[None, :])
    norm = mlp.stats(traj, stride=stride)
    assert norm.shape == (mlp.norm_rows(stride), 3)
    for k in range(1, stride + 1):
        assert np.all(norm[mlp._beta_row(k) + 7] < 1e-6), k
    t7 = 10 * stride
    ring = np.stack([traj[t7 - (7 - i) * stride] for i in range(8)])
    for k in range(1, stride + 1):
        _, _, new = mlp.advance(ring, list(range(8)), norm, y=np.zeros(3), stride=stride,
                                horizon=k, commit=False)
        np.testing.assert_allclose(new, traj[t7 + k], atol=1e-8)


def test_strided_targets_and_forecast_invert():
    # the features' target of horizon k and the forecast with y = target give
    # back the trajectory's vector k steps ahead (to rounding)
    rng = np.random.default_rng(23)
    stride, T, D = 3, 60, 5
    ts = np.arange(T)[:, None]
    traj = np.sin(0.2 * ts * rng.uniform(0.5, 1.5, size=(1, D))) + 1e-3 * rng.normal(size=(T, D))
    norm = mlp.stats(traj, stride=stride)
    t7 = 30
    rows = np.array([[t7 - (7 - i) * stride for i in range(8)]])
    nxt = np.array([[t7 + 1, t7 + 2, t7 + 3]])
    _, tg = mlp.features(traj, rows, norm, next_rows=nxt, per_coeff=True, stride=stride)
    assert tg.shape == (D, stride)
    _, tj = mlp.features(traj, rows, norm, next_rows=nxt, per_coeff=False, stride=stride)
    assert tj.shape == (1, stride * D)
    np.testing.assert_array_equal(tj.reshape(stride, D).T, tg)
    ring = traj[rows[0]]
    for k in range(1, stride + 1):
        _, _, new = mlp.advance(ring, list(range(8)), norm, y=tg[:, k - 1], stride=stride,
                                horizon=k, commit=False)
        scale = np.abs(norm[6] * norm[mlp._beta_row(k) + 7]).max()
        np.testing.assert_allclose(new, traj[t7 + k], atol=1e-6 * scale + 1e-15)
