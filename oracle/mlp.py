"""FP64 CPU oracle of the coefficient-forecasting MLP (the learned part).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone, never by the product
package.  Plain numpy in double precision; a matrix product is the only
library primitive used.  The paper has no learned component: this follows the
idea of reusing expansion coefficients over several time steps (temporal
softening, mentioned at the end of Sec. 4.1) and replaces plain reuse by a
forecast.

The network is a multilayer perceptron with tanh hidden layers and a linear
output layer, trained on the mean squared error with Adam (Kingma & Ba 2015,
Algorithm 1: bias-corrected first and second moment estimates).  Parameters
are one flat vector: for each layer i, W_i (d_i x d_{i+1}, row-major, input
index first) followed by b_i (d_{i+1}).

``quantize=True`` evaluates the network with the same rounding points as the
tensor-core kernels (bf16 operands of every matrix product, everything else
exact): weights, hidden activations entering a product and the back-propagated
error entering a product are rounded to bf16; sums stay in FP64 here.  With
``quantize=False`` the whole network is FP64.

Forecast features (``features``) and the forecast update (``advance``) are
defined on a history of eight true coefficient vectors c_0 .. c_7 (oldest
first) spaced ``stride`` steps apart, through its backward differences, each a
single FP64 subtraction of the previous order: d1_i = c_i - c_{i-1},
d2_i = d1_i - d1_{i-1}, d3_i = d2_i - d2_{i-1}, d4_i = d3_i - d3_{i-1}.
Eight blocks per coefficient:

* block 0: (c_7 - mu) * inv_sigma                  (the state),
* blocks 1, 2, 3: d1_7 * inv_s1, d2_7 * inv_s2, d3_7 * inv_s3,
* blocks 4..7: d4_7, d4_6, d4_5, d4_4, each * inv_s4,

each rounded to float32 and then to bf16 (both round-to-nearest-even), laid
out block-major in one row per history (the joint network sees every
coefficient) or as one row of 8 per coefficient (a network shared by all
coefficients); s_k are the RMS of the k-th differences at that spacing.  The
forecast of the vector k steps after c_7 (horizon k = 1..stride) starts from
the cubic through c_4..c_7 at s = k / stride of a spacing (Newton's backward
form): P_k = ((c_7 + s d1_7) + a2 d2_7) + a3 d3_7 with a2 = (s (s+1)) / 2,
a3 = (a2 (s+2)) / 3.  A linear predictor fitted to the trajectory for each
coefficient and horizon corrects it: its regressors u_0..u_6 are the blocks
1..7 in FP64 (before rounding), its target t_k = (c_{t+k} - P_k) * inv_s4,
and ``stats`` fits beta_k by least squares over every history of the
trajectory whose horizons lie inside it (normal equations with a ridge of
1e-12 times the mean diagonal; beta = 0 where the Gram matrix vanishes) and
records the RMS q_k of the residual t_k - beta_k . u (summed left to right).
The network learns what the fitted predictor misses: the training target of
horizon k is (t_k - beta_k . u) * inv_q_k rounded to float32, and
``advance`` forms P_k + s4 * (beta_k . u + q_k * y).  Without a history
beta = 0 and q = 1.  All FP64 operations are single roundings in the order
written.

Pins: ``tests/test_oracle_mlp.py`` (finite differences, closed forms of a
linear layer and of Adam under a constant gradient, brute-force loops, exact
bf16 codes and torch's bf16 cast, exact polynomial histories).
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------
# bf16
# ---------------------------------------------------------------------------
def bf16_bits(x) -> np.ndarray:
    """float64/float32 -> bf16 codes (uint16): round to float32, then to the
    nearest bf16 with ties to even (IEEE 754 roundTiesToEven on the 16 bits
    kept).  Finite inputs only."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = u + 0x7FFF + ((u >> 16) & 1)
    return (r >> 16).astype(np.uint16)


def bf16_value(bits) -> np.ndarray:
    """bf16 codes -> float64 values (exact)."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def bf16_round(x) -> np.ndarray:
    return bf16_value(bf16_bits(x))


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
def param_count(dims) -> int:
    return int(sum(dims[i] * dims[i + 1] + dims[i + 1] for i in range(len(dims) - 1)))


def unpack(params, dims):
    """Views (W_i, b_i) of the flat parameter vector."""
    out, o = [], 0
    for i in range(len(dims) - 1):
        a, b = dims[i], dims[i + 1]
        w = params[o:o + a * b].reshape(a, b)
        o += a * b
        bias = params[o:o + b]
        o += b
        out.append((w, bias))
    return out


# ---------------------------------------------------------------------------
# forward, loss, backward
# ---------------------------------------------------------------------------
def forward(params, dims, x, quantize=False):
    """Returns (y, cache).  x: (B, d_0) values (already bf16 values when the
    inputs come from ``features``)."""
    q = bf16_round if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    layers = unpack(np.asarray(params, dtype=np.float64), dims)
    a_in = q(x)                     # operand of the first product
    cache = {"a_in": [a_in], "h": []}
    h = None
    for i, (w, b) in enumerate(layers):
        z = a_in @ q(w) + b
        if i == len(layers) - 1:
            return z, cache
        h = np.tanh(z)
        cache["h"].append(h)
        a_in = q(h)
        cache["a_in"].append(a_in)
    raise AssertionError("unreachable")


def loss_grad(params, dims, x, target, quantize=False):
    """Mean squared error over all B x d_L outputs and its gradient with
    respect to the flat parameter vector."""
    q = bf16_round if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    params = np.asarray(params, dtype=np.float64)
    layers = unpack(params, dims)
    y, cache = forward(params, dims, x, quantize)
    bsz, dout = y.shape
    diff = y - np.asarray(target, dtype=np.float64)
    loss = float(np.sum(diff * diff) / (bsz * dout))
    dz = 2.0 * diff / (bsz * dout)
    grads = []
    for i in range(len(layers) - 1, -1, -1):
        w, _ = layers[i]
        dzq = q(dz)
        gw = cache["a_in"][i].T @ dzq
        gb = dz.sum(axis=0)
        grads.append((gw, gb))
        if i > 0:
            dh = dzq @ q(w).T
            h = cache["h"][i - 1]
            dz = dh * (1.0 - h * h)
    grads.reverse()
    g = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, g


def adam(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t >= 1), returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grads
    v = beta2 * v + (1.0 - beta2) * grads * grads
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ---------------------------------------------------------------------------
# forecast glue
# ---------------------------------------------------------------------------
HIST = 8
LIN_FEAT = 7
RIDGE = 1e-12


def norm_rows(stride):
    """Rows of the normaliser array: 7 scales, then 9 per horizon."""
    return 7 + 9 * stride


def _beta_row(k):
    return 7 + 9 * (k - 1)


def _inv(s):
    out = np.zeros_like(s)
    nz = s > 0
    out[nz] = 1.0 / s[nz]
    return out


def stats(traj, stride=1):
    """Normalisers of a coefficient trajectory (T x D, T >= 5): mean mu,
    population standard deviation sigma and the RMS s_k of the k-th backward
    differences at spacing ``stride`` (k = 1..4, over every index where they
    exist) of every coefficient; inv_* = 1/s, or 0 where s == 0; then per
    horizon the fitted linear predictor (see the module notes).  Returns the
    norm_rows(stride) x D array (mu, inv_sigma, inv_s1..inv_s4, s4, then per
    horizon k: beta_k[0..6], q_k, inv_q_k)."""
    c = np.asarray(traj, dtype=np.float64)
    T, D = c.shape
    mu = c.mean(axis=0)
    sigma = np.sqrt(((c - mu) ** 2).mean(axis=0))
    rows = [mu, _inv(sigma)]
    d = c
    for _ in range(4):
        d = d[stride:] - d[:-stride]
        s = np.sqrt((d * d).mean(axis=0)) if len(d) else np.zeros(D)
        rows.append(_inv(s))
    rows.append(s)
    norm = np.concatenate([np.stack(rows), np.zeros((norm_rows(stride) - 7, D))])
    _fit_linear(c, stride, norm)
    return norm


def _regressors(dd, norm):
    """The regressors u_0..u_6 of a history (differences at c_7)."""
    is1, is2, is3, is4 = norm[2], norm[3], norm[4], norm[5]
    return [dd[1][7] * is1, dd[2][7] * is2, dd[3][7] * is3,
            dd[4][7] * is4, dd[4][6] * is4, dd[4][5] * is4, dd[4][4] * is4]


def _lin_predict(u, norm, k):
    b = _beta_row(k)
    s = norm[b] * u[0]
    for i in range(1, LIN_FEAT):
        s = s + norm[b + i] * u[i]
    return s


def cubic_base(c7, d1, d2, d3, k, stride):
    """The cubic through the history's last four vectors, k/stride of a
    spacing after c_7."""
    s = float(k) / float(stride)
    a2 = (s * (s + 1.0)) * 0.5
    a3 = (a2 * (s + 2.0)) / 3.0
    return ((c7 + s * d1) + a2 * d2) + a3 * d3


def _fit_linear(c, stride, norm):
    """Per horizon k = 1..stride: beta_k from the normal equations over every
    history with its horizons inside the trajectory, then q_k and 1/q_k."""
    T, D = c.shape
    ts = list(range((HIST - 1) * stride, T - stride))
    for k in range(1, stride + 1):
        b = _beta_row(k)
        if not ts:
            norm[b:b + 7] = 0.0
            norm[b + 7] = 1.0
            norm[b + 8] = 1.0
            continue
        U = np.zeros((len(ts), LIN_FEAT, D))
        tg = np.zeros((len(ts), D))
        for w, t in enumerate(ts):
            hist = [c[t - (HIST - 1 - i) * stride] for i in range(HIST)]
            dd = _differences(hist)
            U[w] = np.stack(_regressors(dd, norm))
            base = cubic_base(hist[7], dd[1][7], dd[2][7], dd[3][7], k, stride)
            tg[w] = (c[t + k] - base) * norm[5]
        for j in range(D):
            G = U[:, :, j].T @ U[:, :, j]
            h = U[:, :, j].T @ tg[:, j]
            tr = np.trace(G)
            beta = np.zeros(LIN_FEAT)
            if tr > 0:
                beta = np.linalg.solve(G + RIDGE * tr / LIN_FEAT * np.eye(LIN_FEAT), h)
            norm[b:b + 7, j] = beta
        r = np.stack([tg[w] - _lin_predict(U[w], norm, k) for w in range(len(ts))])
        q = np.sqrt((r * r).sum(axis=0) / len(ts))
        norm[b + 7] = q
        norm[b + 8] = _inv(q)


def _differences(c):
    """Backward differences of a list of vectors: d[k][i] = k-th difference
    ending at c[i] (defined for i >= k)."""
    d = [list(c)]
    for k in range(1, 5):
        prev = d[k - 1]
        d.append([None] * k + [prev[i] - prev[i - 1] for i in range(k, len(c))])
    return d


def features(store, rows, norm, next_rows=None, per_coeff=False, stride=1):
    """bf16 feature codes of the histories store[rows[b]] (rows: B x 8
    indices, oldest first): B x 8D (block-major per row) or, per coefficient,
    (B*D) x 8 (one row per coefficient); with next_rows (B x stride: the
    vectors 1..stride steps after each history), float32 targets, (B*D) x
    stride per coefficient or B x (stride*D) (horizon-major) jointly."""
    store = np.asarray(store, dtype=np.float64)
    rows = np.asarray(rows)
    mu, isg, is1, is2, is3, is4 = norm[:6]
    bsz, d = rows.shape[0], store.shape[1]
    x = np.zeros((bsz, HIST * d), dtype=np.uint16)
    tgt = np.zeros((bsz, stride, d), dtype=np.float32) if next_rows is not None else None
    for b in range(bsz):
        c = [store[rows[b, k]] for k in range(HIST)]
        dd = _differences(c)
        blocks = [(c[7] - mu) * isg, dd[1][7] * is1, dd[2][7] * is2, dd[3][7] * is3]
        for k in (7, 6, 5, 4):
            blocks.append(dd[4][k] * is4)
        x[b] = bf16_bits(np.concatenate(blocks))
        if next_rows is not None:
            u = _regressors(dd, norm)
            nr = np.asarray(next_rows).reshape(bsz, stride)
            for k in range(1, stride + 1):
                base = cubic_base(c[7], dd[1][7], dd[2][7], dd[3][7], k, stride)
                tk = (store[nr[b, k - 1]] - base) * is4
                tgt[b, k - 1] = ((tk - _lin_predict(u, norm, k)) * norm[_beta_row(k) + 8]).astype(np.float32)
    if per_coeff:
        x = x.reshape(bsz, HIST, d).transpose(0, 2, 1).reshape(bsz * d, HIST).copy()
        if tgt is not None:
            tgt = tgt.transpose(0, 2, 1).reshape(bsz * d, stride).copy()
    elif tgt is not None:
        tgt = tgt.reshape(bsz, stride * d)
    return x, tgt


def advance(ring, order, norm, y=None, coeffs=None, stride=1, horizon=1, commit=True):
    """Forecast at ``horizon`` (y given, one value per coefficient) or push
    (coeffs given) the next coefficient vector of the ring of HIST vectors.
    order: slots oldest..newest.  Returns (new ring, new order, the vector);
    with commit the vector is written into the oldest slot and order rotated."""
    ring = np.array(ring, dtype=np.float64, copy=True)
    order = list(order)
    if coeffs is not None:
        new = np.asarray(coeffs, dtype=np.float64).copy()
    else:
        c = [ring[order[k]] for k in range(HIST)]
        dd = _differences(c)
        base = cubic_base(c[7], dd[1][7], dd[2][7], dd[3][7], horizon, stride)
        lin = _lin_predict(_regressors(dd, norm), norm, horizon)
        yv = np.asarray(y, dtype=np.float32).astype(np.float64)
        new = base + norm[6] * (lin + norm[_beta_row(horizon) + 7] * yv)
    if not commit:
        return ring, order, new
    ring[order[0]] = new
    return ring, order[1:] + order[:1], new
