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
defined on a history of coefficient vectors c_0 .. c_7 (oldest first) through
its backward differences, each a single FP64 subtraction of the previous
order: d1_k = c_k - c_{k-1}, d2_k = d1_k - d1_{k-1}, d3_k = d2_k - d2_{k-1},
d4_k = d3_k - d3_{k-1}.  Eight blocks per coefficient:

* block 0: (c_7 - mu) * inv_sigma                  (the state),
* blocks 1, 2, 3: d1_7 * inv_s1, d2_7 * inv_s2, d3_7 * inv_s3,
* blocks 4..7: d4_7, d4_6, d4_5, d4_4, each * inv_s4,

each rounded to float32 and then to bf16 (both round-to-nearest-even), laid
out block-major in one row per history (the joint network sees every
coefficient) or as one row of 8 per coefficient (a network shared by all
coefficients).  The base forecast of c_8 is the cubic extrapolation
P = ((c_7 + d1_7) + d2_7) + d3_7; the network learns what it misses, the
next fourth difference: the training target for a next vector c_8 is
d4_8 * inv_s4 rounded to float32 (d1_8 = c_8 - c_7 and so on), and
``advance`` forms c_8 = P + s4 * y.  All FP64 operations are single roundings
in the order written.

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
NORM_ROWS = 7     # mu, inv_sigma, inv_s1, inv_s2, inv_s3, inv_s4, s4


def _diff(c):
    return c[1:] - c[:-1]


def stats(traj):
    """Normalisers of a coefficient trajectory (T x D, T >= 5): mean mu,
    population standard deviation sigma and the RMS s_k of the k-th backward
    differences (k = 1..4) of every coefficient; inv_* = 1/s, or 0 where
    s == 0.  Returns the NORM_ROWS x D array
    (mu, inv_sigma, inv_s1, inv_s2, inv_s3, inv_s4, s4)."""
    c = np.asarray(traj, dtype=np.float64)
    mu = c.mean(axis=0)
    sigma = np.sqrt(((c - mu) ** 2).mean(axis=0))

    def inv(s):
        out = np.zeros_like(s)
        nz = s > 0
        out[nz] = 1.0 / s[nz]
        return out
    rows = [mu, inv(sigma)]
    d = c
    for _ in range(4):
        d = _diff(d)
        s = np.sqrt((d * d).mean(axis=0))
        rows.append(inv(s))
    rows.append(s)
    return np.stack(rows)


def _differences(c):
    """Backward differences of a list of vectors: d[k][i] = k-th difference
    ending at c[i] (defined for i >= k)."""
    d = [list(c)]
    for k in range(1, 5):
        prev = d[k - 1]
        d.append([None] * k + [prev[i] - prev[i - 1] for i in range(k, len(c))])
    return d


def features(store, rows, norm, next_rows=None, per_coeff=False):
    """bf16 feature codes of the histories store[rows[b]] (rows: B x 8
    indices, oldest first): B x 8D (block-major per row) or, per coefficient,
    (B*D) x 8 (one row per coefficient); with next_rows, float32 targets
    (B x D)."""
    store = np.asarray(store, dtype=np.float64)
    rows = np.asarray(rows)
    mu, isg, is1, is2, is3, is4, _ = norm
    bsz, d = rows.shape[0], store.shape[1]
    x = np.zeros((bsz, HIST * d), dtype=np.uint16)
    tgt = np.zeros((bsz, d), dtype=np.float32) if next_rows is not None else None
    for b in range(bsz):
        c = [store[rows[b, k]] for k in range(HIST)]
        dd = _differences(c)
        blocks = [(c[7] - mu) * isg, dd[1][7] * is1, dd[2][7] * is2, dd[3][7] * is3]
        for k in (7, 6, 5, 4):
            blocks.append(dd[4][k] * is4)
        x[b] = bf16_bits(np.concatenate(blocks))
        if next_rows is not None:
            e = _differences(c + [store[next_rows[b]]])
            tgt[b] = (e[4][8] * is4).astype(np.float32)
    if per_coeff:
        x = x.reshape(bsz, HIST, d).transpose(0, 2, 1).reshape(bsz * d, HIST).copy()
    return x, tgt


def advance(ring, order, norm, y=None, coeffs=None):
    """Forecast (y given) or push (coeffs given) the next coefficient vector
    into the ring of HIST vectors.  order: slots oldest..newest.  Returns
    (new ring, new order, the vector written)."""
    ring = np.array(ring, dtype=np.float64, copy=True)
    order = list(order)
    if coeffs is not None:
        new = np.asarray(coeffs, dtype=np.float64).copy()
    else:
        c = [ring[order[k]] for k in range(HIST)]
        dd = _differences(c)
        base = ((c[7] + dd[1][7]) + dd[2][7]) + dd[3][7]
        new = base + norm[6] * np.asarray(y, dtype=np.float32).astype(np.float64)
    ring[order[0]] = new
    return ring, order[1:] + order[:1], new
