"""Coefficient forecasting for SCF time integration (the learned part).

The paper has no learned component.  It notes that the coefficients may be
kept over several steps (temporal softening, end of Sec. 4.1); here the
coefficient pass (the first SCF pass, Sec. 3.3) runs only every
``stride``-th step and the steps between use a forecast of the coefficients
from the last eight recomputed vectors: a cubic base, per-coefficient linear
predictors fitted to a training trajectory, and a small MLP trained on what
those miss.  Plain SCF remains the fallback and the check: on every
recompute step the forecast that step would have used is compared with the
recomputed coefficients through the relative acceleration error on a
particle sample, and a forecast that misses the force-error budget switches
the next block to plain SCF.

Everything numeric runs in ``libetics.so`` kernels (bf16 tensor-core
products, Adam, feature and update kernels); this module only orders the
calls and owns the buffers.

Typical use::

    traj = coefficient_trajectory(posm, vel, steps, dt, n_max, l_max)
    fc = Forecaster(n_max, l_max, stride=3, hidden=256)
    fc.fit(traj[:n_train], iters=2000, batch=256)
    fc.reset(traj)
    stats = run(posm, vel, acc, steps, dt, fc)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import etics, inputs

HIST = 8


class Mlp:
    """An MLP with tanh hidden layers trained by the library's kernels: FP32
    master parameters, their bf16 copy for the tensor-core products, Adam
    moments and gradients, all device-resident."""

    def __init__(self, dims, seed: int = 0, device="cuda"):
        self.dims = [int(d) for d in dims]
        self.n = etics.mlp_param_count(self.dims)
        p = inputs.mlp_params(self.dims, seed)
        self.params = torch.tensor(p, dtype=torch.float32, device=device)
        self.params_bf16 = torch.empty(self.n, dtype=torch.bfloat16, device=device)
        etics.mlp_to_bf16(self.dims, self.params, self.params_bf16)
        self.grads = torch.zeros(self.n, dtype=torch.float32, device=device)
        self.m = torch.zeros_like(self.grads)
        self.v = torch.zeros_like(self.grads)
        self.t = 0
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self._ws: dict = {}

    def ws(self, batch: int) -> torch.Tensor:
        buf = self._ws.get(batch)
        if buf is None:
            buf = etics.mlp_workspace(self.dims, batch, self.params.device)
            self._ws[batch] = buf
        return buf

    def forward(self, x: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
        return etics.mlp_forward(self.dims, self.params, self.params_bf16, x, y,
                                 ws=self.ws(x.shape[0]))

    def loss_grad(self, x: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
        etics.mlp_loss_grad(self.dims, self.params, self.params_bf16, x, target, self.grads,
                            self.loss, ws=self.ws(x.shape[0]))
        return self.loss

    def adam_step(self, lr: float, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
        self.t += 1
        etics.mlp_adam(self.dims, self.params, self.grads, self.m, self.v, self.t, lr,
                       self.params_bf16, beta1, beta2, eps)


class Forecaster:
    """Forecasts SCF coefficient vectors c[n][l*l+l+m] (flattened, D of them)
    for the ``stride`` steps after the newest vector of a history of eight true
    vectors spaced ``stride`` steps apart: in a rollout with one coefficient
    pass every ``stride`` steps those are the passes of the last eight
    recomputations, so no forecast ever enters a history (forecasts fed back
    into the history compound their errors from block to block).  Each
    horizon k = 1..stride has its own per-coefficient linear predictor fitted
    to the training trajectory; the network learns what those miss.

    per_coeff=True (default): one network shared by all coefficients maps a
    coefficient's own eight features to its ``stride`` corrections (HIST ->
    hidden -> ... -> stride, applied to D rows).  per_coeff=False: one network
    sees the features of every coefficient at once (HIST*D -> ... ->
    stride*D)."""

    def __init__(self, n_max: int, l_max: int, stride: int = 3, hidden: int = 256, layers: int = 3,
                 seed: int = 0, per_coeff: bool = True, device="cuda"):
        if not 1 <= stride <= 4:
            raise ValueError("stride must be 1..4")
        self.n_max, self.l_max, self.stride = n_max, l_max, int(stride)
        self.D = (n_max + 1) * (l_max + 1) ** 2
        self.per_coeff = per_coeff
        if per_coeff:
            dims = [HIST] + [hidden] * (layers - 1) + [self.stride]
        else:
            dims = [HIST * self.D] + [hidden] * (layers - 1) + [self.stride * self.D]
        self.net = Mlp(dims, seed=seed, device=device)
        self.device = torch.device(device)
        self.norm = torch.zeros((etics.norm_rows(self.stride), self.D), dtype=torch.float64,
                                device=device)
        self.ring = torch.zeros((HIST, self.D), dtype=torch.float64, device=device)
        self.order = torch.arange(HIST, dtype=torch.int32, device=device)
        self.x1 = self._x(1)
        self.y1 = torch.zeros((self._rows(1), dims[-1]), dtype=torch.float32, device=device)

    def _rows(self, hist: int) -> int:
        return hist * self.D if self.per_coeff else hist

    def _x(self, hist: int) -> torch.Tensor:
        shape = (hist * self.D, HIST) if self.per_coeff else (hist, HIST * self.D)
        return torch.empty(shape, dtype=torch.bfloat16, device=self.device)

    def _features(self, store, rows, nxt=None, x=None, tg=None):
        return etics.coeff_features(store, rows, self.norm, nxt, x, tg, per_coeff=self.per_coeff,
                                    stride=self.stride)

    def _history_rows(self, newest: np.ndarray) -> np.ndarray:
        return newest[..., None] + self.stride * np.arange(-HIST + 1, 1)

    # ---- training ------------------------------------------------------------
    def fit(self, traj: torch.Tensor, iters: int = 2000, batch: int = 256, lr: float = 1e-3,
            seed: int = 0, log_every: int = 0):
        """Trains on a (T, D) float64 trajectory: normalisers and fitted
        predictors from the whole of it, minibatches of ``batch`` histories
        (with their ``stride`` next vectors) drawn with a seeded generator,
        Adam with a cosine learning-rate decay.  Returns the loss every
        ``log_every`` iterations (a list of floats) when asked."""
        traj = traj.contiguous()
        T, S = traj.shape[0], self.stride
        lo, hi = (HIST - 1) * S, T - 1 - S
        if hi < lo:
            raise ValueError(f"need at least {HIST * S + 1} coefficient vectors")
        etics.coeff_stats(traj, S, self.norm)
        rng = np.random.Generator(np.random.Philox(key=[int(seed), 6]))
        last = rng.integers(lo, hi + 1, size=(iters, batch))           # newest history index
        rows = torch.tensor(self._history_rows(last), dtype=torch.int32, device=self.device)
        nxt = torch.tensor(last[:, :, None] + np.arange(1, S + 1), dtype=torch.int32,
                           device=self.device)
        x = self._x(batch)
        tshape = (batch * self.D, S) if self.per_coeff else (batch, S * self.D)
        tg = torch.empty(tshape, dtype=torch.float32, device=self.device)
        losses = []
        for it in range(iters):
            self._features(traj, rows[it], nxt[it], x, tg)
            loss = self.net.loss_grad(x, tg)
            self.net.adam_step(lr * 0.5 * (1.0 + math.cos(math.pi * it / iters)))
            if log_every and (it % log_every == 0 or it == iters - 1):
                losses.append(float(loss.item()))
        return losses

    def horizon_errors(self, traj: torch.Tensor, first: int) -> dict:
        """Forecast errors on true histories whose newest vector is traj[t],
        t >= first: for each horizon k, |c_hat - c_{t+k}| / |c_{t+k} - c_t|
        (arrays), for holding c_t, the cubic base, the fitted predictors and
        the network's forecast.  Evaluated through etics_coeff_advance."""
        T, S = traj.shape[0], self.stride
        newest = np.arange(max(first, (HIST - 1) * S), T - S)
        names = ("cubic", "fitted", "net")
        fore = torch.empty((len(newest), len(names), S, self.D), dtype=torch.float64,
                           device=self.device)
        saved = (self.ring.clone(), self.order.clone(), self.y1.clone())
        base_only = self.norm.clone()
        base_only[7:] = 0.0           # no fitted or network term: the cubic base
        for i, t in enumerate(newest):
            self.ring.copy_(traj[self._history_rows(np.array(t))])
            self.order.copy_(torch.arange(HIST, dtype=torch.int32))
            for n, name in enumerate(names):
                self.predict(net=name == "net")
                for k in range(1, S + 1):
                    etics.coeff_advance(self.ring, self.order,
                                        base_only if name == "cubic" else self.norm,
                                        y=self._y(k), coeffs_out=fore[i, n, k - 1], commit=False,
                                        stride=S, horizon=k, y_stride=self._y_stride())
        self.ring.copy_(saved[0])
        self.order.copy_(saved[1])
        self.y1.copy_(saved[2])
        idx = torch.tensor(newest, device=self.device)
        now = traj[idx]
        out = {}
        for k in range(1, S + 1):
            ref = traj[idx + k]
            step = (ref - now).norm(dim=1)
            out[k] = {"hold": ((now - ref).norm(dim=1) / step).cpu().numpy()}
            for n, name in enumerate(names):
                out[k][name] = ((fore[:, n, k - 1] - ref).norm(dim=1) / step).cpu().numpy()
        return out

    # ---- rollout ---------------------------------------------------------------
    def reset(self, history: torch.Tensor) -> None:
        """Fills the ring with the true vectors history[-1 - stride * i],
        i = 7..0 (oldest first)."""
        T = history.shape[0]
        self.ring.copy_(history[self._history_rows(np.array(T - 1))])
        self.order.copy_(torch.arange(HIST, dtype=torch.int32))

    def push(self, coeffs: torch.Tensor) -> None:
        """Appends a true vector (the newest, one stride after the last)."""
        etics.coeff_advance(self.ring, self.order, coeffs_in=coeffs.reshape(-1))

    def predict(self, net: bool = True) -> None:
        """The network's corrections for every horizon from the current ring
        (kept for ``forecast``); net=False sets them to 0 (the fitted
        predictors alone)."""
        if net:
            self._features(self.ring, self.order.view(1, HIST), x=self.x1)
            self.net.forward(self.x1, self.y1)
        else:
            self.y1.zero_()

    def _y(self, k: int) -> torch.Tensor:
        flat = self.y1.view(-1)
        return flat[k - 1:] if self.per_coeff else flat[(k - 1) * self.D:]

    def _y_stride(self) -> int:
        return self.stride if self.per_coeff else 1

    def forecast(self, out: torch.Tensor, horizon: int) -> torch.Tensor:
        """The vector ``horizon`` steps after the ring's newest into ``out``
        (D float64), from the last ``predict``."""
        etics.coeff_advance(self.ring, self.order, self.norm, y=self._y(horizon),
                            coeffs_out=out.view(-1), commit=False, stride=self.stride,
                            horizon=horizon, y_stride=self._y_stride())
        return out


def coefficient_trajectory(posm: torch.Tensor, vel: torch.Tensor, steps: int, dt: float,
                           n_max: int, l_max: int, acc: torch.Tensor | None = None):
    """Plain-SCF KDK for ``steps`` steps; returns the (steps + 1, D) float64
    coefficients (the first at the initial positions) and the final accpot."""
    D = (n_max + 1) * (l_max + 1) ** 2
    traj = torch.empty((steps + 1, D), dtype=torch.float64, device=posm.device)
    if acc is None:
        acc, c0 = etics.scf_force(posm, n_max, l_max)
        traj[0].copy_(c0.reshape(-1))
    else:
        traj[0].copy_(etics.scf_coeffs(posm, n_max, l_max).reshape(-1))
    for t in range(steps):
        etics.leapfrog_step(posm, vel, acc, dt, etics.SCF, n_max, l_max,
                            coeffs_out=traj[t + 1])
    return traj, acc


@dataclass
class RunStats:
    steps: int = 0
    recomputes: int = 0
    forecasts: int = 0
    fallbacks: int = 0
    checks: list = field(default_factory=list)  # (step, frac > tol_med, frac > tol_p99, max)


def run(posm: torch.Tensor, vel: torch.Tensor, acc: torch.Tensor, steps: int, dt: float,
        fc: Forecaster, tol_med: float = 1e-5, tol_p99: float = 1e-4, sample: int = 4096,
        check: bool = True, mode: str = "forecast", hook=None) -> RunStats:
    """KDK with the coefficient pass on every ``fc.stride``-th step only.

    The forecaster's ring must hold the true vectors of the last eight
    stride points, the newest one step before the first step (``reset`` on
    the trajectory the rollout continues).  Step t is a recompute step when
    (t + 1) % stride == 0; its true vector enters the ring.  The other steps,
    horizon k = (t + 1) % stride after the last recompute, use in mode
    "forecast" the forecast from the ring (fitted predictors plus the
    network), in mode "fitted" the fitted predictors alone, in mode "hold"
    the last recomputed coefficients (plain temporal reuse).  With ``check``
    every recompute step also forms what it would have used had it been a
    forecast step (the forecast at horizon ``stride``, or the held vector)
    and measures the relative acceleration error against the recomputed
    coefficients on the first ``sample`` particles; its median must stay <=
    tol_med and its 99th percentile <= tol_p99, else the next block runs
    plain SCF (the fallback).  The maximum is recorded but not judged: it
    sits at particles whose acceleration nearly vanishes, where a relative
    error means little.  ``hook`` (optional) is called after every step as
    hook(t, kind, coeffs, horizon) with kind "recompute", "forecast",
    "fitted" or "hold"."""
    n_max, l_max, S = fc.n_max, fc.l_max, fc.stride
    st = RunStats()
    c_true = torch.empty(fc.D, dtype=torch.float64, device=posm.device)
    c_use = fc.ring[int(fc.order[HIST - 1])].clone()
    c_fore = torch.empty_like(c_true)
    s = min(sample, posm.shape[0])
    a_ref = torch.empty((s, 4), dtype=posm.dtype, device=posm.device)
    a_fc = torch.empty_like(a_ref)
    err = torch.empty(3, dtype=torch.int64, device=posm.device)
    use_forecast = True
    forecasting = mode in ("forecast", "fitted")
    if forecasting:
        fc.predict(net=mode == "forecast")
    for t in range(steps):
        k = (t + 1) % S
        if k == 0:
            if check and forecasting:
                fc.forecast(c_fore, S)
            etics.leapfrog_step(posm, vel, acc, dt, etics.SCF, n_max, l_max, coeffs_out=c_true)
            fc.push(c_true)
            st.recomputes += 1
            if check:
                ref = c_fore if forecasting else c_use
                etics.scf_field(posm[:s], c_true.view(n_max + 1, -1), n_max, l_max, out=a_ref)
                etics.scf_field(posm[:s], ref.view(n_max + 1, -1), n_max, l_max, out=a_fc)
                etics.force_error(a_fc, a_ref, tol_med, tol_p99, out=err)
                e = err.cpu().numpy()
                mx = float(np.array([e[2]], dtype=np.int64).view(np.float64)[0])
                st.checks.append((t, float(e[0]) / s, float(e[1]) / s, mx))
                ok = 2 * e[0] <= s and 100 * e[1] <= s
                if not ok:
                    st.fallbacks += 1
                use_forecast = bool(ok)
            if forecasting:
                fc.predict(net=mode == "forecast")
            c_use.copy_(c_true)
            kind, hz = "recompute", 0
        elif use_forecast:
            if forecasting:
                fc.forecast(c_use, k)
            etics.leapfrog_step_coeffs(posm, vel, acc, dt, n_max, l_max, c_use)
            st.forecasts += 1
            kind, hz = mode, k
        else:
            etics.leapfrog_step(posm, vel, acc, dt, etics.SCF, n_max, l_max, coeffs_out=c_true)
            c_use.copy_(c_true)
            st.recomputes += 1
            kind, hz = "recompute", 0
        st.steps += 1
        if hook is not None:
            hook(t, kind, c_use, hz)
    return st
