"""Coefficient forecasting for SCF time integration (the learned part).

The paper has no learned component.  It notes that the coefficients may be
kept over several steps (temporal softening, end of Sec. 4.1); here a small
MLP instead forecasts the next coefficient vector from the last eight, so the
coefficient pass (the first SCF pass, Sec. 3.3) runs only every ``period``-th
step.  Plain SCF remains the fallback and the judge: on every recompute step
the forecast the network would have made is compared with the recomputed
coefficients through the relative acceleration error on a particle sample,
and a forecast that misses the force-error budget switches the next block to
plain SCF.

Everything numeric runs in ``libetics.so`` kernels (bf16 tensor-core
products, Adam, feature and update kernels); this module only orders the
calls and owns the buffers.

Typical use::

    traj = coefficient_trajectory(posm, vel, steps, dt, n_max, l_max)
    fc = Forecaster(n_max, l_max, hidden=256)
    fc.fit(traj[:n_train], iters=2000, batch=256)
    stats = run(posm, vel, acc, steps, dt, fc, period=4)
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
    one step ahead from the last HIST vectors, autoregressively.

    per_coeff=True (default): one network shared by all coefficients maps a
    coefficient's own eight features to its forecast (HIST -> hidden -> ... ->
    1, applied to D rows).  per_coeff=False: one network sees the features of
    every coefficient at once (HIST*D -> hidden -> ... -> D)."""

    def __init__(self, n_max: int, l_max: int, hidden: int = 256, layers: int = 3, seed: int = 0,
                 per_coeff: bool = True, device="cuda"):
        self.n_max, self.l_max = n_max, l_max
        self.D = (n_max + 1) * (l_max + 1) ** 2
        self.per_coeff = per_coeff
        if per_coeff:
            dims = [HIST] + [hidden] * (layers - 1) + [1]
        else:
            dims = [HIST * self.D] + [hidden] * (layers - 1) + [self.D]
        self.net = Mlp(dims, seed=seed, device=device)
        self.device = torch.device(device)
        self.norm = torch.zeros((etics.NORM_ROWS, self.D), dtype=torch.float64, device=device)
        self.ring = torch.zeros((HIST, self.D), dtype=torch.float64, device=device)
        self.order = torch.arange(HIST, dtype=torch.int32, device=device)
        self.x1 = self._x(1)
        self.y1 = torch.empty((self._rows(1), dims[-1]), dtype=torch.float32, device=device)
        self.filled = 0

    def _rows(self, hist: int) -> int:
        return hist * self.D if self.per_coeff else hist

    def _x(self, hist: int) -> torch.Tensor:
        shape = (hist * self.D, HIST) if self.per_coeff else (hist, HIST * self.D)
        return torch.empty(shape, dtype=torch.bfloat16, device=self.device)

    def _features(self, store, rows, nxt=None, x=None, tg=None):
        return etics.coeff_features(store, rows, self.norm, nxt, x, tg, per_coeff=self.per_coeff)

    # ---- training ------------------------------------------------------------
    def fit(self, traj: torch.Tensor, iters: int = 2000, batch: int = 256, lr: float = 1e-3,
            seed: int = 0, log_every: int = 0):
        """Trains on a (T, D) float64 trajectory: normalisers from the whole of
        it, minibatches of ``batch`` (8-vector history, next vector) pairs (so
        batch * D network rows per coefficient network) drawn with a
        seeded generator, Adam with a cosine learning-rate decay.  Returns the
        loss every ``log_every`` iterations (a list of floats) when asked."""
        traj = traj.contiguous()
        T = traj.shape[0]
        if T < HIST + 1:
            raise ValueError("need at least 9 coefficient vectors")
        etics.coeff_stats(traj, self.norm)
        rng = np.random.Generator(np.random.Philox(key=[int(seed), 6]))
        last = rng.integers(HIST - 1, T - 1, size=(iters, batch))      # newest history index
        rows = torch.tensor(last[:, :, None] + np.arange(-HIST + 1, 1)[None, None, :],
                            dtype=torch.int32, device=self.device)
        nxt = torch.tensor(last + 1, dtype=torch.int32, device=self.device)
        x = self._x(batch)
        tg = torch.empty((batch, self.D), dtype=torch.float32, device=self.device)
        tgv = tg.view(self._rows(batch), -1)
        losses = []
        for it in range(iters):
            self._features(traj, rows[it], nxt[it], x, tg)
            loss = self.net.loss_grad(x, tgv)
            self.net.adam_step(lr * 0.5 * (1.0 + math.cos(math.pi * it / iters)))
            if log_every and (it % log_every == 0 or it == iters - 1):
                losses.append(float(loss.item()))
        return losses

    def one_step_errors(self, traj: torch.Tensor, first: int):
        """One-step forecast errors on true histories of traj[first - 7 ..]:
        |c_hat - c| / |c - c_prev| over each next vector, for hold-last, linear
        and cubic extrapolation and the network (arrays)."""
        T = traj.shape[0]
        last = np.arange(max(first, HIST - 1), T - 1)
        rows = torch.tensor(last[:, None] + np.arange(-HIST + 1, 1)[None, :], dtype=torch.int32,
                            device=self.device)
        x, _ = self._features(traj, rows)
        y = self.net.forward(x).double().view(len(last), self.D)
        c4, c5, c6, c7 = (traj[last - k] for k in (3, 2, 1, 0))
        c8 = traj[last + 1]
        step = (c8 - c7).norm(dim=1)
        lin = c7 + (c7 - c6)
        cubic = 4 * c7 - 6 * c6 + 4 * c5 - c4
        net = cubic + self.norm[6][None, :] * y
        err = lambda c: ((c - c8).norm(dim=1) / step).cpu().numpy()  # noqa: E731
        return err(c7), err(lin), err(cubic), err(net)

    # ---- rollout ---------------------------------------------------------------
    def reset(self, history: torch.Tensor) -> None:
        """Fills the ring with the last HIST true vectors (oldest first)."""
        self.ring.copy_(history[-HIST:])
        self.order.copy_(torch.arange(HIST, dtype=torch.int32))
        self.filled = HIST

    def push(self, coeffs: torch.Tensor) -> None:
        etics.coeff_advance(self.ring, self.order, coeffs_in=coeffs.reshape(-1))
        self.filled = min(HIST, self.filled + 1)

    def forecast(self, out: torch.Tensor, commit: bool = True) -> torch.Tensor:
        """The next vector into ``out`` (D float64); appended to the ring when
        ``commit``."""
        self._features(self.ring, self.order.view(1, HIST), x=self.x1)
        self.net.forward(self.x1, self.y1)
        etics.coeff_advance(self.ring, self.order, self.norm, y=self.y1.view(-1),
                            coeffs_out=out.view(-1), commit=commit)
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
        fc: Forecaster, period: int = 4, tol_med: float = 1e-5, tol_p99: float = 1e-4,
        sample: int = 4096, check: bool = True, mode: str = "forecast",
        hook=None) -> RunStats:
    """KDK with the coefficient pass on every ``period``-th step only.

    mode "forecast": the other steps use the network's forecast; "hold": they
    reuse the last recomputed coefficients (plain temporal reuse).  The
    forecaster's ring must hold the last HIST true coefficient vectors
    (``reset``).  With ``check`` every recompute step also forecasts the
    recomputed vector and measures the relative acceleration error on the
    first ``sample`` particles (the last substep's error bounds the earlier
    ones'); its median must stay <= tol_med and its 99th percentile <=
    tol_p99, else the next block runs plain SCF (the fallback).  The maximum
    is recorded but not judged: it sits at particles whose acceleration
    nearly vanishes, where a relative error means little.  ``hook``
    (optional) is called after every step as hook(t, kind, coeffs) with kind
    "recompute", "forecast" or "hold" and the coefficients the step used."""
    n_max, l_max = fc.n_max, fc.l_max
    st = RunStats()
    c_true = torch.empty(fc.D, dtype=torch.float64, device=posm.device)
    c_use = torch.empty_like(c_true)
    c_fore = torch.empty_like(c_true)
    s = min(sample, posm.shape[0])
    a_ref = torch.empty((s, 4), dtype=posm.dtype, device=posm.device)
    a_fc = torch.empty_like(a_ref)
    err = torch.empty(3, dtype=torch.int64, device=posm.device)
    use_forecast = True
    for t in range(steps):
        if t % period == 0:
            if check and mode == "forecast":
                fc.forecast(c_fore, commit=False)
            etics.leapfrog_step(posm, vel, acc, dt, etics.SCF, n_max, l_max, coeffs_out=c_true)
            fc.push(c_true)
            st.recomputes += 1
            if check:
                ref = c_fore if mode == "forecast" else c_use
                if mode == "hold" and t == 0:
                    ref = c_true
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
            c_use.copy_(c_true)
            kind = "recompute"
        elif use_forecast:
            if mode == "forecast":
                fc.forecast(c_use, commit=True)
            etics.leapfrog_step_coeffs(posm, vel, acc, dt, n_max, l_max, c_use)
            st.forecasts += 1
            kind = mode
        else:
            etics.leapfrog_step(posm, vel, acc, dt, etics.SCF, n_max, l_max, coeffs_out=c_true)
            fc.push(c_true)
            c_use.copy_(c_true)
            st.recomputes += 1
            kind = "recompute"
        st.steps += 1
        if hook is not None:
            hook(t, kind, c_use)
    return st
