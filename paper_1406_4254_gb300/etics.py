"""Thin Python binding of ``libetics.so`` (the C ABI in ``include/etics.h``).

Argument marshalling only: every step of the force calculation runs in the
library's CUDA kernels.  PyTorch supplies device memory and the current CUDA
stream.  There is no CPU fallback: if the library is missing or no GPU is
present the calls raise.

Particle tensors are (N, 4) CUDA tensors (x, y, z, m): float32 selects the
mixed-precision path, float64 the FP64 path.  Outputs are (N, 4) tensors
(ax, ay, az, Phi) in the input's particle order.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

SCF, MEX = 0, 1
FP64, MIXED = 0, 1
OUT_ACC, OUT_POT = 1, 2
NMAX_LIMIT, LMAX_LIMIT, MEX_LMAX_LIMIT = 16, 14, 10
ERR_ARG, ERR_CUDA, ERR_WORKSPACE, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
STATIC_SCRATCH_BYTES = 4 << 20      # ETICS_STATIC_SCRATCH_BYTES
WAIT_LOOKBACK, WAIT_MBARRIER = 0, 1
TIMEOUT_PROBE_N = 8192              # keys of the lookback probe

_STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA runtime error", -3: "workspace too small",
           -4: "non-finite input or FP32 overflow", -5: "inter-block wait timed out",
           -6: "parameters beyond the compiled limits"}

_lock = threading.Lock()
_lib = None
_ws_cache: dict = {}


class MlpShape(ctypes.Structure):
    _fields_ = [("nlayers", ctypes.c_int), ("dims", ctypes.c_int * 5)]

    @classmethod
    def of(cls, dims) -> "MlpShape":
        dims = [int(d) for d in dims]
        if not 2 <= len(dims) <= 5:
            raise ValueError("an MLP has 1 to 4 layers")
        return cls(len(dims) - 1, (ctypes.c_int * 5)(*(dims + [0] * (5 - len(dims)))))


class EticsError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_STATUS.get(status, 'unknown')} ({status})")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libetics.so (building it first if asked and needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError(f"libetics.so not built ({_build.LIB})")
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        vp, i64, i32, sz, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t,
                                 ctypes.c_double)
        lib.etics_workspace_bytes.argtypes = [i64, i32, i32, i32, i32]
        lib.etics_workspace_bytes.restype = sz
        lib.etics_scf_coeffs.argtypes = [vp, i64, i32, i32, i32, vp, vp, sz, vp]
        lib.etics_scf_field.argtypes = [vp, i64, i32, i32, i32, vp, vp, i32, vp]
        lib.etics_mex_field.argtypes = [vp, i64, i32, i32, vp, i32, vp, sz, vp]
        lib.etics_radial_sort.argtypes = [vp, i64, i32, vp, vp, sz, vp]
        lib.etics_radial_keys.argtypes = [vp, i64, i32, vp, vp]
        lib.etics_scf_coeffs_noalloc.argtypes = [vp, i64, i32, i32, i32, vp, vp]
        lib.etics_scf_batch_plan.argtypes = [vp, i32, vp, i32, vp, sz, ctypes.POINTER(sz),
                                             ctypes.POINTER(sz), ctypes.POINTER(i64)]
        lib.etics_scf_batch.argtypes = [vp, vp, vp, i32, vp, vp, i32, vp, sz, vp]
        lib.etics_leapfrog_step.argtypes = [vp, vp, vp, i64, dbl, i32, i32, i32, i32, vp, vp, sz,
                                            vp]
        lib.etics_scf_coeffs_basis.argtypes = [vp, i64, i32, i32, i32, i32, vp, vp, sz, vp]
        lib.etics_scf_field_basis.argtypes = [vp, i64, i32, i32, i32, i32, vp, vp, i32, vp]
        lib.etics_leapfrog_step_coeffs.argtypes = [vp, vp, vp, i64, dbl, i32, i32, i32, vp, vp]
        mp = ctypes.POINTER(MlpShape)
        lib.etics_mlp_param_count.argtypes = [mp]
        lib.etics_mlp_param_count.restype = i64
        lib.etics_mlp_workspace_bytes.argtypes = [mp, i32]
        lib.etics_mlp_workspace_bytes.restype = sz
        lib.etics_mlp_forward.argtypes = [mp, vp, vp, vp, i32, vp, vp, sz, vp]
        lib.etics_mlp_loss_grad.argtypes = [mp, vp, vp, vp, vp, i32, vp, vp, vp, sz, vp]
        flt = ctypes.c_float
        lib.etics_mlp_adam.argtypes = [mp, vp, vp, vp, vp, i64, flt, flt, flt, flt, vp, vp]
        lib.etics_mlp_to_bf16.argtypes = [mp, vp, vp, vp]
        lib.etics_coeff_stats.argtypes = [vp, i32, i32, i32, vp, vp]
        lib.etics_coeff_features.argtypes = [vp, vp, vp, i32, i32, i32, vp, i32, vp, vp, vp]
        lib.etics_coeff_advance.argtypes = [vp, vp, i32, i32, i32, vp, vp, i32, vp, vp, i32, vp]
        lib.etics_force_error.argtypes = [vp, vp, i64, i32, dbl, dbl, vp, vp]
        lib.etics_get_error.argtypes = [vp]
        lib.etics_strerror.argtypes = [i32]
        lib.etics_strerror.restype = ctypes.c_char_p
        lib.etics_launch_count.restype = ctypes.c_uint64
        lib.etics_set_stage_events.argtypes = [ctypes.POINTER(ctypes.c_void_p), i32]
        lib.etics_set_wait_limit.argtypes = [i64]
        lib.etics_fma_peak.argtypes = [i32, i32, i64, vp, ctypes.POINTER(dbl), vp]
        lib.etics_test_wait_timeout.argtypes = [i32, i64, vp, sz, vp]
        for name in ("etics_scf_coeffs", "etics_scf_field", "etics_mex_field",
                     "etics_radial_sort", "etics_radial_keys", "etics_leapfrog_step",
                     "etics_scf_coeffs_noalloc", "etics_scf_batch_plan", "etics_scf_batch",
                     "etics_leapfrog_step_coeffs", "etics_mlp_forward",
                     "etics_scf_coeffs_basis", "etics_scf_field_basis", "etics_mlp_loss_grad",
                     "etics_mlp_adam", "etics_mlp_to_bf16", "etics_coeff_stats",
                     "etics_coeff_features", "etics_coeff_advance", "etics_force_error",
                     "etics_get_error", "etics_set_wait_limit", "etics_test_wait_timeout",
                     "etics_fma_peak",
                     "etics_set_stage_events"):
            getattr(lib, name).restype = i32
        _lib = lib
        return lib


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _precision(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return MIXED
    if t.dtype == torch.float64:
        return FP64
    raise TypeError("particle arrays must be float32 (mixed) or float64 (FP64)")


def _particles(t: torch.Tensor, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dim() != 2 or t.shape[1] != 4 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous (N, 4) tensor")
    return t


def _check(rc: int, what: str):
    if rc != 0:
        raise EticsError(rc, what)


def workspace_bytes(n: int, n_max: int, l_max: int, method: int, precision: int) -> int:
    return int(load().etics_workspace_bytes(int(n), int(n_max), int(l_max), int(method),
                                            int(precision)))


def workspace(n: int, n_max: int, l_max: int, method: int, precision: int, device=None,
              extra: int = 0) -> torch.Tensor:
    """A cached uint8 device buffer large enough for the call."""
    dev = torch.device(device) if device is not None else torch.device("cuda",
                                                                        torch.cuda.current_device())
    need = workspace_bytes(n, n_max, l_max, method, precision) + extra
    if need <= 0:
        raise EticsError(-1, "workspace_bytes")
    key = (dev.index, method)
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < need:
        buf = torch.empty(need + 256, dtype=torch.uint8, device=dev)
        _ws_cache[key] = buf
    return buf


def _aligned_ptr(buf: torch.Tensor) -> tuple[int, int]:
    p = buf.data_ptr()
    q = (p + 255) // 256 * 256
    return q, buf.numel() - (q - p)


BASIS_HO, BASIS_CB = 0, 1


def scf_coeffs(posm: torch.Tensor, n_max: int, l_max: int, out: torch.Tensor | None = None,
               ws: torch.Tensor | None = None, stream=None, basis: int = BASIS_HO) -> torch.Tensor:
    """SCF coefficients c[n, l*l+l+m] (float64, shape (n_max+1, (l_max+1)^2));
    basis BASIS_HO (Hernquist-Ostriker, default) or BASIS_CB (Clutton-Brock)."""
    posm = _particles(posm, "posm")
    prec = _precision(posm)
    n = posm.shape[0]
    if out is None:
        out = torch.empty((n_max + 1, (l_max + 1) ** 2), dtype=torch.float64, device=posm.device)
    if ws is None:
        ws = workspace(n, n_max, l_max, SCF, prec, posm.device)
    wp, wb = _aligned_ptr(ws)
    if basis == BASIS_HO:
        rc = load().etics_scf_coeffs(posm.data_ptr(), n, n_max, l_max, prec, out.data_ptr(), wp,
                                     wb, _stream(stream))
    else:
        rc = load().etics_scf_coeffs_basis(posm.data_ptr(), n, n_max, l_max, int(basis), prec,
                                           out.data_ptr(), wp, wb, _stream(stream))
    _check(rc, "etics_scf_coeffs")
    return out


def scf_coeffs_noalloc(posm: torch.Tensor, n_max: int, l_max: int,
                       out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """SCF coefficients through etics_scf_coeffs_noalloc: no workspace is
    passed and the library allocates nothing (its scratch is a fixed array
    inside the library; concurrent calls on the same GPU race)."""
    posm = _particles(posm, "posm")
    if out is None:
        out = torch.empty((n_max + 1, (l_max + 1) ** 2), dtype=torch.float64, device=posm.device)
    _check(load().etics_scf_coeffs_noalloc(posm.data_ptr(), posm.shape[0], n_max, l_max,
                                           _precision(posm), out.data_ptr(), _stream(stream)),
           "etics_scf_coeffs_noalloc")
    return out


def scf_field(posm: torch.Tensor, coeffs: torch.Tensor, n_max: int, l_max: int,
              out: torch.Tensor | None = None, out_mask: int = OUT_ACC | OUT_POT,
              stream=None, basis: int = BASIS_HO) -> torch.Tensor:
    """SCF (ax, ay, az, Phi) at each particle of posm."""
    posm = _particles(posm, "posm")
    prec = _precision(posm)
    if coeffs.dtype != torch.float64 or not coeffs.is_cuda or not coeffs.is_contiguous():
        raise ValueError("coeffs must be a contiguous float64 CUDA tensor")
    if coeffs.numel() != (n_max + 1) * (l_max + 1) ** 2:
        raise ValueError("coefficient count does not match (n_max, l_max)")
    if out is None:
        out = torch.empty_like(posm)
    if basis == BASIS_HO:
        rc = load().etics_scf_field(posm.data_ptr(), posm.shape[0], n_max, l_max, prec,
                                    coeffs.data_ptr(), out.data_ptr(), out_mask, _stream(stream))
    else:
        rc = load().etics_scf_field_basis(posm.data_ptr(), posm.shape[0], n_max, l_max,
                                          int(basis), prec, coeffs.data_ptr(), out.data_ptr(),
                                          out_mask, _stream(stream))
    _check(rc, "etics_scf_field")
    return out


def scf_force(posm: torch.Tensor, n_max: int, l_max: int, out=None, stream=None,
              basis: int = BASIS_HO):
    """Both SCF passes; returns (accpot, coeffs)."""
    c = scf_coeffs(posm, n_max, l_max, stream=stream, basis=basis)
    return scf_field(posm, c, n_max, l_max, out=out, stream=stream, basis=basis), c


def mex_field(posm: torch.Tensor, l_max: int, out: torch.Tensor | None = None,
              out_mask: int = OUT_ACC | OUT_POT, ws: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
    """MEX (ax, ay, az, Phi) at each particle."""
    posm = _particles(posm, "posm")
    prec = _precision(posm)
    n = posm.shape[0]
    if out is None:
        out = torch.empty_like(posm)
    if ws is None:
        ws = workspace(n, 0, l_max, MEX, prec, posm.device)
    wp, wb = _aligned_ptr(ws)
    _check(load().etics_mex_field(posm.data_ptr(), n, l_max, prec, out.data_ptr(), out_mask, wp,
                                  wb, _stream(stream)), "etics_mex_field")
    return out


def radial_order(posm: torch.Tensor, ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Particle indices in MEX's radial order (int64 tensor)."""
    posm = _particles(posm, "posm")
    prec = _precision(posm)
    n = posm.shape[0]
    order = torch.empty(max(n, 1), dtype=torch.int32, device=posm.device)
    if ws is None:
        ws = workspace(n, 0, 0, MEX, prec, posm.device)
    wp, wb = _aligned_ptr(ws)
    _check(load().etics_radial_sort(posm.data_ptr(), n, prec, order.data_ptr(), wp, wb,
                                    _stream(stream)), "etics_radial_sort")
    return order[:n].to(torch.int64) & 0xFFFFFFFF


def radial_keys(posm: torch.Tensor, stream=None) -> torch.Tensor:
    """High 32 bits of the FP64 r^2 bit pattern per particle (int64 tensor)."""
    posm = _particles(posm, "posm")
    n = posm.shape[0]
    keys = torch.empty(max(n, 1), dtype=torch.int32, device=posm.device)
    _check(load().etics_radial_keys(posm.data_ptr(), n, _precision(posm), keys.data_ptr(),
                                    _stream(stream)), "etics_radial_keys")
    return keys[:n].to(torch.int64) & 0xFFFFFFFF


def leapfrog_step(posm: torch.Tensor, vel: torch.Tensor, accpot: torch.Tensor, dt: float,
                  method: int, n_max: int, l_max: int, coeffs_out: torch.Tensor | None = None,
                  ws: torch.Tensor | None = None, stream=None) -> None:
    """One in-place KDK step; accpot holds a(x) on entry and (a, Phi) after."""
    posm = _particles(posm, "posm")
    vel = _particles(vel, "vel")
    accpot = _particles(accpot, "accpot")
    prec = _precision(posm)
    if vel.dtype != posm.dtype or accpot.dtype != posm.dtype:
        raise TypeError("posm, vel and accpot must share a dtype")
    n = posm.shape[0]
    extra = ((n_max + 1) * (l_max + 1) ** 2 * 8 + 255) // 256 * 256 if method == SCF else 0
    if ws is None:
        ws = workspace(n, n_max, l_max, method, prec, posm.device, extra=extra)
    wp, wb = _aligned_ptr(ws)
    cp = coeffs_out.data_ptr() if coeffs_out is not None else None
    _check(load().etics_leapfrog_step(posm.data_ptr(), vel.data_ptr(), accpot.data_ptr(), n,
                                      float(dt), method, n_max, l_max, prec, cp, wp, wb,
                                      _stream(stream)), "etics_leapfrog_step")


def leapfrog_step_coeffs(posm: torch.Tensor, vel: torch.Tensor, accpot: torch.Tensor, dt: float,
                         n_max: int, l_max: int, coeffs: torch.Tensor, stream=None) -> None:
    """One in-place KDK step whose new force uses the given SCF coefficients."""
    posm = _particles(posm, "posm")
    vel = _particles(vel, "vel")
    accpot = _particles(accpot, "accpot")
    if vel.dtype != posm.dtype or accpot.dtype != posm.dtype:
        raise TypeError("posm, vel and accpot must share a dtype")
    _vector(coeffs, torch.float64, (n_max + 1) * (l_max + 1) ** 2, "coeffs")
    _check(load().etics_leapfrog_step_coeffs(posm.data_ptr(), vel.data_ptr(), accpot.data_ptr(),
                                             posm.shape[0], float(dt), n_max, l_max,
                                             _precision(posm), coeffs.data_ptr(),
                                             _stream(stream)), "etics_leapfrog_step_coeffs")


# ---- coefficient-forecasting MLP ----------------------------------------------
def _vector(t: torch.Tensor, dtype, numel: int | None, name: str) -> torch.Tensor:
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return t


def mlp_param_count(dims) -> int:
    n = int(load().etics_mlp_param_count(ctypes.byref(MlpShape.of(dims))))
    if n < 0:
        raise EticsError(-1, "etics_mlp_param_count")
    return n


def mlp_workspace(dims, batch: int, device=None) -> torch.Tensor:
    need = int(load().etics_mlp_workspace_bytes(ctypes.byref(MlpShape.of(dims)), int(batch)))
    if need <= 0:
        raise EticsError(-1, "etics_mlp_workspace_bytes")
    return torch.empty(need + 256, dtype=torch.uint8, device=device or "cuda")


def mlp_forward(dims, params: torch.Tensor, params_bf16: torch.Tensor, x: torch.Tensor,
                y: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """y = network(x); x: (batch, dims[0]) bfloat16, y: (batch, dims[-1]) float32."""
    n = mlp_param_count(dims)
    _vector(params, torch.float32, n, "params")
    _vector(params_bf16, torch.bfloat16, n, "params_bf16")
    _vector(x, torch.bfloat16, None, "x")
    b = x.shape[0]
    if x.numel() != b * dims[0]:
        raise ValueError("x must be (batch, dims[0])")
    if y is None:
        y = torch.empty((b, dims[-1]), dtype=torch.float32, device=x.device)
    _vector(y, torch.float32, b * dims[-1], "y")
    if ws is None:
        ws = mlp_workspace(dims, b, x.device)
    wp, wb = _aligned_ptr(ws)
    _check(load().etics_mlp_forward(ctypes.byref(MlpShape.of(dims)), params.data_ptr(),
                                    params_bf16.data_ptr(), x.data_ptr(), b, y.data_ptr(), wp, wb,
                                    _stream(stream)), "etics_mlp_forward")
    return y


def mlp_loss_grad(dims, params: torch.Tensor, params_bf16: torch.Tensor, x: torch.Tensor,
                  target: torch.Tensor, grads: torch.Tensor, loss: torch.Tensor,
                  ws: torch.Tensor | None = None, stream=None) -> None:
    """loss (float64, 1 element) = MSE(network(x), target); grads = its gradient."""
    n = mlp_param_count(dims)
    _vector(params, torch.float32, n, "params")
    _vector(params_bf16, torch.bfloat16, n, "params_bf16")
    _vector(grads, torch.float32, n, "grads")
    _vector(loss, torch.float64, 1, "loss")
    _vector(x, torch.bfloat16, None, "x")
    b = x.shape[0]
    _vector(target, torch.float32, b * dims[-1], "target")
    if ws is None:
        ws = mlp_workspace(dims, b, x.device)
    wp, wb = _aligned_ptr(ws)
    _check(load().etics_mlp_loss_grad(ctypes.byref(MlpShape.of(dims)), params.data_ptr(),
                                      params_bf16.data_ptr(), x.data_ptr(), target.data_ptr(), b,
                                      grads.data_ptr(), loss.data_ptr(), wp, wb, _stream(stream)),
           "etics_mlp_loss_grad")


def mlp_adam(dims, params, grads, m, v, t: int, lr: float, params_bf16, beta1=0.9, beta2=0.999,
             eps=1e-8, stream=None) -> None:
    n = mlp_param_count(dims)
    for name, tt in (("params", params), ("grads", grads), ("m", m), ("v", v)):
        _vector(tt, torch.float32, n, name)
    _vector(params_bf16, torch.bfloat16, n, "params_bf16")
    _check(load().etics_mlp_adam(ctypes.byref(MlpShape.of(dims)), params.data_ptr(),
                                 grads.data_ptr(), m.data_ptr(), v.data_ptr(), int(t), float(lr),
                                 float(beta1), float(beta2), float(eps), params_bf16.data_ptr(),
                                 _stream(stream)), "etics_mlp_adam")


def mlp_to_bf16(dims, params, params_bf16, stream=None) -> None:
    n = mlp_param_count(dims)
    _vector(params, torch.float32, n, "params")
    _vector(params_bf16, torch.bfloat16, n, "params_bf16")
    _check(load().etics_mlp_to_bf16(ctypes.byref(MlpShape.of(dims)), params.data_ptr(),
                                    params_bf16.data_ptr(), _stream(stream)), "etics_mlp_to_bf16")


def norm_rows(stride: int) -> int:
    """Rows of the forecasting normalisers for histories of this stride."""
    return 7 + 9 * int(stride)


def coeff_stats(traj: torch.Tensor, stride: int = 1, norm: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """(7 + 9 stride, D) normalisers of a (T, D) float64 coefficient
    trajectory: scales of the state and of its differences at spacing
    ``stride``, then per horizon k = 1..stride the fitted linear predictor and
    the RMS of its residual."""
    _vector(traj, torch.float64, None, "traj")
    t, d = traj.shape
    rows = norm_rows(stride)
    if norm is None:
        norm = torch.empty((rows, d), dtype=torch.float64, device=traj.device)
    _vector(norm, torch.float64, rows * d, "norm")
    _check(load().etics_coeff_stats(traj.data_ptr(), t, d, int(stride), norm.data_ptr(),
                                    _stream(stream)), "etics_coeff_stats")
    return norm


FEAT_JOINT, FEAT_PER_COEFF = 0, 1


def coeff_features(store: torch.Tensor, rows: torch.Tensor, norm: torch.Tensor,
                   next_rows: torch.Tensor | None = None, x: torch.Tensor | None = None,
                   target: torch.Tensor | None = None, per_coeff: bool = False, stride: int = 1,
                   stream=None):
    """Network inputs of the histories store[rows] (rows: (batch, 8) int32,
    oldest first): (batch, 8D) bfloat16 in the joint layout, (batch*D, 8) per
    coefficient; with next_rows ((batch, stride) int32: the vectors 1..stride
    steps after each history) also the targets, float32 (batch*D, stride) per
    coefficient or (batch, stride*D) jointly."""
    _vector(store, torch.float64, None, "store")
    _vector(rows, torch.int32, None, "rows")
    d = store.shape[1]
    b = rows.shape[0]
    _vector(norm, torch.float64, norm_rows(stride) * d, "norm")
    if x is None:
        shape = (b * d, 8) if per_coeff else (b, 8 * d)
        x = torch.empty(shape, dtype=torch.bfloat16, device=store.device)
    _vector(x, torch.bfloat16, b * 8 * d, "x")
    np_ = tp = None
    if next_rows is not None:
        _vector(next_rows, torch.int32, b * stride, "next_rows")
        if target is None:
            shape = (b * d, stride) if per_coeff else (b, stride * d)
            target = torch.empty(shape, dtype=torch.float32, device=store.device)
        _vector(target, torch.float32, b * d * stride, "target")
        np_, tp = next_rows.data_ptr(), target.data_ptr()
    _check(load().etics_coeff_features(store.data_ptr(), rows.data_ptr(), np_, b, d, int(stride),
                                       norm.data_ptr(), FEAT_PER_COEFF if per_coeff else FEAT_JOINT,
                                       x.data_ptr(), tp, _stream(stream)),
           "etics_coeff_features")
    return x, target


def coeff_advance(ring: torch.Tensor, order: torch.Tensor, norm: torch.Tensor | None = None,
                  coeffs_in: torch.Tensor | None = None, y: torch.Tensor | None = None,
                  coeffs_out: torch.Tensor | None = None, commit: bool = True, stride: int = 1,
                  horizon: int = 1, y_stride: int = 1, stream=None) -> None:
    """Forecast at ``horizon`` from the ring (y: one network output per
    coefficient, y[j * y_stride]) or push coeffs_in; commit writes the vector
    into the oldest slot and rotates ``order``."""
    _vector(ring, torch.float64, None, "ring")
    _vector(order, torch.int32, 8, "order")
    d = ring.shape[1]
    ptr = lambda t: t.data_ptr() if t is not None else None  # noqa: E731
    _check(load().etics_coeff_advance(ring.data_ptr(), order.data_ptr(), d, int(stride),
                                      int(horizon), ptr(coeffs_in), ptr(y), int(y_stride),
                                      ptr(norm), ptr(coeffs_out), int(bool(commit)),
                                      _stream(stream)), "etics_coeff_advance")


def force_error(a: torch.Tensor, r: torch.Tensor, tol_a: float, tol_b: float,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Device int64[3]: #(e > tol_a), #(e > tol_b), bits of max e, for the
    relative acceleration error e of accpot a against accpot r."""
    a = _particles(a, "a")
    r = _particles(r, "r")
    if a.dtype != r.dtype or a.shape != r.shape:
        raise ValueError("a and r must match")
    if out is None:
        out = torch.empty(3, dtype=torch.int64, device=a.device)
    _check(load().etics_force_error(a.data_ptr(), r.data_ptr(), a.shape[0], _precision(a),
                                    float(tol_a), float(tol_b), out.data_ptr(), _stream(stream)),
           "etics_force_error")
    return out


class _BatchItem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_max", ctypes.c_int), ("l_max", ctypes.c_int)]


class BatchTuning(ctypes.Structure):
    """Launch shape of a batch (0 = library default)."""
    _fields_ = [("tile", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("field_threads", ctypes.c_int), ("field_chunk", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchPlan:
    """A batch plan: host bytes, their device copy, workspace, and the packed
    coefficient offsets of every system."""

    def __init__(self, sizes, n_maxes, l_maxes, precision=MIXED, tuning=None, device=None):
        lib = load()
        ninst = len(sizes)
        items = (_BatchItem * ninst)(*[_BatchItem(int(n), int(a), int(b))
                                       for n, a, b in zip(sizes, n_maxes, l_maxes)])
        need, ws, cc = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int64()
        tp = ctypes.addressof(tuning) if tuning is not None else None
        _check(lib.etics_scf_batch_plan(ctypes.addressof(items), ninst, tp, precision, None, 0,
                                        ctypes.byref(need), ctypes.byref(ws), ctypes.byref(cc)),
               "etics_scf_batch_plan")
        self.host = (ctypes.c_uint8 * need.value)()
        _check(lib.etics_scf_batch_plan(ctypes.addressof(items), ninst, tp, precision,
                                        ctypes.addressof(self.host), need.value,
                                        ctypes.byref(need), ctypes.byref(ws), ctypes.byref(cc)),
               "etics_scf_batch_plan")
        dev = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.dev = torch.frombuffer(bytearray(self.host), dtype=torch.uint8).to(dev)
        self.ws = torch.empty(ws.value + 256, dtype=torch.uint8, device=dev)
        self.coeff_count = int(cc.value)
        self.precision = precision
        self.sizes = [int(n) for n in sizes]
        self.n_maxes = [int(a) for a in n_maxes]
        self.l_maxes = [int(b) for b in l_maxes]
        offs, o = [], 0
        for a, b in zip(self.n_maxes, self.l_maxes):
            offs.append(o)
            o += (a + 1) * (b + 1) ** 2
        self.coeff_offsets = offs
        self.particle_offsets = [0]
        for n in self.sizes:
            self.particle_offsets.append(self.particle_offsets[-1] + n)

    def coeffs_of(self, packed: torch.Tensor, i: int) -> torch.Tensor:
        a, b = self.n_maxes[i], self.l_maxes[i]
        o = self.coeff_offsets[i]
        return packed[o:o + (a + 1) * (b + 1) ** 2].view(a + 1, (b + 1) ** 2)


def scf_batch(posm: torch.Tensor, plan: BatchPlan, coeffs: torch.Tensor | None = None,
              out: torch.Tensor | None = None, out_mask: int = OUT_ACC | OUT_POT,
              with_field: bool = True, stream=None):
    """SCF coefficients (packed float64) and field of every system of the plan."""
    posm = _particles(posm, "posm")
    if _precision(posm) != plan.precision:
        raise TypeError("particle dtype does not match the plan's precision")
    if posm.shape[0] != plan.particle_offsets[-1]:
        raise ValueError("posm does not hold the plan's particles")
    if coeffs is None:
        coeffs = torch.empty(max(plan.coeff_count, 1), dtype=torch.float64, device=posm.device)
    if with_field and out is None:
        out = torch.empty_like(posm)
    wp, wb = _aligned_ptr(plan.ws)
    _check(load().etics_scf_batch(posm.data_ptr(), ctypes.addressof(plan.host),
                                  plan.dev.data_ptr(), plan.precision, coeffs.data_ptr(),
                                  out.data_ptr() if with_field else None, out_mask, wp, wb,
                                  _stream(stream)), "etics_scf_batch")
    return coeffs, out


def get_error(stream=None) -> int:
    """Synchronise the stream and return/clear the device error status."""
    return int(load().etics_get_error(_stream(stream)))


def check_error(stream=None):
    rc = get_error(stream)
    if rc:
        raise EticsError(rc, "device")


def set_wait_limit(spins: int) -> None:
    """Bound (in polls) of the radial sort's lookback waits; 0 = default."""
    _check(load().etics_set_wait_limit(int(spins)), "etics_set_wait_limit")


def probe_wait_timeout(which: int, spins: int, ws: torch.Tensor | None = None,
                      stream=None) -> None:
    """Make one bounded device wait run out (WAIT_LOOKBACK or WAIT_MBARRIER);
    the outcome is read with get_error()."""
    wp, wb = 0, 0
    if which == WAIT_LOOKBACK:
        if ws is None:
            ws = workspace(TIMEOUT_PROBE_N, 0, 0, MEX, MIXED)
        wp, wb = _aligned_ptr(ws)
    _check(load().etics_test_wait_timeout(int(which), int(spins), wp or None, wb,
                                          _stream(stream)), "etics_test_wait_timeout")


PEAK_FFMA, PEAK_FFMA2, PEAK_DFMA = 0, 1, 2


def fma_peak(kind: int, blocks: int, iters: int, sink: torch.Tensor, stream=None) -> float:
    """Launch the FMA-rate microbenchmark; returns the launch's flop count."""
    if sink.dtype != torch.float32 or not sink.is_cuda or sink.numel() < blocks * 256:
        raise ValueError("sink must be a float32 CUDA tensor of blocks * 256 elements")
    flops = ctypes.c_double()
    _check(load().etics_fma_peak(int(kind), int(blocks), int(iters), sink.data_ptr(),
                                 ctypes.byref(flops), _stream(stream)), "etics_fma_peak")
    return float(flops.value)


def launch_count() -> int:
    return int(load().etics_launch_count())


def set_stage_events(events) -> None:
    """Have later calls record these raw cudaEvent_t handles (ints or
    c_void_p) at their stage boundaries; None disables."""
    lib = load()
    if not events:
        _check(lib.etics_set_stage_events(None, 0), "etics_set_stage_events")
        set_stage_events._keep = None
        return
    arr = (ctypes.c_void_p * len(events))(
        *[e if isinstance(e, ctypes.c_void_p) else ctypes.c_void_p(int(e)) for e in events])
    set_stage_events._keep = arr
    _check(lib.etics_set_stage_events(arr, len(events)), "etics_set_stage_events")


def to_host_force(posm_host: torch.Tensor, method: int, n_max: int, l_max: int,
                  out_host: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """End-to-end convenience: host (pinned) particles in, host (ax, ay, az, Phi) out.

    Copies the particles to the device, runs the force calculation and copies
    the result back, all on one stream."""
    dev = torch.device("cuda", torch.cuda.current_device())
    s = stream if stream is not None else torch.cuda.current_stream()
    with torch.cuda.stream(s):
        d = posm_host.to(dev, non_blocking=True)
        if method == SCF:
            res, _ = scf_force(d, n_max, l_max, stream=s)
        else:
            res = mex_field(d, l_max, stream=s)
        if out_host is None:
            out_host = torch.empty(res.shape, dtype=res.dtype, pin_memory=True)
        out_host.copy_(res, non_blocking=True)
    return out_host
