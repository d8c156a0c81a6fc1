"""Shared helpers for the GPU parity tests (inputs, error metrics)."""
import numpy as np
import torch

from paper_1406_4254_gb300 import inputs

DTYPES = {"mixed": torch.float32, "fp64": torch.float64}

# tolerances on the relative acceleration error eps_i = |a - a_ref| / |a_ref|
# (the paper's eq. 23): FP64 path vs oracle, and the mixed path's stated bound
TOL = {"fp64": {"median": 1e-13, "max": 1e-10},
       "mixed": {"median": 1e-5, "max": 1e-4}}


def device_particles(pm: np.ndarray, precision: str) -> torch.Tensor:
    return torch.tensor(pm, dtype=DTYPES[precision], device="cuda").contiguous()


def rounded(pm: np.ndarray, precision: str) -> np.ndarray:
    """The particle values the GPU actually sees, in float64 (for the oracle)."""
    if precision == "mixed":
        return pm.astype(np.float32).astype(np.float64)
    return pm.copy()


def rel_acc_err(a_gpu: np.ndarray, a_ref: np.ndarray) -> np.ndarray:
    num = np.linalg.norm(a_gpu - a_ref, axis=1)
    den = np.linalg.norm(a_ref, axis=1)
    return num / np.where(den > 0, den, 1.0)


def rel_pot_err(p_gpu: np.ndarray, p_ref: np.ndarray) -> np.ndarray:
    return np.abs(p_gpu - p_ref) / np.maximum(np.abs(p_ref), 1e-300)


def assert_field_close(accpot: np.ndarray, acc_ref: np.ndarray, pot_ref: np.ndarray,
                       precision: str, what: str = ""):
    ea = rel_acc_err(accpot[:, :3], acc_ref)
    ep = rel_pot_err(accpot[:, 3], pot_ref)
    tol = TOL[precision]
    msg = (f"{what} {precision}: acc median {np.median(ea):.3e} p99 {np.quantile(ea, 0.99):.3e} "
           f"max {ea.max():.3e}; pot median {np.median(ep):.3e} max {ep.max():.3e}")
    assert np.median(ea) <= tol["median"], msg
    assert ea.max() <= tol["max"], msg
    assert np.median(ep) <= tol["median"], msg
    assert ep.max() <= tol["max"], msg
    return ea, ep


def hernquist(n, seed=0, axes=(1.0, 0.8, 0.6)):
    return inputs.hernquist(n, seed=seed, axes=axes)
