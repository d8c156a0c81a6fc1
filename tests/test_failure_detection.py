"""Failure detection on the GPU without faulting it.

* Every inter-block wait in the kernels is bounded.  Two of them are made to
  run out on purpose: the radix sort's decoupled lookback (a predecessor tile
  that never publishes) and the tcgen05 products' mbarrier wait (a barrier
  nothing arrives on, with tensor memory held).  Each must return, leave
  ETICS_ERR_TIMEOUT in the device error word, and leave the context usable:
  a later ordinary call gives the same bits as before.
* A whole MEX call whose lookback bound is cut to one poll must also return
  without touching memory outside its buffers (an order entry >= N is skipped
  downstream) and report the timeout.
* Data errors: a NaN or Inf particle gives ETICS_ERR_NONFINITE from SCF, MEX
  and the leapfrog step.
* A workspace one byte short is refused synchronously with
  ETICS_ERR_WORKSPACE by every call that takes one.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1406_4254_gb300 import etics, inputs

pytestmark = pytest.mark.gpu


def _particles(n, seed, dtype=torch.float32):
    return torch.tensor(inputs.hernquist(n, seed=seed, axes=(1.0, 0.8, 0.6)), dtype=dtype,
                        device="cuda")


def test_lookback_wait_runs_out_and_the_context_stays_usable():
    x = _particles(50000, 3)
    ref = etics.mex_field(x, 6)
    assert etics.get_error() == 0
    etics.probe_wait_timeout(etics.WAIT_LOOKBACK, 64)
    assert etics.get_error() == etics.ERR_TIMEOUT
    assert etics.get_error() == 0          # the word was cleared by the read
    again = etics.mex_field(x, 6)
    assert etics.get_error() == 0
    assert torch.equal(again, ref)


def test_mbarrier_wait_runs_out_and_frees_tensor_memory():
    # a product large enough for the tcgen05 kernel (both output sides >= 64)
    dims = [256, 256]
    from paper_1406_4254_gb300 import surrogate
    net = surrogate.Mlp(dims, seed=5, device=torch.device("cuda"))
    g = torch.Generator(device="cuda").manual_seed(5)
    xb = torch.randn((512, 256), generator=g, device="cuda").to(torch.bfloat16)
    y0 = torch.empty((512, 256), dtype=torch.float32, device="cuda")
    net.forward(xb, y0)
    assert etics.get_error() == 0
    for _ in range(3):          # several times: tensor memory must come back each time
        etics.probe_wait_timeout(etics.WAIT_MBARRIER, 64)
        assert etics.get_error() == etics.ERR_TIMEOUT
    y1 = torch.empty_like(y0)
    net.forward(xb, y1)
    assert etics.get_error() == 0
    assert torch.equal(y0, y1)


def test_mex_call_with_a_one_poll_lookback_bound_returns_and_reports():
    n = 1 << 20
    x = _particles(n, 11)
    ws = etics.workspace(n, 0, 6, etics.MEX, etics.MIXED)
    ref = etics.mex_field(x, 6, ws=ws)
    assert etics.get_error() == 0
    seen = []
    try:
        etics.set_wait_limit(1)
        for _ in range(20):
            out = etics.mex_field(x, 6, ws=ws)
            seen.append(etics.get_error())
            if etics.ERR_TIMEOUT in seen:
                break
    finally:
        etics.set_wait_limit(0)
    assert etics.ERR_TIMEOUT in seen, seen
    # every error seen is the timeout (it is recorded first; later kernels
    # only skip what the broken order would have written out of bounds)
    assert set(seen) <= {0, etics.ERR_TIMEOUT}, seen
    again = etics.mex_field(x, 6, ws=ws)
    assert etics.get_error() == 0
    assert torch.equal(again, ref)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_nonfinite_particle_is_reported(bad, dtype):
    x = _particles(9000, 4, dtype)
    x[1234, 1] = bad
    etics.scf_coeffs(x, 10, 6)
    assert etics.get_error() == etics.ERR_NONFINITE
    etics.mex_field(x, 6)
    assert etics.get_error() == etics.ERR_NONFINITE
    # the leapfrog step: a non-finite velocity drifts the particle to NaN
    y = _particles(9000, 4, dtype)
    v = torch.zeros_like(y)
    v[77, 0] = bad
    acc, _ = etics.scf_force(y, 10, 6)
    assert etics.get_error() == 0
    etics.leapfrog_step(y, v, acc, 0.01, etics.SCF, 10, 6)
    assert etics.get_error() == etics.ERR_NONFINITE


@pytest.mark.parametrize("prec", [etics.MIXED, etics.FP64])
def test_short_workspace_is_refused(prec):
    lib = etics.load()
    dtype = torch.float32 if prec == etics.MIXED else torch.float64
    n = 20000
    x = _particles(n, 6, dtype)
    out = torch.empty_like(x)
    vel = torch.zeros_like(x)
    coeffs = torch.empty((11, 49), dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    need_scf = etics.workspace_bytes(n, 10, 6, etics.SCF, prec)
    need_mex = etics.workspace_bytes(n, 0, 6, etics.MEX, prec)
    assert need_scf > 0 and need_mex > 0
    big = torch.empty(max(need_scf, need_mex) + 4096, dtype=torch.uint8, device="cuda")
    wp, _ = etics._aligned_ptr(big)
    assert lib.etics_scf_coeffs(x.data_ptr(), n, 10, 6, prec, coeffs.data_ptr(), wp,
                                need_scf - 1, s) == etics.ERR_WORKSPACE
    assert lib.etics_mex_field(x.data_ptr(), n, 6, prec, out.data_ptr(), 3, wp, need_mex - 1,
                               s) == etics.ERR_WORKSPACE
    # leapfrog with SCF and no coefficient output keeps the coefficients at
    # the end of its workspace: it needs that much more
    extra = ((11 * 49 * 8 + 255) // 256) * 256
    assert lib.etics_leapfrog_step(x.data_ptr(), vel.data_ptr(), out.data_ptr(), n, 0.01,
                                   etics.SCF, 10, 6, prec, None, wp, need_scf + extra - 1,
                                   s) == etics.ERR_WORKSPACE
    assert lib.etics_leapfrog_step(x.data_ptr(), vel.data_ptr(), out.data_ptr(), n, 0.01,
                                   etics.MEX, 0, 6, prec, None, wp, need_mex - 1,
                                   s) == etics.ERR_WORKSPACE
    assert lib.etics_test_wait_timeout(etics.WAIT_LOOKBACK, 8, wp,
                                       etics.workspace_bytes(etics.TIMEOUT_PROBE_N, 0, 0,
                                                             etics.MEX, etics.MIXED) - 1,
                                       s) == etics.ERR_WORKSPACE
    # nothing was launched, so nothing was recorded
    assert etics.get_error() == 0
    np.testing.assert_equal(torch.isfinite(x).all().item(), True)
