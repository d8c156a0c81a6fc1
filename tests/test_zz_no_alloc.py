"""The allocation-free SCF coefficient entry point (etics_scf_coeffs_noalloc).

It serves callers that cannot allocate device memory or hand the library a
buffer (a hard real-time loop, or a host that owns all device memory); its
scratch is a fixed array inside the library.  This file is collected last on
purpose so that a run stopping at the first failure has already run every
other test.
"""
import ctypes

import pytest
import torch

from paper_1406_4254_gb300 import etics, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_noalloc_matches_workspace_entry_point_twice(dtype):
    """Two calls in a row through the C ABI give the bits of etics_scf_coeffs:
    the same kernels with the same fixed-order reduction run on both."""
    pm = inputs.hernquist(30011, seed=41, axes=(1.0, 0.8, 0.6))
    x = torch.tensor(pm, dtype=dtype, device="cuda")
    for n_max, l_max in [(10, 6), (4, 2)]:
        ref = etics.scf_coeffs(x, n_max, l_max)
        for _ in range(2):
            got = etics.scf_coeffs_noalloc(x, n_max, l_max)
            etics.check_error()
            assert torch.equal(got, ref)


def test_noalloc_rejects_expansions_beyond_its_scratch():
    """(n_max, l_max) = (16, 14) needs more scratch than the fixed array holds
    on a GPU of this size; the call is refused with ETICS_ERR_WORKSPACE."""
    lib = etics.load()
    x = torch.tensor(inputs.hernquist(1000, seed=1), dtype=torch.float32, device="cuda")
    need = etics.workspace_bytes(1000, 16, 14, etics.SCF, etics.MIXED)
    assert need > etics.STATIC_SCRATCH_BYTES
    out = torch.empty((17, 225), dtype=torch.float64, device="cuda")
    rc = lib.etics_scf_coeffs_noalloc(x.data_ptr(), 1000, 16, 14, etics.MIXED, out.data_ptr(),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == etics.ERR_WORKSPACE
    etics.check_error()
