"""chemora_rk4_step_noalloc: RK4 steps for callers that cannot allocate
device memory (allocator hooks, host callbacks, frameworks that must account
for every allocation, real-time loops).  Its scratch is a fixed array inside
the library, so its results must equal those of chemora_rk4_step, which
allocates its own work states.

Called through the C ABI directly (ctypes), two calls in a row, compared
with the allocating entry point under the same tolerance as the other RK4
parity tests.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1410_1764_gb300 import synth
from helpers import scaled_err, to_gpu, to_np

RK4_TOL = 1e-10


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1764_gb300 import api as A
    A.lib()
    return A


def _noalloc(api, sysm, t, dt, nsteps):
    import torch
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return api.lib().chemora_rk4_step_noalloc(sysm.handle, ctypes.c_void_p(t.data_ptr()),
                                              ctypes.c_double(dt), nsteps, s)


@pytest.mark.gpu
@pytest.mark.parametrize("kind,n", [("wave", 32), ("bssn", 20)])
def test_noalloc_matches_allocating_step(api, kind, n):
    import torch
    if kind == "wave":
        y0, h = synth.plane_wave(n, 2)
        K = api.WAVE
    else:
        y0 = synth.pad(synth.BSSN_FLAT[:, None, None, None]
                       + 1e-3 * np.random.default_rng(9).standard_normal((24, n, n, n)), 3)
        h = 1.0 / n
        K = api.BSSN
    dt = 0.25 * h
    ref_sys = api.make_system(K, n, n, n, h)
    na_sys = api.make_system(K, n, n, n, h)
    ref = to_gpu(y0)
    got = to_gpu(y0)
    for call in range(2):
        ref_sys.rk4_step(ref, dt, 3)
        rc = _noalloc(api, na_sys, got, dt, 3)
        assert rc == 0, api.lib().chemora_last_error()
        g = 3 if K == api.BSSN else 2
        assert scaled_err(to_np(got), to_np(ref), g) <= RK4_TOL, "call %d" % call
    # after its first call on the device, a further call leaves free device
    # memory unchanged
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _noalloc(api, na_sys, got, dt, 1) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


@pytest.mark.gpu
def test_noalloc_rejects_oversize(api):
    n = 40  # 24 * 46^3 doubles per state: three of them exceed the static scratch
    sysm = api.make_system(api.BSSN, n, n, n, 1.0 / n)
    t = to_gpu(np.zeros(sysm.grid.shape))
    rc = _noalloc(api, sysm, t, 0.01, 1)
    assert rc == -1  # CHEMORA_EINVAL
    assert b"static scratch" in api.lib().chemora_last_error()
