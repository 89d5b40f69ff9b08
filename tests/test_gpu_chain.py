"""Launch-chained RK4 steps of the order-4 scalar wave
(chemora_system_set_chain: stage kernels reading periodic images, chained by
programmatic dependent launches): bit-equal to the per-stage kernels on
every grid shape, including step counts that are not a multiple of the
graph's 8 steps, and equal to the oracle on the 32^3 plane-wave workload."""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth
from helpers import scaled_err, to_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1764_gb300 import api as A
    A.lib()
    return A


@pytest.mark.parametrize("dims,steps", [((32, 32, 32), 19), ((21, 13, 9), 5), ((3, 2, 4), 4), ((64, 40, 24), 3)])
def test_chain_bit_equal_to_stage_kernels(api, dims, steps):
    nx, ny, nz = dims
    rng = np.random.default_rng(nx * 7 + ny)
    y0 = synth.pad(rng.standard_normal((2, nz, ny, nx)), 2)
    h = 1.0 / nx
    sysm = api.make_system(api.WAVE, nx, ny, nz, h)
    assert sysm.set_chain(0) == 0
    a = to_gpu(y0)
    sysm.rk4_step(a, 0.25 * h, steps)
    assert sysm.set_chain(1) == 1
    b = to_gpu(y0)
    sysm.rk4_step(b, 0.25 * h, steps)
    assert np.array_equal(to_np(a), to_np(b))  # ghosts included: filled at the end of the call
    sysm.rk4_step(b, 0.25 * h, 0)
    assert np.array_equal(to_np(a), to_np(b))


def test_chain_plane_wave_100_steps_matches_oracle(api, orc):
    n, g = 32, 2
    y0, h = synth.plane_wave(n, g)
    want = orc.rk4(orc.WAVE, y0, g, h, 0.25 * h, 100)
    sysm = api.make_system(api.WAVE, n, n, n, h)
    sysm.set_chain(1)
    t = to_gpu(y0)
    sysm.rk4_step(t, 0.25 * h, 100)
    assert scaled_err(to_np(t), want, g) <= 1e-10


def test_chain_unavailable_for_other_systems(api):
    from paper_1410_1764_gb300._native import ChemoraError
    sysm = api.make_system(api.BSSN, 8, 8, 8, 1.0 / 8)
    with pytest.raises(ChemoraError):
        sysm.set_chain(1)
    w6 = api.make_system(api.WAVE, 8, 8, 8, 1.0 / 8, params=api.default_params(fd_order=6), nghost=3)
    with pytest.raises(ChemoraError):
        w6.set_chain(1)
    assert w6.set_chain(-1) == 0


def test_chain_state_pointer_change_recaptures(api):
    """The captured graphs are keyed by the state pointer and dt: stepping
    another state, or with another dt, gives the per-stage kernels' bits."""
    n = 12
    rng = np.random.default_rng(9)
    y0 = synth.pad(rng.standard_normal((2, n, n, n)), 2)
    y1 = synth.pad(rng.standard_normal((2, n, n, n)), 2)
    h = 1.0 / n
    sysm = api.make_system(api.WAVE, n, n, n, h)
    ref = api.make_system(api.WAVE, n, n, n, h)
    sysm.set_chain(1)
    for y, dt in ((y0, 0.25 * h), (y1, 0.25 * h), (y1, 0.2 * h)):
        a, b = to_gpu(y), to_gpu(y)
        sysm.rk4_step(a, dt, 11)
        ref.rk4_step(b, dt, 11)
        assert np.array_equal(to_np(a), to_np(b))


def test_autotune_keeps_a_mode_with_equal_results(api):
    n = 32
    y0, h = synth.plane_wave(n, 2)
    sysm = api.make_system(api.WAVE, n, n, n, h)
    t = to_gpu(y0)
    sysm.autotune(t)
    chosen = sysm.set_chain(-1)
    assert chosen in (0, 1)
    a = to_gpu(y0)
    sysm.rk4_step(a, 0.25 * h, 10)
    sysm.set_chain(0)
    b = to_gpu(y0)
    sysm.rk4_step(b, 0.25 * h, 10)
    assert np.array_equal(to_np(a), to_np(b))
