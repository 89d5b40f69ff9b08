"""GPU-vs-oracle parity of the fused stencil/RHS/RK4 kernels, through the
C ABI (ctypes binding).  Gate: scaled error <= 1e-12 after one RHS and
<= 1e-10 after many RK4 steps (per variable v: |a-b| / max(|b|, max|b_v|))."""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth
from helpers import scaled_err, to_gpu, to_np

pytestmark = pytest.mark.gpu

RHS_TOL = 1e-12
RK4_TOL = 1e-10


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1764_gb300 import api as A
    A.lib()
    return A


@pytest.mark.parametrize("dims,g,nv", [((17, 9, 11), 3, 24), ((32, 32, 32), 2, 2), ((5, 7, 4), 3, 2)])
def test_ghost_fill_bitwise(api, orc, dims, g, nv):
    nx, ny, nz = dims
    kind = api.BSSN if nv == 24 else api.WAVE
    sysm = api.make_system(kind, nx, ny, nz, 1.0 / nx, nghost=g)
    rng = np.random.default_rng(0)
    a = rng.standard_normal((nv, nz + 2 * g, ny + 2 * g, nx + 2 * g))
    t = to_gpu(a)
    sysm.fill_ghosts(t)
    want = a.copy()
    orc.fill_ghosts(want, g)
    assert np.array_equal(to_np(t), want)


def _wave_cases():
    return [(12, 16, 20), (32, 32, 32), (33, 9, 7)]


@pytest.mark.parametrize("dims", _wave_cases())
def test_wave_rhs(api, orc, dims):
    nx, ny, nz = dims
    g, h = 2, 1.0 / nx
    rng = np.random.default_rng(1)
    st = synth.pad(rng.standard_normal((2, nz, ny, nx)), g)
    orc.fill_ghosts(st, g)
    want = orc.wave_rhs(st, g, h)
    sysm = api.make_system(api.WAVE, nx, ny, nz, h)
    got = to_np(sysm.rhs(to_gpu(st)))
    assert scaled_err(got, want, g) <= RHS_TOL


def test_wave_plane_100_steps(api, orc):
    """The 32^3 plane-wave workload: 100 RK4 steps, dt = h/4."""
    n, g = 32, 2
    y0, h = synth.plane_wave(n, g)
    want = orc.rk4(orc.WAVE, y0, g, h, 0.25 * h, 100)
    sysm = api.make_system(api.WAVE, n, n, n, h)
    t = to_gpu(y0)
    sysm.rk4_step(t, 0.25 * h, 100)
    got = to_np(t)
    assert scaled_err(got, want, g) <= RK4_TOL
    assert np.array_equal(got[:, :g], got[:, n:n + g])  # ghosts refilled on return


def test_wave_pulses(api, orc):
    n, g = 48, 2
    y0, h = synth.gaussian_pulses(n, g, seed=1)
    want = orc.rk4(orc.WAVE, y0, g, h, 0.25 * h, 20)
    sysm = api.make_system(api.WAVE, n, n, n, h)
    t = to_gpu(y0)
    sysm.rk4_step(t, 0.25 * h, 20)
    assert scaled_err(to_np(t), want, g) <= RK4_TOL


@pytest.mark.parametrize("dims", [(12, 16, 20), (32, 32, 32)])
def test_varc_rhs(api, orc, dims):
    nx, ny, nz = dims
    g, h = 2, 1.0 / nx
    rng = np.random.default_rng(2)
    st = synth.pad(rng.standard_normal((2, nz, ny, nx)), g)
    orc.fill_ghosts(st, g)
    c = synth.pad(1.0 + 0.2 * rng.uniform(-1, 1, (nz, ny, nx)), g)[0]
    s = (c * c).copy()
    orc.fill_ghosts(s, g)
    want = orc.varc_rhs(st, s, g, h)
    sysm = api.make_system(api.WAVE_VARC, nx, ny, nz, h)
    sysm.set_speed(to_gpu(c))
    got = to_np(sysm.rhs(to_gpu(st)))
    assert scaled_err(got, want, g) <= RHS_TOL


def _bssn_random(dims, amp, seed, g=3):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    st = synth.pad(synth.BSSN_FLAT[:, None, None, None] + amp * rng.standard_normal((24, nz, ny, nx)), g)
    return st


@pytest.mark.parametrize("dims,amp", [((17, 9, 11), 1e-10), ((17, 9, 11), 3e-2), ((32, 32, 32), 1e-10),
                                      ((40, 12, 9), 3e-2)])
def test_bssn_rhs(api, orc, dims, amp):
    nx, ny, nz = dims
    g, h = 3, 1.0 / nx
    st = _bssn_random(dims, amp, seed=3)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h)
    sysm = api.make_system(api.BSSN, nx, ny, nz, h)
    got = to_np(sysm.rhs(to_gpu(st)))
    assert scaled_err(got, want, g) <= RHS_TOL


@pytest.mark.parametrize("slicing,shift", [(1, 1), (2, 1), (0, 1), (1, 0)])
def test_bssn_rhs_gauge_options(api, orc, slicing, shift):
    dims = (16, 12, 10)
    g, h = 3, 1.0 / 16
    st = _bssn_random(dims, 3e-2, seed=4)
    orc.fill_ghosts(st, g)
    prm_o = orc.Params(0.1, 1.5, slicing, shift)
    want = orc.bssn_rhs(st, g, h, prm_o)
    sysm = api.make_system(api.BSSN, *dims, h, params=api.default_params(0.1, 1.5, slicing, shift))
    got = to_np(sysm.rhs(to_gpu(st)))
    assert scaled_err(got, want, g) <= RHS_TOL


def test_bssn_rk4_noise(api, orc):
    n, g = 24, 3
    st, h = synth.bssn_noise(n, n, n, g, seed=2)
    want = orc.rk4(orc.BSSN, st, g, h, 0.25 * h, 20)
    sysm = api.make_system(api.BSSN, n, n, n, h)
    t = to_gpu(st)
    sysm.rk4_step(t, 0.25 * h, 20)
    assert scaled_err(to_np(t), want, g) <= RK4_TOL


def test_bssn_rk4_strong(api, orc):
    """Large perturbations drive every nonlinear term."""
    dims = (20, 14, 12)
    g, h = 3, 1.0 / 20
    st = _bssn_random(dims, 1e-2, seed=5)
    want = orc.rk4(orc.BSSN, st, g, h, 0.25 * h, 10)
    sysm = api.make_system(api.BSSN, *dims, h)
    t = to_gpu(st)
    sysm.rk4_step(t, 0.25 * h, 10)
    assert scaled_err(to_np(t), want, g) <= RK4_TOL


@pytest.mark.slow
def test_bssn_128_rhs_full_size(api, orc):
    """The BSSN 128^3 workload (flat + 1e-10 noise): one RHS, every point."""
    n, g = 128, 3
    st, h = synth.bssn_noise(n, n, n, g, seed=2)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h)
    sysm = api.make_system(api.BSSN, n, n, n, h)
    got = to_np(sysm.rhs(to_gpu(st)))
    assert scaled_err(got, want, g) <= RHS_TOL


@pytest.mark.slow
def test_bssn_100_steps(api, orc):
    """100 RK4 steps of flat + 1e-10 noise (64^3, the oracle's affordable
    size for the 100-step gate)."""
    n, g = 64, 3
    st, h = synth.bssn_noise(n, n, n, g, seed=2)
    want = orc.rk4(orc.BSSN, st, g, h, 0.25 * h, 100)
    sysm = api.make_system(api.BSSN, n, n, n, h)
    t = to_gpu(st)
    sysm.rk4_step(t, 0.25 * h, 100)
    assert scaled_err(to_np(t), want, g) <= RK4_TOL
