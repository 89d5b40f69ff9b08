"""Run-time specialised BSSN stage kernels (NVRTC; Sec. 3.2.3's run-time
compilation with the parameter values known): parity with the oracle and with
the ahead-of-time kernels, for every kind of launch shape, through the C ABI."""
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


def _state(dims, amp, seed, g=3):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    return synth.pad(synth.BSSN_FLAT[:, None, None, None] + amp * rng.standard_normal((24, nz, ny, nx)), g)


def _shapes(api):
    """Launch shapes by body: direct, x lanes, x lanes + shared y."""
    out = {"direct": [], "x": [], "xy": []}
    for v in range(api.lib().chemora_variant_count(api.BSSN)):
        out[("direct", "x", "xy")[api.variant_info(api.BSSN, v)[3]]].append(v)
    return out


@pytest.mark.parametrize("kind,nth", [("direct", 0), ("x", 1), ("xy", 0), ("xy", 1)])
def test_specialised_rhs_matches_oracle_and_aot(api, orc, kind, nth, tmp_path):
    dims = (64, 32, 10)      # several x warps and y blocks; every body applies
    g, h = 3, 1.0 / 64
    st = _state(dims, 3e-2, seed=11)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h)
    sysm = api.make_system(api.BSSN, *dims, h)
    sysm.variant(_shapes(api)[kind][nth])
    aot = to_np(sysm.rhs(to_gpu(st)))
    sysm.specialize(True, cache_dir=tmp_path)
    jit = to_np(sysm.rhs(to_gpu(st)))
    assert scaled_err(jit, want, g) <= RHS_TOL
    # same expression DAG and exact constants: at most contraction-order differences
    assert scaled_err(jit, aot, g) <= 1e-14


def test_specialised_ragged_grid_falls_back_to_direct_body(api, orc, tmp_path):
    """A grid the sharing bodies cannot tile (nx % 32 != 0): the specialised
    kernel takes the direct body, like the ahead-of-time dispatch."""
    dims = (17, 9, 11)
    g, h = 3, 1.0 / 17
    st = _state(dims, 1e-10, seed=3)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h)
    sysm = api.make_system(api.BSSN, *dims, h)
    sysm.variant(_shapes(api)["xy"][1])
    sysm.specialize(True, cache_dir=tmp_path)
    assert scaled_err(to_np(sysm.rhs(to_gpu(st))), want, g) <= RHS_TOL


@pytest.mark.parametrize("slicing,shift", [(1, 1), (2, 0)])
def test_specialised_gauge_constants(api, orc, slicing, shift, tmp_path):
    """The gauge switches and eta become compile-time constants."""
    dims = (32, 16, 8)
    g, h = 3, 1.0 / 32
    st = _state(dims, 3e-2, seed=4)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h, orc.Params(0.07, 1.5, slicing, shift))
    sysm = api.make_system(api.BSSN, *dims, h, params=api.default_params(0.07, 1.5, slicing, shift))
    sysm.variant(_shapes(api)["xy"][1])
    sysm.specialize(True, cache_dir=tmp_path)
    assert scaled_err(to_np(sysm.rhs(to_gpu(st))), want, g) <= RHS_TOL


def test_specialised_rk4_steps(api, orc, tmp_path):
    """Every stage mode's kernel, inside the captured RK4 step graph."""
    n, g = 32, 3
    h = 1.0 / n
    st = _state((n, n, n), 1e-3, seed=7)
    want = orc.rk4(orc.BSSN, st, g, h, 0.25 * h, 10)
    sysm = api.make_system(api.BSSN, n, n, n, h)
    sysm.variant(_shapes(api)["xy"][1])
    sysm.specialize(True, cache_dir=tmp_path)
    t = to_gpu(st)
    sysm.rk4_step(t, 0.25 * h, 10)
    assert scaled_err(to_np(t), want, g) <= RK4_TOL


def test_cache_toggle_and_variant_change(api, tmp_path):
    n, g = 32, 3
    h = 1.0 / n
    st = _state((n, n, n), 1e-3, seed=8)
    xy = _shapes(api)["xy"][1]
    a = api.make_system(api.BSSN, n, n, n, h)
    a.variant(xy)
    a.specialize(True, cache_dir=tmp_path)
    b = api.make_system(api.BSSN, n, n, n, h)
    b.variant(xy)
    assert b.specialize(True, cache_dir=tmp_path) == 0.0   # every cubin from the cache
    ref = to_np(a.rhs(to_gpu(st)))
    l0 = api.launch_count()
    got = to_np(b.rhs(to_gpu(st)))
    assert api.launch_count() - l0 == 1
    assert np.array_equal(got, ref)
    # back to the ahead-of-time kernel, then on again (kept module: no compile)
    b.specialize(False)
    aot = to_np(b.rhs(to_gpu(st)))
    assert scaled_err(aot, ref, g) <= 1e-14
    assert b.specialize(True, cache_dir="") == 0.0
    # another launch shape: the ahead-of-time kernels run until re-specialised
    b.variant(0)
    assert scaled_err(to_np(b.rhs(to_gpu(st))), ref, g) <= 1e-14


@pytest.mark.parametrize("dims", [(32, 13, 5), (64, 3, 4), (32, 1, 6)])
def test_xy_bodies_on_ragged_rows(api, orc, dims, tmp_path):
    """ny not a multiple of the block's rows (and ny below it): the last row
    of blocks computes its clamped prologue rows, passes the barrier and
    leaves; every x/y-sharing shape, ahead-of-time and specialised."""
    g, h = 3, 1.0 / dims[0]
    st = _state(dims, 3e-2, seed=12)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h)
    for v in _shapes(api)["xy"]:
        sysm = api.make_system(api.BSSN, *dims, h)
        sysm.variant(v)
        assert sysm.opcount()[0] < api.opcount(api.BSSN)[0]   # the x/y body runs, no fall-back
        assert scaled_err(to_np(sysm.rhs(to_gpu(st))), want, g) <= RHS_TOL, v
        sysm.specialize(True, cache_dir=tmp_path)
        assert scaled_err(to_np(sysm.rhs(to_gpu(st))), want, g) <= RHS_TOL, v


@pytest.mark.slow
def test_bench_configuration_full_size(api, orc, tmp_path):
    """The timed configuration of the bench: BSSN 128^3, flat space with
    1e-10 noise, the autotuned launch shape compiled at run time; one RHS on
    every point (1e-12) and one RK4 step (1e-10) against the oracle."""
    import torch
    n, g = 128, 3
    st, h = synth.bssn_noise(n, n, n, g, seed=2)
    sysm = api.make_system(api.BSSN, n, n, n, h)
    t = torch.from_numpy(st).cuda()
    sysm.autotune(t)
    sysm.specialize(True, cache_dir=tmp_path)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h)
    assert scaled_err(to_np(sysm.rhs(to_gpu(st))), want, g) <= RHS_TOL
    y = orc.rk4(orc.BSSN, st, g, h, 0.25 * h, 1)
    t = to_gpu(st)
    sysm.rk4_step(t, 0.25 * h, 1)
    assert scaled_err(to_np(t), y, g) <= RK4_TOL
