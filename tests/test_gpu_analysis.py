"""GPU analysis kernels: BSSN constraints against the oracle (and their 4th-
order convergence on the gauge wave, measured on the GPU), the discrete wave
energy against its definition evaluated with the oracle's Laplacian."""
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


@pytest.mark.parametrize("dims,amp", [((17, 9, 11), 3e-2), ((24, 24, 24), 1e-10)])
def test_constraints_match_oracle(api, orc, dims, amp):
    nx, ny, nz = dims
    g, h = 3, 1.0 / nx
    rng = np.random.default_rng(8)
    st = synth.pad(synth.BSSN_FLAT[:, None, None, None] + amp * rng.standard_normal((24, nz, ny, nx)), g)
    orc.fill_ghosts(st, g)
    want = orc.bssn_constraints(st, g, h)
    sysm = api.make_system(api.BSSN, nx, ny, nz, h)
    got = to_np(sysm.constraints(to_gpu(st)))
    assert scaled_err(got, want, g) <= 1e-12


def test_constraints_gauge_wave_converge(api):
    from test_oracle_bssn import gauge_wave_state
    errs = []
    for nx in (32, 64, 128):
        st, h = gauge_wave_state(nx, 6, 6, 0.0)
        sysm = api.make_system(api.BSSN, nx, 6, 6, h)
        c = to_np(sysm.constraints(to_gpu(st)))
        errs.append(np.abs(synth.interior(c, 3)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.5 and 14.0 < r2 < 18.0, errs


def test_wave_energy(api, orc):
    n, g = 24, 2
    y, h = synth.gaussian_pulses(n, g, seed=1, width=0.1)
    sysm = api.make_system(api.WAVE, n, n, n, h)
    t = to_gpu(y)
    sysm.fill_ghosts(t)
    yy = to_np(t)
    lap = orc.wave_rhs(np.stack([yy[0], yy[0]]), g, h)[1]
    want = 0.5 * np.sum(synth.interior(yy[1], g) ** 2 - synth.interior(yy[0], g) * synth.interior(lap, g)) * h ** 3
    E0 = sysm.energy(t)
    assert E0 == pytest.approx(want, rel=1e-12)
    assert sysm.energy(t) == E0  # deterministic
    prev = E0
    for _ in range(5):
        sysm.rk4_step(t, 0.25 * h, 2)
        E = sysm.energy(t)
        assert E <= prev * (1 + 1e-14)
        prev = E
    assert prev < E0
