"""Batched patches on the GPU: every patch equals the oracle's single-grid
RK4 on that patch, and the batched (persistent + graph) schedule is bitwise
identical to per-patch launches."""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth
from helpers import scaled_err, to_np

pytestmark = pytest.mark.gpu

DIMS = [(12, 9, 7), (16, 16, 16), (5, 20, 11), (33, 8, 9), (17, 13, 19), (1, 3, 2)]


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1764_gb300 import api as A
    A.lib()
    return A


def _load(batch, states):
    for p, st in enumerate(states):
        v = batch.state(p)
        v.copy_(__import__("torch").from_numpy(st))


@pytest.mark.parametrize("kind", ["bssn", "wave"])
def test_batched_matches_oracle_and_per_patch(api, orc, kind):
    rng = np.random.default_rng(4)
    if kind == "bssn":
        K, g, nv, okind = api.BSSN, 3, 24, orc.BSSN
        states = [synth.pad(synth.BSSN_FLAT[:, None, None, None]
                            + 1e-3 * rng.standard_normal((nv, nz, ny, nx)), g) for nx, ny, nz in DIMS]
    else:
        K, g, nv, okind = api.WAVE, 2, 2, orc.WAVE
        states = [synth.pad(rng.standard_normal((nv, nz, ny, nx)), g) for nx, ny, nz in DIMS]
    h = 1.0 / 64
    dt = 0.25 * h
    b0 = api.Batch(DIMS, g, h, kind=K)
    b1 = api.Batch(DIMS, g, h, kind=K)
    _load(b0, states)
    _load(b1, states)
    b0.step(dt, 3, mode=0)
    b1.step(dt, 3, mode=1)
    for p, st in enumerate(states):
        a0 = to_np(b0.state(p))
        a1 = to_np(b1.state(p))
        assert np.array_equal(a0, a1), "patch %d: batched and per-patch differ" % p
        want = orc.rk4(okind, st, g, h, dt, 3)
        assert scaled_err(a0, want, g) <= 1e-10, "patch %d" % p


def test_batched_dt_change_recaptures(api, orc):
    rng = np.random.default_rng(5)
    dims = DIMS[:3]
    states = [synth.pad(rng.standard_normal((2, nz, ny, nx)), 2) for nx, ny, nz in dims]
    h = 1.0 / 32
    b = api.Batch(dims, 2, h, kind=api.WAVE)
    _load(b, states)
    b.step(0.25 * h, 2, mode=0)
    b.step(0.125 * h, 2, mode=0)
    for p, st in enumerate(states):
        want = orc.rk4(orc.WAVE, orc.rk4(orc.WAVE, st, 2, h, 0.25 * h, 2), 2, h, 0.125 * h, 2)
        assert scaled_err(to_np(b.state(p)), want, 2) <= 1e-10


def test_batched_cfg_sizes(api, orc):
    """Patch sizes from the 64-patch recipe (first 4 patches, sides in
    [16, 96]), flat + 1e-10 noise, 2 steps: batched vs oracle per patch."""
    states, dims, h = synth.bssn_patches(seed=3, npatch=4)
    b = api.Batch([tuple(d) for d in dims], 3, h, kind=api.BSSN)
    _load(b, states)
    dt = 0.25 * h
    b.step(dt, 2, mode=0)
    for p, st in enumerate(states):
        want = orc.rk4(orc.BSSN, st, 3, h, dt, 2)
        assert scaled_err(to_np(b.state(p)), want, 3) <= 1e-10, p
