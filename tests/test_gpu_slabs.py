"""z-slab decomposition on one GPU (several slabs in one process, halos by
device copies): RK4 through chemora_stage and chemora_fill_ghosts_axes on
the slabs equals the single-grid chemora_rk4_step bit for bit."""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth
from helpers import to_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1764_gb300 import api as A
    A.lib()
    return A


@pytest.mark.parametrize("kind,dims,parts", [("bssn", (20, 16, 30), 3), ("wave", (24, 10, 17), 3),
                                             ("wave", (16, 16, 16), 1)])
def test_slabs_equal_single_grid(api, kind, dims, parts):
    from paper_1410_1764_gb300 import slabs
    nx, ny, nz = dims
    rng = np.random.default_rng(2)
    if kind == "bssn":
        K, g = api.BSSN, 3
        st = synth.pad(synth.BSSN_FLAT[:, None, None, None] + 1e-3 * rng.standard_normal((24, nz, ny, nx)), g)
    else:
        K, g = api.WAVE, 2
        st = synth.pad(rng.standard_normal((2, nz, ny, nx)), g)
    h = 1.0 / nx
    whole = api.make_system(K, nx, ny, nz, h)
    ref = to_gpu(st)
    for _ in range(3):
        whole.rk4_step(ref, 0.25 * h, 1)
    pz = slabs.zslabs(nz, parts)
    states = [to_gpu(np.ascontiguousarray(st[:, z0:z0 + n + 2 * g])) for z0, n in pz]
    drv = slabs.SlabRK4(K, nx, ny, h, pz, slabs.LocalExchange(g))
    drv.step(states, 0.25 * h, 3)
    R = to_np(ref)
    for (z0, n), s in zip(pz, states):
        assert np.array_equal(to_np(s), R[:, z0:z0 + n + 2 * g])
