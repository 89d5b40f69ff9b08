"""Arbitrary-order stencils and the first-order form of Eq. 1 on the GPU
against the oracle (which computes its weights by a different method: the
closed-form factorial expression; the generator solves moment conditions)."""
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


CASES = [("wave", 2), ("wave", 6), ("wave", 8), ("wave1", 2), ("wave1", 4), ("wave1", 6), ("wave1", 8)]


def _state(kind, dims, g, rng):
    nx, ny, nz = dims
    nv = 2 if kind == "wave" else 5
    return synth.pad(rng.standard_normal((nv, nz, ny, nx)), g)


@pytest.mark.parametrize("kind,order", CASES)
def test_rhs_and_rk4(api, orc, kind, order):
    dims = (19, 12, 10)
    g = max(2, order // 2)
    h = 1.0 / 19
    rng = np.random.default_rng(order)
    st = _state(kind, dims, g, rng)
    orc.fill_ghosts(st, g)
    K = api.WAVE if kind == "wave" else api.WAVE1
    okind = orc.WAVE if kind == "wave" else orc.WAVE1
    prm = orc.default_params(order)
    want = orc.rhs(okind, st, g, h, params=prm)
    sysm = api.make_system(K, *dims, h, params=api.default_params(fd_order=order), nghost=g)
    got = to_np(sysm.rhs(to_gpu(st)))
    assert scaled_err(got, want, g) <= 1e-12
    y = orc.rk4(okind, st, g, h, 0.25 * h, 12, params=prm)
    t = to_gpu(st)
    sysm.rk4_step(t, 0.25 * h, 12)
    assert scaled_err(to_np(t), y, g) <= 1e-10


def test_wave1_shapes_identical(api):
    n, g = 21, 2
    st = _state("wave1", (n, 13, 9), g, np.random.default_rng(3))
    sysm = api.make_system(api.WAVE1, n, 13, 9, 1.0 / n)
    T = to_gpu(st)
    sysm.fill_ghosts(T)
    outs = []
    for v in range(api.lib().chemora_variant_count(api.WAVE1)):
        sysm.variant(v)
        outs.append(to_np(sysm.rhs(T)))
    assert all(np.array_equal(o, outs[0]) for o in outs)
