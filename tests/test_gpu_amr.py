"""Two-level mesh refinement with Berger-Oliger subcycling on the GPU
against the oracle: coarse and fine interiors after several coarse steps."""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth
from helpers import scaled_err, to_gpu, to_np
from test_oracle_amr import _coarse_coords, _fine_coords, _plane

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1764_gb300 import api as A
    A.lib()
    return A


@pytest.mark.parametrize("nc,lo,hi,steps", [(24, (6, 6, 6), (15, 15, 15), 3), (28, (4, 7, 5), (13, 20, 18), 4)])
def test_amr_matches_oracle(api, orc, nc, lo, hi, steps):
    H = 1.0 / nc
    cfg = orc.amr(nc, lo, hi, H)
    Zc, Yc, Xc = _coarse_coords(nc, 2, H)
    Zf, Yf, Xf = _fine_coords(cfg)
    rng = np.random.default_rng(nc)
    coarse = np.ascontiguousarray(_plane(Xc, Yc, Zc, 0.0) + 0.01 * rng.standard_normal(Xc.shape))
    fine = np.ascontiguousarray(_plane(Xf, Yf, Zf, 0.0))
    amr = api.Amr(nc, lo, hi, H)
    amr.state(0).copy_(to_gpu(coarse))
    amr.state(1).copy_(to_gpu(fine))
    dt = 0.25 * H
    orc.amr_step(cfg, coarse, fine, dt, steps)
    amr.step(dt, steps - 1)
    amr.step(dt, 1)  # two calls continue where the first stopped
    gc = to_np(amr.state(0))
    gf = to_np(amr.state(1))
    assert scaled_err(gc, coarse, 2) <= 1e-10
    assert scaled_err(gf, fine, cfg.gf) <= 1e-10


def test_amr_rejects_boxes_too_close_to_the_edge(api):
    from paper_1410_1764_gb300._native import ChemoraError
    with pytest.raises(ChemoraError):
        api.Amr(16, (3, 4, 4), (8, 8, 8), 1.0 / 16)
    with pytest.raises(ChemoraError):
        api.Amr(16, (4, 4, 4), (12, 8, 8), 1.0 / 16)
