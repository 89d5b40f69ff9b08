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


def _boxes_state(orc, kind, nc, boxes, H, seed):
    """Coarse and box states with smooth data plus small random
    perturbations (wave: a plane wave; BSSN: flat space + 1e-3 noise)."""
    rng = np.random.default_rng(seed)
    r = 3 if kind == orc.BSSN else 2
    gc, gf = r, 4 * r
    nv = 24 if kind == orc.BSSN else 2
    base = synth.BSSN_FLAT if kind == orc.BSSN else np.zeros(2)
    amp = 1e-3 if kind == orc.BSSN else 1.0
    coarse = synth.pad(base[:, None, None, None] + amp * rng.standard_normal((nv, nc[2], nc[1], nc[0])), gc)
    orc.fill_ghosts(coarse, gc)
    fines = []
    for lo, hi in boxes:
        nf = [2 * (hi[d] - lo[d]) for d in range(3)]
        fines.append(synth.pad(base[:, None, None, None] + amp * rng.standard_normal((nv, nf[2], nf[1], nf[0])), gf))
    return coarse, fines, gc, gf


AMR_BOX_CASES = [
    ("wave", (26, 22, 24), [((4, 4, 5), (9, 10, 11)), ((12, 5, 4), (19, 9, 9)), ((5, 12, 12), (10, 17, 19))], 3),
    ("bssn", (24, 20, 22), [((5, 5, 5), (9, 9, 10)), ((11, 6, 6), (17, 10, 11)), ((5, 10, 12), (8, 14, 16))], 2),
]


@pytest.mark.parametrize("name,nc,boxes,steps", AMR_BOX_CASES)
def test_amr_boxes_match_oracle(api, orc, name, nc, boxes, steps):
    """Several boxes of uneven sizes on a non-cubic coarse grid, both the
    batched schedule (one persistent launch per fine stage over every box)
    and box-by-box launches, against the oracle's two-level step; the two
    schedules agree bit for bit."""
    kind_o = orc.BSSN if name == "bssn" else orc.WAVE
    kind_g = api.BSSN if name == "bssn" else api.WAVE
    H = 1.0 / nc[0]
    coarse, fines, gc, gf = _boxes_state(orc, kind_o, nc, boxes, H, seed=7)
    got = {}
    for mode in (0, 1):
        amr = api.AmrBoxes(kind_g, nc, boxes, H)
        amr.state(0).copy_(to_gpu(coarse))
        for b, f in enumerate(fines):
            amr.state(1 + b).copy_(to_gpu(f))
        amr.step(0.25 * H, steps - 1, mode=mode)
        amr.step(0.25 * H, 1, mode=mode)  # two calls continue where the first stopped
        got[mode] = [to_np(amr.state(0))] + [to_np(amr.state(1 + b)) for b in range(len(boxes))]
    cfg = orc.amrn(nc, boxes, H, gc, gf)
    orc.amrn_step(cfg, kind_o, coarse, fines, 0.25 * H, steps)
    assert scaled_err(got[0][0], coarse, gc) <= 1e-10
    for b, f in enumerate(fines):
        assert scaled_err(got[0][1 + b], f, gf) <= 1e-10, b
    assert np.array_equal(got[0][0], got[1][0])
    for b in range(len(boxes)):
        assert np.array_equal(synth.interior(got[0][1 + b], gf), synth.interior(got[1][1 + b], gf))


def test_amr_boxes_single_box_wave_is_the_first_interface(api):
    """chemora_amr_create is the one-box scalar-wave case of
    chemora_amr_create_boxes: same layout, bit-equal steps."""
    import torch
    nc, lo, hi = 20, (4, 5, 6), (12, 11, 14)
    H = 1.0 / nc
    rng = np.random.default_rng(3)
    coarse = to_gpu(synth.pad(rng.standard_normal((2, nc, nc, nc)), 2))
    a = api.Amr(nc, lo, hi, H)
    b = api.AmrBoxes(api.WAVE, (nc, nc, nc), [(lo, hi)], H)
    assert a.state(1).shape == b.state(1).shape
    fine = to_gpu(rng.standard_normal(tuple(a.state(1).shape)))
    for m in (a, b):
        m.state(0).copy_(coarse)
        m.state(1).copy_(fine)
    a.step(0.25 * H, 2)
    b.step(0.25 * H, 2)
    torch.cuda.synchronize()
    assert torch.equal(a.state(0), b.state(0))
    assert torch.equal(a.state(1)[:, 8:-8, 8:-8, 8:-8], b.state(1)[:, 8:-8, 8:-8, 8:-8])


def test_amr_boxes_autotuned_coarse_kernel_matches_oracle(api, orc):
    """With the coarse stage kernel's launch shape picked by timing (on a
    coarse grid whose rows fill whole warps, so the lane-sharing bodies are
    candidates) the two-level BSSN step still matches the oracle."""
    nc, boxes, steps = (32, 20, 22), [((5, 5, 5), (11, 9, 10)), ((14, 6, 6), (24, 11, 12))], 2
    H = 1.0 / nc[0]
    coarse, fines, gc, gf = _boxes_state(orc, orc.BSSN, nc, boxes, H, seed=11)
    amr = api.AmrBoxes(api.BSSN, nc, boxes, H)
    amr.state(0).copy_(to_gpu(coarse))
    for b, f in enumerate(fines):
        amr.state(1 + b).copy_(to_gpu(f))
    v = amr.autotune()
    assert 0 <= v < api.lib().chemora_variant_count(api.BSSN)
    amr.state(0).copy_(to_gpu(coarse))  # autotuning overwrote only scratch; restore anyway
    amr.step(0.25 * H, steps)
    orc.amrn_step(orc.amrn(nc, boxes, H, gc, gf), orc.BSSN, coarse, fines, 0.25 * H, steps)
    assert scaled_err(to_np(amr.state(0)), coarse, gc) <= 1e-10
    for b, f in enumerate(fines):
        assert scaled_err(to_np(amr.state(1 + b)), f, gf) <= 1e-10


@pytest.mark.slow
def test_amr_boxes_bssn_gauge_wave_converges_on_gpu(api):
    """The BSSN gauge wave (harmonic slicing, zero shift: an exact solution)
    evolved by the library's two-level step with two refined boxes converges
    to the exact solution at 4th order on the coarse level and inside the
    boxes, through the buffer-zone interface (the oracle's pin, on the GPU
    path)."""
    from test_oracle_bssn import gauge_wave_state
    prm = api.default_params(slicing=1, shift=1)
    errs = []
    for nx in (20, 40, 80):
        m, gc, gf = 14, 3, 12
        H = 1.0 / nx
        s = nx // 20
        boxes = [((5 * s, 5, 5), (10 * s, 8, 8)), ((12 * s, 5, 5), (14 * s, 8, 8))]

        def exact_fine(lo, hi, t):
            big, _ = gauge_wave_state(2 * nx, 2 * m + 2 * gf, 2 * m + 2 * gf, t)
            sl = [slice(3 + 2 * lo[d] - gf + (gf if d else 0), 3 + 2 * hi[d] + gf + (gf if d else 0)) for d in range(3)]
            return np.ascontiguousarray(big[:, sl[2], sl[1], sl[0]])

        amr = api.AmrBoxes(api.BSSN, (nx, m, m), boxes, H, params=prm)
        amr.state(0).copy_(to_gpu(gauge_wave_state(nx, m, m, 0.0)[0]))
        for b, (lo, hi) in enumerate(boxes):
            amr.state(1 + b).copy_(to_gpu(exact_fine(lo, hi, 0.0)))
        dt = 0.25 * H
        nsteps = int(round(0.125 / dt))
        amr.step(dt, nsteps)
        t = nsteps * dt
        ec = np.abs(synth.interior(to_np(amr.state(0)) - gauge_wave_state(nx, m, m, t)[0], gc)).max()
        ef = max(np.abs(synth.interior(to_np(amr.state(1 + b)) - exact_fine(lo, hi, t), gf)).max()
                 for b, (lo, hi) in enumerate(boxes))
        errs.append((ec, ef))
    for q in (0, 1):
        e = [r[q] for r in errs]
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert 12.0 < r1 < 18.0 and 14.0 < r2 < 18.0, errs


@pytest.mark.parametrize("name,nc,boxes", [
    # boxes at the smallest allowed distance from the faces, one-point-thick
    # boxes (two fine points per axis), and boxes that touch each other
    ("wave", (15, 12, 13), [((4, 4, 4), (9, 5, 8)), ((9, 4, 4), (10, 7, 8))]),
    ("bssn", (17, 16, 18), [((5, 5, 5), (6, 10, 12)), ((6, 5, 5), (11, 6, 7))]),
])
def test_amr_edge_boxes_match_oracle(api, orc, name, nc, boxes):
    kind_o = orc.BSSN if name == "bssn" else orc.WAVE
    kind_g = api.BSSN if name == "bssn" else api.WAVE
    H = 1.0 / nc[0]
    coarse, fines, gc, gf = _boxes_state(orc, kind_o, nc, boxes, H, seed=21)
    amr = api.AmrBoxes(kind_g, nc, boxes, H)
    amr.state(0).copy_(to_gpu(coarse))
    for b, f in enumerate(fines):
        amr.state(1 + b).copy_(to_gpu(f))
    amr.step(0.25 * H, 2)
    orc.amrn_step(orc.amrn(nc, boxes, H, gc, gf), kind_o, coarse, fines, 0.25 * H, 2)
    assert scaled_err(to_np(amr.state(0)), coarse, gc) <= 1e-10
    for b, f in enumerate(fines):
        assert scaled_err(to_np(amr.state(1 + b)), f, gf) <= 1e-10, b
