"""Parity at the full sizes of the benchmarked workloads, in the launch
configurations the benchmark times (autotuned shapes, batched schedules),
against the oracle on every point or on whole sampled patches, and by
properties that hold at any length:

- scalar wave 256^3, 8 Gaussian pulses: 10 RK4 steps of the autotuned
  kernel against the oracle; over the configured 200 steps the discrete
  energy never increases (RK4 damps every mode) and stays finite;
- 64 batched BSSN patches (sides 16-96, flat space + 1e-10 noise): two
  batched RK4 steps bit-equal to per-patch launches on every patch, and
  equal to the oracle's single-grid RK4 on sampled patches (the smallest,
  the largest and two more);
- two-level BSSN refinement, coarse 128^3 with 8 boxes (sides 16-40): one
  coarse step of the batched schedule with the autotuned coarse kernel
  against the oracle's two-level step on both levels (1e-3 perturbations of
  flat space), and bit-equal to the box-by-box schedule.
"""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth
from helpers import scaled_err, to_gpu, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

RK4_TOL = 1e-10


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1764_gb300 import api as A
    A.lib()
    return A


def test_wave_256_pulses_full_size(api, orc):
    n, g = 256, 2
    y0, h = synth.gaussian_pulses(n, g, seed=1)
    dt = 0.25 * h
    sysm = api.make_system(api.WAVE, n, n, n, h)
    t = to_gpu(y0)
    sysm.autotune(t)
    want = orc.rk4(orc.WAVE, y0, g, h, dt, 10)
    sysm.rk4_step(t, dt, 10)
    assert scaled_err(to_np(t), want, g) <= RK4_TOL
    e_prev = sysm.energy(t)
    assert np.isfinite(e_prev) and e_prev > 0
    for _ in range(19):  # to the configured 200 steps
        sysm.rk4_step(t, dt, 10)
        e = sysm.energy(t)
        assert np.isfinite(e) and e <= e_prev * (1 + 1e-13), (e, e_prev)
        e_prev = e


def test_patches_64_full_configuration(api, orc):
    import torch
    states, dims, h = synth.bssn_patches(seed=3, npatch=64)
    dt = 0.25 * h
    batches = []
    for mode in (0, 1):
        b = api.Batch([tuple(int(v) for v in d) for d in dims], 3, h, kind=api.BSSN)
        for p, st in enumerate(states):
            b.state(p).copy_(torch.from_numpy(st))
        b.step(dt, 2, mode=mode)
        batches.append(b)
    torch.cuda.synchronize()
    for p in range(len(states)):
        assert torch.equal(batches[0].state(p), batches[1].state(p)), p
    sizes = [int(np.prod(d)) for d in dims]
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 40})
    for p in sample:
        want = orc.rk4(orc.BSSN, states[p], 3, h, dt, 2)
        assert scaled_err(to_np(batches[0].state(p)), want, 3) <= RK4_TOL, p


def test_amr_bssn_bench_configuration(api, orc):
    """The benchmark's two-level configuration (sizes, boxes, schedules) with
    1e-3 instead of 1e-10 perturbations: the prolongation interpolates the
    O(1) background in a different order on the two sides (three separable
    passes against the oracle's tensor-product sum), and one ulp of that
    background is 2e-6 of a 1e-10 perturbation, so the benchmark's own data
    would compare rounding, not the method (the conditioning of the 100-step
    noise case)."""
    nc, seed = 128, 5
    boxes = synth.amr_boxes(seed, nc, lo=16, hi=40)
    H = 1.0 / nc
    coarse, _ = synth.bssn_noise(nc, nc, nc, 3, None, amp=1e-3, r=synth.rng(seed + 2))
    r = synth.rng(seed + 1)
    fines = []
    for lo, hi in boxes:
        nf = [2 * (hi[d] - lo[d]) for d in range(3)]
        fb, _ = synth.bssn_noise(nf[0], nf[1], nf[2], 12, None, amp=1e-3, r=r)
        fines.append(fb)
    got = {}
    for mode in (0, 1):
        a = api.AmrBoxes(api.BSSN, (nc, nc, nc), boxes, H)
        a.state(0).copy_(to_gpu(coarse))
        for b, f in enumerate(fines):
            a.state(1 + b).copy_(to_gpu(f))
        a.autotune()
        a.state(0).copy_(to_gpu(coarse))
        a.step(0.25 * H, 1, mode=mode)
        got[mode] = [to_np(a.state(0))] + [to_np(a.state(1 + b)) for b in range(len(boxes))]
        del a
    cfg = orc.amrn((nc, nc, nc), boxes, H, 3, 12)
    orc.amrn_step(cfg, orc.BSSN, coarse, fines, 0.25 * H, 1)
    assert scaled_err(got[0][0], coarse, 3) <= RK4_TOL
    assert np.array_equal(got[0][0], got[1][0])
    for b, f in enumerate(fines):
        assert scaled_err(got[0][1 + b], f, 12) <= RK4_TOL, b
        assert np.array_equal(synth.interior(got[0][1 + b], 12), synth.interior(got[1][1 + b], 12)), b
