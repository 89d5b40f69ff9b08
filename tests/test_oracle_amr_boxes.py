"""Pins of the oracle's two-level refinement with several boxes and of its
BSSN form (Sec. 4: the Carpet driver's AMR with subcycling in time):
  - prolongation into every box's buffer is exact on tensor-product quintics
    for every variable;
  - restriction is injection at coincident points of every box;
  - the single-box scalar-wave interface is the general routine with one box;
  - exact flat space stays exactly flat on both levels (prolongation weights
    sum to one in binary, the flat right-hand side is zero);
  - the BSSN gauge wave (an exact solution with harmonic slicing and zero
    shift) evolved on two levels with two refined boxes converges to the
    exact solution at 4th order on the coarse level and inside both boxes,
    through the buffer-zone interface (buffer 12 = stencil radius 3 x 4
    stages); a configuration whose prolongation would read outside the
    padded coarse grid, or overlapping boxes, is refused.
"""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth

from test_oracle_bssn import gauge_wave_state


def _axis_coords(n, g, h, off=0):
    return (off + np.arange(n + 2 * g) - g) * h


def _coarse_xyz(nc, gc, H):
    return np.meshgrid(_axis_coords(nc[2], gc, H), _axis_coords(nc[1], gc, H), _axis_coords(nc[0], gc, H),
                       indexing="ij")  # Z, Y, X


def _fine_xyz(lo, hi, gf, H):
    ax = [_axis_coords(2 * (hi[d] - lo[d]), gf, H / 2, 2 * lo[d]) for d in range(3)]
    return np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")


def _quintic(X, Y, Z, v):
    return (0.3 * v + X - 2 * X ** 5 + 0.5 * Y ** 2 * X + (1 + 0.1 * v) * Y ** 5 - Z ** 3 * X ** 2 * Y
            + 0.7 * Z ** 5 * (1 - 0.05 * v))


BOXES = [((5, 6, 5), (9, 10, 8)), ((11, 5, 6), (14, 9, 9)), ((6, 11, 9), (8, 13, 12))]
NC = (20, 19, 18)


def test_prolongation_exact_every_box_and_variable(orc):
    H, gc, gf, nv = 0.07, 3, 12, 24
    cfg = orc.amrn(NC, BOXES, H, gc, gf)
    Zc, Yc, Xc = _coarse_xyz(NC, gc, H)
    coarse = np.ascontiguousarray(np.stack([_quintic(Xc, Yc, Zc, v) for v in range(nv)]))
    for b, (lo, hi) in enumerate(BOXES):
        Zf, Yf, Xf = _fine_xyz(lo, hi, gf, H)
        fine = np.zeros((nv,) + Xf.shape)
        orc.amrn_prolong(cfg, b, [coarse], [1.0], fine)
        mask = np.ones(Xf.shape, bool)
        mask[gf:-gf, gf:-gf, gf:-gf] = False
        for v in (0, 7, 23):
            want = _quintic(Xf, Yf, Zf, v)
            np.testing.assert_allclose(fine[v][mask], want[mask], rtol=0, atol=1e-11)
        assert np.all(fine[:, ~mask] == 0)  # the interior is left alone


def test_restriction_is_injection_every_box(orc):
    H, gc, gf, nv = 0.07, 3, 12, 24
    cfg = orc.amrn(NC, BOXES, H, gc, gf)
    rng = np.random.default_rng(1)
    coarse = synth.pad(rng.standard_normal((nv, NC[2], NC[1], NC[0])), gc)
    before = coarse.copy()
    covered = np.zeros(coarse.shape[1:], bool)
    for b, (lo, hi) in enumerate(BOXES):
        nf = [2 * (hi[d] - lo[d]) for d in range(3)]
        fine = rng.standard_normal((nv, nf[2] + 2 * gf, nf[1] + 2 * gf, nf[0] + 2 * gf))
        orc.amrn_restrict(cfg, b, fine, coarse)
        sl = tuple(slice(lo[d] + gc, hi[d] + gc) for d in (2, 1, 0))
        np.testing.assert_array_equal(coarse[(slice(None),) + sl], fine[:, gf:-gf:2, gf:-gf:2, gf:-gf:2])
        covered[sl] = True
    np.testing.assert_array_equal(coarse[:, ~covered], before[:, ~covered])


def test_single_box_interface_is_the_general_routine(orc):
    nc, H = 22, 1.0 / 22
    lo, hi = (5, 6, 4), (12, 14, 11)
    rng = np.random.default_rng(2)
    coarse = synth.pad(rng.standard_normal((2, nc, nc, nc)), 2)
    nf = [2 * (hi[d] - lo[d]) for d in range(3)]
    fine = synth.pad(rng.standard_normal((2, nf[2], nf[1], nf[0])), 8)
    c1, f1, c2, f2 = coarse.copy(), fine.copy(), coarse.copy(), fine.copy()
    orc.amr_step(orc.amr(nc, lo, hi, H), c1, f1, 0.25 * H, 2)
    orc.amrn_step(orc.amrn((nc, nc, nc), [(lo, hi)], H, 2, 8), orc.WAVE, c2, [f2], 0.25 * H, 2,
                  params=orc.Params(0.0, 0.0, 0, 0, 0))
    assert np.array_equal(c1, c2) and np.array_equal(f1, f2)


def test_flat_space_stays_exactly_flat(orc):
    H, gc, gf = 1.0 / 20, 3, 12
    cfg = orc.amrn(NC, BOXES[:2], H, gc, gf)
    flat = synth.BSSN_FLAT[:, None, None, None]
    coarse = np.ascontiguousarray(np.broadcast_to(flat, (24, NC[2] + 6, NC[1] + 6, NC[0] + 6)).copy())
    fines = []
    for lo, hi in BOXES[:2]:
        nf = [2 * (hi[d] - lo[d]) + 2 * gf for d in range(3)]
        fines.append(np.ascontiguousarray(np.broadcast_to(flat, (24, nf[2], nf[1], nf[0])).copy()))
    orc.amrn_step(cfg, orc.BSSN, coarse, fines, 0.25 * H, 2)
    assert np.array_equal(coarse, np.broadcast_to(flat, coarse.shape))
    for f in fines:
        assert np.array_equal(f[:, gf:-gf, gf:-gf, gf:-gf], np.broadcast_to(flat, f[:, gf:-gf, gf:-gf, gf:-gf].shape))


def _gauge_wave_amr(orc, nx, T, m=14):
    """Coarse nx x m x m (h = 1/nx), two boxes: x in [nx/4, nx/2) and
    [3nx/5, 7nx/10), y and z in [5, 8); gauge wave sampled on both levels;
    returns max errors (coarse interior, box interiors) at time T."""
    prm = orc.Params(0.1, 2.0, 1, 1, 0)  # harmonic slicing, frozen (zero) shift
    H, gc, gf = 1.0 / nx, 3, 12
    s = nx // 20
    boxes = [((5 * s, 5, 5), (10 * s, 8, 8)), ((12 * s, 5, 5), (14 * s, 8, 8))]
    cfg = orc.amrn((nx, m, m), boxes, H, gc, gf)

    def exact_coarse(t):
        st, _ = gauge_wave_state(nx, m, m, t)
        return st

    def exact_fine(lo, hi, t):
        # box (lo, hi)'s padded fine points are points of a grid of spacing
        # H/2 starting at fine index 2 lo - gf along each axis
        big, _ = gauge_wave_state(2 * nx, 2 * m + 2 * gf, 2 * m + 2 * gf, t)
        g0 = 3  # ghosts of gauge_wave_state
        sl = [slice(g0 + 2 * lo[d] - gf + (gf if d else 0), g0 + 2 * hi[d] + gf + (gf if d else 0))
              for d in range(3)]
        return np.ascontiguousarray(big[:, sl[2], sl[1], sl[0]])

    coarse = np.ascontiguousarray(exact_coarse(0.0))
    fines = [exact_fine(lo, hi, 0.0) for lo, hi in boxes]
    dt = 0.25 * H
    nsteps = int(round(T / dt))
    orc.amrn_step(cfg, orc.BSSN, coarse, fines, dt, nsteps, params=prm)
    t = nsteps * dt
    ec = np.abs(synth.interior(coarse - exact_coarse(t), gc)).max()
    ef = max(np.abs(synth.interior(f - exact_fine(lo, hi, t), gf)).max() for f, (lo, hi) in zip(fines, boxes))
    return ec, ef


def test_invalid_boxes_are_refused(orc):
    """A box whose prolongation would read beyond the padded coarse grid, or
    two overlapping boxes, are refused (no out-of-range access)."""
    H, gc, gf = 1.0 / 20, 3, 12
    coarse = np.zeros((24, 20, 20, 26))
    for boxes in ([((4, 5, 5), (8, 8, 8))], [((5, 5, 5), (15, 8, 8))],
                  [((5, 5, 5), (9, 8, 8)), ((8, 6, 6), (10, 8, 8))]):
        cfg = orc.amrn((20, 14, 14), boxes, H, gc, gf)
        with pytest.raises(RuntimeError):
            orc.amrn_step(cfg, orc.BSSN, coarse, [np.zeros((24, 30, 30, 30))] * len(boxes), 0.01, 1)


@pytest.mark.slow
def test_bssn_gauge_wave_converges_through_the_interface(orc):
    res = [_gauge_wave_amr(orc, nx, 0.125) for nx in (20, 40, 80)]
    ec = [r[0] for r in res]
    ef = [r[1] for r in res]
    for e in (ec, ef):
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert 12.0 < r1 < 18.0 and 14.0 < r2 < 18.0, (ec, ef)
