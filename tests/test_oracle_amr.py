"""Pins of the oracle's two-level mesh refinement with Berger-Oliger
subcycling (Sec. 4: AMR with subcycling in time):
  - prolongation is exact on tensor-product quintics (quintic Lagrange) and,
    with cubic Hermite weights, on cubics in time;
  - restriction is injection at coincident points;
  - a spatially constant state stays constant;
  - a plane wave evolved on two levels converges to the continuum solution
    at 4th order through the interface (buffer zones filled at fine step
    starts, quintic prolongation, cubic Hermite time interpolation), and the
    fine level is about as accurate as a coarse-only evolution.
"""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth


def _coarse_coords(nc, gc, H):
    c = (np.arange(nc + 2 * gc) - gc) * H
    return np.meshgrid(c, c, c, indexing="ij")  # Z, Y, X


def _fine_coords(cfg):
    H, gf = cfg.H, cfg.gf
    axes = []
    for d in range(3):
        nf = 2 * (cfg.hi[d] - cfg.lo[d])
        axes.append((2 * cfg.lo[d] + np.arange(nf + 2 * gf) - gf) * (H / 2))
    return np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")


def _poly(X, Y, Z, t=0.0):
    return (0.3 + X - 2 * X ** 5 + 0.5 * Y ** 2 * X + Y ** 5 - Z ** 3 * X ** 4 * Y ** 5 + 0.7 * Z
            + t * (1 + X * Y) + t * t * (0.5 - Z ** 2))


def _dpoly_dt(X, Y, Z, t):
    return (1 + X * Y) + 2 * t * (0.5 - Z ** 2) + 3 * t * t * X


def test_prolongation_exact_on_quintics_in_space_and_cubics_in_time(orc):
    nc, H = 20, 0.1
    cfg = orc.amr(nc, (5, 6, 4), (9, 13, 11), H)
    Zc, Yc, Xc = _coarse_coords(nc, 2, H)
    Zf, Yf, Xf = _fine_coords(cfg)
    dt = 0.05
    P = lambda X, Y, Z, t: _poly(X, Y, Z, t) + t ** 3 * X
    st = lambda t: np.ascontiguousarray(np.stack([P(Xc, Yc, Zc, t), 2 * P(Xc, Yc, Zc, t)]))
    dst = lambda t: np.ascontiguousarray(np.stack([_dpoly_dt(Xc, Yc, Zc, t), 2 * _dpoly_dt(Xc, Yc, Zc, t)]))
    levels = [st(0.0), dst(0.0), st(dt), dst(dt)]
    for th in (0.0, 0.25, 0.5, 1.0):
        tw = [2 * th ** 3 - 3 * th ** 2 + 1, dt * (th ** 3 - 2 * th ** 2 + th), -2 * th ** 3 + 3 * th ** 2,
              dt * (th ** 3 - th ** 2)]
        fine = np.zeros((2,) + Xf.shape)
        orc.amr_prolong(cfg, levels, tw, fine)
        want = P(Xf, Yf, Zf, th * dt)
        g = cfg.gf
        mask = np.ones(Xf.shape, bool)
        mask[g:-g, g:-g, g:-g] = False
        np.testing.assert_allclose(fine[0][mask], want[mask], rtol=0, atol=1e-11)
        np.testing.assert_allclose(fine[1][mask], 2 * want[mask], rtol=0, atol=2e-11)
        assert np.all(fine[:, g:-g, g:-g, g:-g] == 0)  # interior untouched


def test_restriction_is_injection(orc):
    nc, H = 16, 0.1
    cfg = orc.amr(nc, (4, 5, 6), (8, 12, 11), H)
    rng = np.random.default_rng(0)
    Zf, Yf, Xf = _fine_coords(cfg)
    fine = rng.standard_normal((2,) + Xf.shape)
    coarse = np.zeros((2, nc + 4, nc + 4, nc + 4))
    orc.amr_restrict(cfg, fine, coarse)
    g, gf = 2, cfg.gf
    for K in range(nc):
        for J in range(nc):
            for I in range(nc):
                inside = all(cfg.lo[d] <= q < cfg.hi[d] for d, q in enumerate((I, J, K)))
                got = coarse[:, K + g, J + g, I + g]
                if inside:
                    want = fine[:, 2 * (K - cfg.lo[2]) + gf, 2 * (J - cfg.lo[1]) + gf, 2 * (I - cfg.lo[0]) + gf]
                    assert np.array_equal(got, want)
                else:
                    assert np.all(got == 0)


def _plane(X, Y, Z, t):
    k = 2 * np.pi
    w = k * np.sqrt(3)
    ph = k * (X + Y + Z) - w * t
    return np.stack([np.sin(ph), -w * np.cos(ph)])


def _run(orc, nc, steps, amr=True):
    H = 1.0 / nc
    q = nc // 4
    cfg = orc.amr(nc, (q, q, q), (3 * q - 1, 3 * q - 1, 3 * q - 1), H)
    Zc, Yc, Xc = _coarse_coords(nc, 2, H)
    Zf, Yf, Xf = _fine_coords(cfg)
    coarse = np.ascontiguousarray(_plane(Xc, Yc, Zc, 0.0))
    fine = np.ascontiguousarray(_plane(Xf, Yf, Zf, 0.0))
    dt = 0.25 * H
    if amr:
        orc.amr_step(cfg, coarse, fine, dt, steps)
    else:
        coarse = orc.rk4(orc.WAVE, coarse, 2, H, dt, steps)
    T = steps * dt
    ec = np.abs(synth.interior(coarse, 2) - synth.interior(_plane(Xc, Yc, Zc, T), 2)).max()
    ef = np.abs(synth.interior(fine, cfg.gf) - synth.interior(_plane(Xf, Yf, Zf, T), cfg.gf)).max() if amr else None
    return ec, ef


def test_constant_state_preserved(orc):
    nc, H = 16, 1.0 / 16
    cfg = orc.amr(nc, (4, 4, 4), (11, 11, 11), H)
    coarse = np.zeros((2, 20, 20, 20))
    coarse[0] = 0.75
    fine = np.zeros((2, 30, 30, 30))
    fine[0] = 0.75
    orc.amr_step(cfg, coarse, fine, 0.25 * H, 4)
    g = cfg.gf
    assert np.abs(coarse[0] - 0.75).max() < 1e-14 and np.abs(coarse[1]).max() < 1e-12
    assert np.abs(fine[0, g:-g, g:-g, g:-g] - 0.75).max() < 1e-14
    assert np.abs(fine[1, g:-g, g:-g, g:-g]).max() < 1e-12


def test_plane_wave_converges_through_the_interface(orc):
    T_steps = {16: 8, 32: 16}
    errs = {n: _run(orc, n, s) for n, s in T_steps.items()}
    coarse_only = {n: _run(orc, n, s, amr=False)[0] for n, s in T_steps.items()}
    (c16, f16), (c32, f32) = errs[16], errs[32]
    assert c16 / c32 > 10.0 and f16 / f32 > 10.0, errs
    for n in T_steps:
        assert errs[n][1] <= 1.15 * coarse_only[n], (errs, coarse_only)
