"""Pins of the oracle's scalar-wave RHS and RK4 (Sec. 3 Eq. 1, Sec. 2).

- closed form of the fully discrete solution for a Fourier mode;
- 4th-order convergence to the continuum plane wave;
- discrete energy: exact per-mode RK4 factor, monotone decay for pulses;
- linearity and translation (roll) invariance.
"""
import numpy as np

from paper_1410_1764_gb300 import synth

G = 2


def _lambda(h, thetas):
    return sum((30 - 32 * np.cos(t) + 2 * np.cos(2 * t)) / (12 * h * h) for t in thetas)


def _rk4_matrix(dt, lam):
    M = np.array([[0.0, 1.0], [-lam, 0.0]])
    z = dt * M
    I = np.eye(2)
    return I + z + z @ z / 2 + z @ z @ z / 6 + z @ z @ z @ z / 24


def test_plane_wave_closed_form(orc):
    """u = a sin(k.x) + b cos(k.x) stays in span; the coefficient pairs evolve
    by P(dt M)^n, M = [[0,1],[-Lambda,0]], P the RK4 polynomial."""
    n, steps = 16, 40
    y0, h = synth.plane_wave(n, G)
    dt = 0.25 * h
    y = orc.rk4(orc.WAVE, y0, G, h, dt, steps)
    theta = 2 * np.pi * h
    lam = _lambda(h, [theta] * 3)
    A = np.linalg.matrix_power(_rk4_matrix(dt, lam), steps)
    # initial: sin coefficient (1, 0), cos coefficient (0, -w)
    w = 2 * np.pi * np.sqrt(3)
    s_coef = A @ np.array([1.0, 0.0])
    c_coef = A @ np.array([0.0, -w])
    X, Y, Z, _ = synth.coords(n, n, n)
    ph = 2 * np.pi * (X + Y + Z)
    for v in range(2):
        want = s_coef[v] * np.sin(ph) + c_coef[v] * np.cos(ph)
        got = synth.interior(y, G)[v]
        np.testing.assert_allclose(got, want, rtol=0, atol=2e-12 * max(1, w * v))


def test_convergence_order4(orc):
    """Error against the continuum solution sin(k.x - w t) at fixed T shrinks
    by ~16 per halving of h (dt = h/4)."""
    T = 0.125
    errs = []
    for n in (16, 32, 64):
        y0, h = synth.plane_wave(n, G)
        dt = 0.25 * h
        steps = int(round(T / dt))
        y = orc.rk4(orc.WAVE, y0, G, h, dt, steps)
        X, Y, Z, _ = synth.coords(n, n, n)
        w = 2 * np.pi * np.sqrt(3)
        exact = np.sin(2 * np.pi * (X + Y + Z) - w * T)
        errs.append(np.abs(synth.interior(y, G)[0] - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.0 and 14.0 < r2 < 18.0, errs


def _energy(orc, y, h):
    yy = y.copy()
    orc.fill_ghosts(yy, G)
    lap = orc.wave_rhs(np.stack([yy[0], yy[0]]), G, h)[1]
    u = synth.interior(yy, G)[0]
    rho = synth.interior(yy, G)[1]
    return 0.5 * np.sum(rho * rho - u * synth.interior(lap, G)) * h ** 3


def test_energy_mode_factor(orc):
    """Single Fourier mode: E_{n+1}/E_n = |P(i w dt)|^2
    = 1 - (w dt)^6/72 + (w dt)^8/576 with w^2 = Lambda."""
    n = 16
    y0, h = synth.plane_wave(n, G)
    dt = 0.25 * h
    lam = _lambda(h, [2 * np.pi * h] * 3)
    z = np.sqrt(lam) * dt
    factor = 1 - z ** 6 / 72 + z ** 8 / 576
    E0 = _energy(orc, y0, h)
    y = orc.rk4(orc.WAVE, y0, G, h, dt, 10)
    E1 = _energy(orc, y, h)
    np.testing.assert_allclose(E1 / E0, factor ** 10, rtol=1e-12)


def test_energy_pulses_nonincreasing(orc):
    n = 24
    y, h = synth.gaussian_pulses(n, G, seed=1, width=0.1)
    dt = 0.25 * h
    E = [_energy(orc, y, h)]
    for _ in range(8):
        y = orc.rk4(orc.WAVE, y, G, h, dt, 2)
        E.append(_energy(orc, y, h))
    E = np.array(E)
    assert E[0] > 0
    assert np.all(np.diff(E) <= 1e-14 * E[0]), E
    assert E[-1] < E[0]


def test_linearity_and_roll(orc):
    n = 12
    rng = np.random.default_rng(0)
    a = synth.pad(rng.standard_normal((2, n, n, n)), G)
    b = synth.pad(rng.standard_normal((2, n, n, n)), G)
    h = 1.0 / n
    dt = 0.25 * h
    ya = orc.rk4(orc.WAVE, a, G, h, dt, 3)
    yb = orc.rk4(orc.WAVE, b, G, h, dt, 3)
    yab = orc.rk4(orc.WAVE, a + 2 * b, G, h, dt, 3)
    np.testing.assert_allclose(yab, ya + 2 * yb, rtol=0, atol=1e-10)
    shift = (1, 3, 5)
    ar = synth.pad(np.roll(synth.interior(a, G), shift, axis=(1, 2, 3)), G)
    yr = orc.rk4(orc.WAVE, ar, G, h, dt, 3)
    assert np.array_equal(synth.interior(yr, G),
                          np.roll(synth.interior(ya, G), shift, axis=(1, 2, 3)))
