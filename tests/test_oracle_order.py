"""Pins of the oracle's arbitrary-order finite differencing (Sec. 3.2.2) and
of the first-order form of Eq. 1 (u, rho, v_i):
  - order 2 reproduces the paper's printed stencils ([+1,-2,+1]/h^2 and the
    central difference (f[i+1] - f[i-1])/(2 dx) of the Sec. 3 listing);
  - order 4 reproduces the 4th-order operators used everywhere else;
  - order-p D1 is exact on polynomials of degree <= p, D2 of degree <= p+1;
  - the RHS converges to the continuum RHS at order p;
  - the semi-discrete first-order system conserves 1/2 sum(rho^2 + |v|^2)
    (skew-symmetric D1), so RK4 multiplies the energy of a discrete mode by
    exactly |P(i w dt)|^2 per step; the order-p two-variable wave follows
    the closed form P(dt M)^n of its discrete Fourier mode.
"""

import numpy as np
import pytest

from paper_1410_1764_gb300 import synth


def _inner(a, g):
    return a[..., g:-g, g:-g, g:-g]


def test_order2_is_the_papers_stencils(orc):
    rng = np.random.default_rng(0)
    g, h = 1, 0.1
    f = rng.standard_normal((8, 9, 10))
    for ax in range(3):
        sl = lambda k: np.roll(f, -k, axis=2 - ax)
        np.testing.assert_allclose(_inner(orc.deriv_order(f, g, h, 2, 1, ax), g),
                                   _inner((sl(1) - 2 * f + sl(-1)) / h ** 2, g), rtol=1e-13, atol=1e-11)
        np.testing.assert_allclose(_inner(orc.deriv_order(f, g, h, 2, 0, ax), g),
                                   _inner((sl(1) - sl(-1)) / (2 * h), g), rtol=1e-13, atol=1e-12)


def test_order4_matches_fourth_order_operators(orc):
    rng = np.random.default_rng(1)
    g, h = 3, 0.07
    f = rng.standard_normal((12, 11, 13))
    for ax in range(3):
        np.testing.assert_allclose(orc.deriv_order(f, g, h, 4, 0, ax), orc.deriv(f, g, h, 0, ax),
                                   rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(orc.deriv_order(f, g, h, 4, 1, ax), orc.deriv(f, g, h, 1, ax),
                                   rtol=1e-13, atol=1e-10)


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_polynomial_exactness(orc, order):
    rng = np.random.default_rng(order)
    g, h, n = order // 2, 0.1, 6
    c = (np.arange(n + 2 * g) - g) * h + 0.05
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    for deg, kind in ((order, 0), (order + 1, 1)):
        for ax, Q in enumerate((X, Y, Z)):
            coef = rng.uniform(-1, 1, deg + 1)
            f = sum(cf * Q ** p for p, cf in enumerate(coef)) + 0.3 * (X + Y + Z) ** 0
            if kind == 0:
                want = sum(p * cf * Q ** (p - 1) for p, cf in enumerate(coef) if p >= 1)
            else:
                want = sum(p * (p - 1) * cf * Q ** (p - 2) for p, cf in enumerate(coef) if p >= 2)
            got = orc.deriv_order(np.ascontiguousarray(f), g, h, order, kind, ax)
            np.testing.assert_allclose(_inner(got, g), _inner(want * np.ones_like(f), g),
                                       rtol=0, atol=2e-9)


def _wave1_plane(n, g, t=0.0):
    X, Y, Z, h = synth.coords(n, n, n)
    k = 2 * np.pi
    w = k * np.sqrt(3)
    ph = k * (X + Y + Z) - w * t
    u = np.sin(ph)
    rho = -w * np.cos(ph)
    v = k * np.cos(ph)
    st = synth.pad(np.stack([u, rho, v, v, v]), g)
    return st, h, ph, k, w


@pytest.mark.parametrize("order", [2, 4, 6])
def test_wave1_rhs_converges_at_order_p(orc, order):
    errs = []
    g = order // 2
    for n in (16, 32, 64):
        st, h, ph, k, w = _wave1_plane(n, g)
        orc.fill_ghosts(st, g)
        r = _inner(orc.wave1_rhs(st, g, h, order), g)
        # continuum: u_t = rho, rho_t = div v = -3 k^2 sin, v_t = grad rho = k w sin
        want = np.stack([-w * np.cos(ph), -3 * k * k * np.sin(ph)] + [k * w * np.sin(ph)] * 3)
        errs.append(np.abs(r - want).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    lo = 2 ** order * 0.8
    assert lo < r1 < 2 ** order * 1.3 and lo < r2 < 2 ** order * 1.3, errs


@pytest.mark.parametrize("order", [2, 4, 8])
def test_wave1_energy_mode_factor(orc, order):
    n = 16
    g = order // 2
    X, Y, Z, h = synth.coords(n, n, n)
    th = 2 * np.pi * h
    ph = 2 * np.pi * (X + Y + Z)
    st = synth.pad(np.stack([np.zeros_like(X), np.cos(ph), 0 * X, 0 * X, 0 * X]), g)
    a, _ = orc.fd_weights(order)
    s = (2.0 / h) * sum(ak * np.sin((k + 1) * th) for k, ak in enumerate(a))
    z = np.sqrt(3 * s * s) * 0.25 * h
    factor = 1 - z ** 6 / 72 + z ** 8 / 576
    E = lambda y: 0.5 * np.sum(_inner(y[1:], g) ** 2)
    prm = orc.default_params(order)
    y = orc.rk4(orc.WAVE1, st, g, h, 0.25 * h, 6, params=prm)
    np.testing.assert_allclose(E(y) / E(st), factor ** 6, rtol=1e-12)


@pytest.mark.parametrize("order", [2, 6, 8])
def test_wave_order_p_closed_form(orc, order):
    n, g, steps = 16, order // 2, 20
    y0, h = synth.plane_wave(n, g)
    dt = 0.25 * h
    y = orc.rk4(orc.WAVE, y0, g, h, dt, steps, params=orc.default_params(order))
    _, b = orc.fd_weights(order)
    th = 2 * np.pi * h
    lam = 3 * sum(bk * (2 - 2 * np.cos((k + 1) * th)) for k, bk in enumerate(b)) / h ** 2
    M = np.array([[0.0, 1.0], [-lam, 0.0]]) * dt
    P = np.eye(2) + M + M @ M / 2 + M @ M @ M / 6 + M @ M @ M @ M / 24
    A = np.linalg.matrix_power(P, steps)
    w = 2 * np.pi * np.sqrt(3)
    sc, cc = A @ np.array([1.0, 0.0]), A @ np.array([0.0, -w])
    X, Y, Z, _ = synth.coords(n, n, n)
    ph = 2 * np.pi * (X + Y + Z)
    for v in range(2):
        np.testing.assert_allclose(_inner(y, g)[v], sc[v] * np.sin(ph) + cc[v] * np.cos(ph),
                                   rtol=0, atol=1e-11 * max(1, w))
