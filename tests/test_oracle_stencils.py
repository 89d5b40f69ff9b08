"""Pins of the oracle's finite-difference operators (Sec. 3.2.2).

Independent of the oracle's own arithmetic: exactness on polynomials,
Fourier symbols in closed form, and the 4th-order operators rebuilt by
Richardson combination from the paper's own 2nd-order examples (the
[+1,-2,+1]/h^2 stencil of Sec. 3.2.2 and the (f[i+1]-f[i-1])/(2dx) loop of
Sec. 3).
"""
import itertools

import numpy as np
import pytest

G = 3


def _poly_field(coef, n, h, x0):
    """Padded array of a polynomial sum c_abc x^a y^b z^c, and the callable."""
    p = n + 2 * G
    idx = (np.arange(p) - G) * h
    Z, Y, X = np.meshgrid(idx + x0[2], idx + x0[1], idx + x0[0], indexing="ij")
    f = np.zeros_like(X)
    for (a, b, c), v in coef.items():
        f += v * X ** a * Y ** b * Z ** c
    return f, (X, Y, Z)


def _poly_deriv(coef, da):
    """Coefficients of the derivative of the polynomial along multi-index da."""
    out = {}
    for (a, b, c), v in coef.items():
        e = [a, b, c]
        fac = v
        for ax, m in enumerate(da):
            for _ in range(m):
                fac *= e[ax]
                e[ax] -= 1
        if fac != 0 and min(e) >= 0:
            out[tuple(e)] = out.get(tuple(e), 0.0) + fac
    return out


def _random_poly(rng, degree):
    coef = {}
    for a, b, c in itertools.product(range(degree + 1), repeat=3):
        if a + b + c <= degree:
            coef[(a, b, c)] = rng.uniform(-1, 1)
    return coef


def _eval(coef, XYZ):
    X, Y, Z = XYZ
    f = np.zeros_like(X)
    for (a, b, c), v in coef.items():
        f += v * X ** a * Y ** b * Z ** c
    return f


def _inner(a):
    return a[G:-G, G:-G, G:-G]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_d1_exact_degree4(orc, axis):
    rng = np.random.default_rng(1)
    coef = _random_poly(rng, 4)
    h = 0.1
    f, XYZ = _poly_field(coef, 8, h, (0.3, -0.2, 0.1))
    got = orc.deriv(f, G, h, 0, axis)
    da = [0, 0, 0]
    da[axis] = 1
    want = _eval(_poly_deriv(coef, da), XYZ)
    np.testing.assert_allclose(_inner(got), _inner(want), rtol=0, atol=1e-12)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_d2_exact_degree5(orc, axis):
    rng = np.random.default_rng(2)
    coef = _random_poly(rng, 5)
    h = 0.1
    f, XYZ = _poly_field(coef, 8, h, (0.1, 0.2, -0.3))
    got = orc.deriv(f, G, h, 1, axis)
    da = [0, 0, 0]
    da[axis] = 2
    want = _eval(_poly_deriv(coef, da), XYZ)
    np.testing.assert_allclose(_inner(got), _inner(want), rtol=0, atol=1e-10)


@pytest.mark.parametrize("a,b", [(0, 1), (0, 2), (1, 2), (1, 0)])
def test_mixed_exact_degree4(orc, a, b):
    rng = np.random.default_rng(3)
    coef = _random_poly(rng, 4)
    h = 0.1
    f, XYZ = _poly_field(coef, 8, h, (-0.2, 0.1, 0.25))
    got = orc.deriv(f, G, h, 2, a, b)
    da = [0, 0, 0]
    da[a] += 1
    da[b] += 1
    want = _eval(_poly_deriv(coef, da), XYZ)
    np.testing.assert_allclose(_inner(got), _inner(want), rtol=0, atol=1e-10)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ko_annihilates_degree5(orc, axis):
    rng = np.random.default_rng(4)
    coef = _random_poly(rng, 5)
    h = 0.1
    f, _ = _poly_field(coef, 8, h, (0.05, 0.1, 0.15))
    got = orc.deriv(f, G, h, 3, axis)
    assert np.abs(_inner(got)).max() < 1e-11


def _mode(n, theta_axis, theta, kind="cos"):
    p = n + 2 * G
    i = np.arange(p) - G
    arr = np.cos(theta * i) if kind == "cos" else np.sin(theta * i)
    shape = [1, 1, 1]
    shape[2 - theta_axis] = p
    return np.broadcast_to(arr.reshape(shape), (p, p, p)).copy()


@pytest.mark.parametrize("theta", [np.pi / 8, np.pi / 3, 0.9 * np.pi, np.pi])
def test_fourier_symbols(orc, theta):
    """D2 symbol (-2cos2t + 32cos t - 30)/(12h^2), D1 symbol
    (8 sin t - sin 2t)/(6h), KO symbol -(eps/h) sin^6(t/2) (eps = 1)."""
    h = 0.05
    n = 8
    for ax in range(3):
        c = _mode(n, ax, theta, "cos")
        s = _mode(n, ax, theta, "sin")
        d2 = orc.deriv(c, G, h, 1, ax)
        sym2 = (-2 * np.cos(2 * theta) + 32 * np.cos(theta) - 30) / (12 * h * h)
        np.testing.assert_allclose(_inner(d2), sym2 * _inner(c), rtol=0, atol=1e-9)
        d1 = orc.deriv(s, G, h, 0, ax)
        sym1 = (8 * np.sin(theta) - np.sin(2 * theta)) / (6 * h)
        np.testing.assert_allclose(_inner(d1), sym1 * _inner(c), rtol=0, atol=1e-11)
        ko = orc.deriv(c, G, h, 3, ax)
        symk = -(1.0 / h) * np.sin(theta / 2) ** 6
        np.testing.assert_allclose(_inner(ko), symk * _inner(c), rtol=0, atol=1e-11)


def test_nyquist_damping(orc):
    """u_j = (-1)^j: the KO term along one direction is -eps/h u."""
    h = 1.0 / 16
    f = _mode(8, 0, np.pi, "cos")
    ko = orc.deriv(f, G, h, 3, 0)
    np.testing.assert_allclose(_inner(ko), -(1.0 / h) * _inner(f), rtol=1e-14)


def test_richardson_from_paper_second_order_stencils(orc):
    """4th-order D2 = 4/3 [1,-2,1]/h^2 - 1/3 [1,-2,1]/(2h)^2 and
    4th-order D1 = 4/3 central(h) - 1/3 central(2h), built from the paper's
    printed 2nd-order examples on random data."""
    rng = np.random.default_rng(5)
    n, h = 8, 0.07
    f = rng.standard_normal((n + 2 * G,) * 3)
    for ax in range(3):
        sl = lambda k: np.roll(f, -k, axis=2 - ax)
        lap_h = (sl(1) - 2 * f + sl(-1)) / h ** 2
        lap_2h = (sl(2) - 2 * f + sl(-2)) / (2 * h) ** 2
        cen_h = (sl(1) - sl(-1)) / (2 * h)
        cen_2h = (sl(2) - sl(-2)) / (4 * h)
        d2 = orc.deriv(f, G, h, 1, ax)
        d1 = orc.deriv(f, G, h, 0, ax)
        np.testing.assert_allclose(_inner(d2), _inner(4 / 3 * lap_h - 1 / 3 * lap_2h),
                                   rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(_inner(d1), _inner(4 / 3 * cen_h - 1 / 3 * cen_2h),
                                   rtol=1e-12, atol=1e-11)


def test_mixed_is_product_of_1d(orc):
    """Mixed D_x D_y equals D1_y applied to the D1_x field (tensor product)."""
    rng = np.random.default_rng(6)
    n, h = 10, 0.1
    f = rng.standard_normal((n + 2 * G,) * 3)
    # D1_x on every row including ghost rows in y, via shifts
    fx = (8 * (np.roll(f, -1, 2) - np.roll(f, 1, 2)) - (np.roll(f, -2, 2) - np.roll(f, 2, 2))) / (12 * h)
    fxy = (8 * (np.roll(fx, -1, 1) - np.roll(fx, 1, 1)) - (np.roll(fx, -2, 1) - np.roll(fx, 2, 1))) / (12 * h)
    got = orc.deriv(f, G, h, 2, 0, 1)
    np.testing.assert_allclose(_inner(got), _inner(fxy), rtol=1e-12, atol=1e-10)


def test_ghost_fill_periodic(orc):
    rng = np.random.default_rng(7)
    nx, ny, nz, g = 5, 7, 4, 3
    inner = rng.standard_normal((2, nz, ny, nx))
    a = np.zeros((2, nz + 2 * g, ny + 2 * g, nx + 2 * g))
    a[:, g:g + nz, g:g + ny, g:g + nx] = inner
    orc.fill_ghosts(a, g)
    k = (np.arange(nz + 2 * g) - g) % nz
    j = (np.arange(ny + 2 * g) - g) % ny
    i = (np.arange(nx + 2 * g) - g) % nx
    want = inner[:, k][:, :, j][:, :, :, i]
    assert np.array_equal(a, want)
