"""Pins of the oracle's variable-speed wave right-hand side against the PDE.

The continuum system is u_t = rho, rho_t = div(s grad u) with s = c^2 a
grid function (the variable-speed wave equation u_tt = div(c^2 grad u)).
The oracle evaluates it in the expanded, non-conservative form
s Lap_h u + sum_d D_d s D_d u with the 4th-order centred operators.  These
tests never use that form: the expected value is the divergence of the flux
s du/dx_d, formed by multiplying the polynomials (or by symbolic
differentiation of the product), so a sign, a factor or a swapped operand
in either term of the oracle fails them.

- exactness: for polynomial u and s of total degree <= 4 the 4th-order D1
  is exact and D2 is exact, so rho_t must equal div(s grad u) to round-off
  at every interior point of a non-periodic array whose ghosts hold the
  polynomial's own values;
- convergence: for smooth periodic u and s the error against the exact
  div(s grad u) falls by 16 per halving of h (4th order).
"""
import itertools

import numpy as np
import pytest

G = 2


def _random_poly(rng, degree):
    return {e: rng.uniform(-1, 1) for e in itertools.product(range(degree + 1), repeat=3)
            if sum(e) <= degree}


def _mul(p, q):
    out = {}
    for ea, va in p.items():
        for eb, vb in q.items():
            e = (ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2])
            out[e] = out.get(e, 0.0) + va * vb
    return out


def _dx(p, axis):
    out = {}
    for e, v in p.items():
        if e[axis] == 0:
            continue
        f = list(e)
        f[axis] -= 1
        out[tuple(f)] = out.get(tuple(f), 0.0) + v * e[axis]
    return out


def _eval(p, XYZ):
    X, Y, Z = XYZ
    f = np.zeros_like(X)
    for (a, b, c), v in p.items():
        f += v * X ** a * Y ** b * Z ** c
    return f


def _coords(n, h, x0):
    idx = (np.arange(n + 2 * G) - G) * h
    Z, Y, X = np.meshgrid(idx + x0[2], idx + x0[1], idx + x0[0], indexing="ij")
    return X, Y, Z


def _inner(a):
    return a[..., G:-G, G:-G, G:-G]


@pytest.mark.parametrize("seed,h", [(0, 0.1), (1, 0.05), (2, 0.2)])
def test_varc_rhs_exact_on_polynomials(orc, seed, h):
    rng = np.random.default_rng(100 + seed)
    pu, ps, pr = _random_poly(rng, 4), _random_poly(rng, 4), _random_poly(rng, 3)
    ps[(0, 0, 0)] += 2.0  # s = c^2 > 0 on the box, as a squared speed is
    XYZ = _coords(9, h, (0.15, -0.3, 0.2))
    st = np.stack([_eval(pu, XYZ), _eval(pr, XYZ)])
    s = _eval(ps, XYZ)
    got = orc.varc_rhs(np.ascontiguousarray(st), np.ascontiguousarray(s), G, h)
    # div(s grad u) as the divergence of the flux polynomial s * du/dx_d.
    div = {}
    for d in range(3):
        for e, v in _dx(_mul(ps, _dx(pu, d)), d).items():
            div[e] = div.get(e, 0.0) + v
    want = _eval(div, XYZ)
    scale = np.abs(_inner(want)).max()
    assert scale > 1.0
    assert np.abs(_inner(got[1]) - _inner(want)).max() <= 1e-11 * scale
    np.testing.assert_array_equal(_inner(got[0]), _inner(st[1]))


def _periodic_case(n):
    """Smooth periodic u, s on [0,1)^3 and the exact div(s grad u), from
    sympy (symbolic derivatives of the flux, not of the expanded form)."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    tp = 2 * sp.pi
    u = sp.sin(tp * (x + 2 * y)) * sp.cos(tp * z) + sp.Rational(1, 2) * sp.cos(tp * (x - z))
    s = 1 + sp.Rational(3, 10) * sp.sin(tp * x) * sp.cos(tp * y) + sp.Rational(1, 5) * sp.sin(tp * (y + z))
    div = sum(sp.diff(s * sp.diff(u, v), v) for v in (x, y, z))
    fu, fs, fd = (sp.lambdify((x, y, z), e, "numpy") for e in (u, s, div))
    h = 1.0 / n
    X, Y, Z = _coords(n, h, (0.0, 0.0, 0.0))  # ghosts hold the periodic values
    uu = np.broadcast_to(fu(X, Y, Z), X.shape).astype(np.float64)
    ss = np.broadcast_to(fs(X, Y, Z), X.shape).astype(np.float64)
    dd = np.broadcast_to(fd(X, Y, Z), X.shape).astype(np.float64)
    st = np.ascontiguousarray(np.stack([uu, np.zeros_like(uu)]))
    return st, np.ascontiguousarray(ss), dd, h


def test_varc_rhs_converges_4th_order(orc):
    errs = []
    for n in (16, 32, 64):
        st, s, want, h = _periodic_case(n)
        got = orc.varc_rhs(st, s, G, h)
        errs.append(np.abs(_inner(got[1]) - _inner(want)).max() / np.abs(_inner(want)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert errs[2] < 1e-4
    assert 14.0 < r1 < 18.0 and 15.0 < r2 < 17.0, (errs, r1, r2)


def test_varc_rhs_periodic_ghost_fill_is_the_exact_extension(orc):
    """The periodic ghost fill gives the same right-hand side as ghosts that
    hold the analytic periodic values (the case above sets them directly)."""
    st, s, _, h = _periodic_case(16)
    st2, s2 = st.copy(), s.copy()
    orc.fill_ghosts(st2, G)
    orc.fill_ghosts(s2, G)
    a = orc.varc_rhs(st, s, G, h)
    b = orc.varc_rhs(st2, s2, G, h)
    assert np.abs(_inner(a) - _inner(b)).max() <= 1e-10 * np.abs(_inner(a)).max()
