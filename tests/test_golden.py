"""Pins against the stencils the paper prints (tests/golden/printed_stencils.txt,
each line citing its passage): the oracle's and the generator's order-2
operators, and the oracle's first-order wave system of Eq. 1 on data that
varies along one axis, which is the 1-D loop the paper lists in Sec. 3."""
import os
from fractions import Fraction

import numpy as np

from paper_1410_1764_gb300.gen import stencil

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "printed_stencils.txt")


def _printed():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, w, div, cite = [x.strip() for x in line.split("|")]
        weights = [Fraction(x) for x in w.split()]
        scale, power = (Fraction(2), 1) if div == "2 dx" else (Fraction(1), 2)
        out[name] = ([x / scale for x in weights], power, cite)
    return out


def test_fixture_has_citations():
    p = _printed()
    assert set(p) == {"d1_centred_order2", "d2_centred_order2"}
    for w, power, cite in p.values():
        assert cite.startswith("Sec. ")


def test_oracle_order2_weights_are_the_printed_ones(orc):
    p = _printed()
    a, b = orc.fd_weights(2)
    w1 = p["d1_centred_order2"][0]                # [-1/2, 0, 1/2] per dx
    w2 = p["d2_centred_order2"][0]                # [1, -2, 1] per dx^2
    # D1 f = (1/h) a_1 (f_1 - f_-1); D2 f = (1/h^2) b_1 ((f_1 - f_0) + (f_-1 - f_0))
    assert a[0] == float(w1[2]) == -float(w1[0]) and w1[1] == 0
    assert b[0] == float(w2[0]) == float(w2[2]) and float(w2[1]) == -2 * b[0]


def test_generator_order2_weights_are_the_printed_ones():
    p = _printed()
    a, b = stencil.fd_weights(2)
    assert a == [p["d1_centred_order2"][0][2]]
    assert b == [p["d2_centred_order2"][0][0]]


def test_first_order_wave_is_the_printed_loop(orc):
    """Eq. 1 at order 2 on fields varying along x only: rho_t = D_x v_x and
    (v_x)_t = D_x rho with the printed centred difference, u_t = rho."""
    w1 = [float(x) for x in _printed()["d1_centred_order2"][0]]
    n, g = 16, 2
    h = 1.0 / n
    x = np.arange(n) * h
    rng = np.random.default_rng(0)
    rho1 = np.sin(2 * np.pi * x) + 0.1 * rng.standard_normal(n)
    v1 = np.cos(4 * np.pi * x) + 0.1 * rng.standard_normal(n)
    st = np.zeros((5, 4 + 2 * g, 5 + 2 * g, n + 2 * g))
    st[1, :, :, g:-g] = rho1
    st[2, :, :, g:-g] = v1
    st[0, :, :, g:-g] = 0.5
    orc.fill_ghosts(st, g)
    got = orc.wave1_rhs(st, g, h, 2)

    def d1(f):  # the printed loop, periodic
        return sum(wk * np.roll(f, -k) for k, wk in zip((-1, 0, 1), w1)) / h

    inner = (slice(g, -g),) * 3
    np.testing.assert_allclose(got[0][inner], np.broadcast_to(rho1, got[0][inner].shape), rtol=0, atol=1e-15)
    np.testing.assert_allclose(got[1][inner], np.broadcast_to(d1(v1), got[1][inner].shape), rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(got[2][inner], np.broadcast_to(d1(rho1), got[2][inner].shape), rtol=1e-13, atol=1e-12)
    for v in (3, 4):  # v_y, v_z: no y or z variation of rho
        np.testing.assert_allclose(got[v][inner], 0.0, atol=1e-12)
