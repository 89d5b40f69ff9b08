"""Finite-difference stencils built as DAG nodes over neighbour values
(Sec. 3.2.2: centred 4th-order operators and 5th-order Kreiss-Oliger
dissipation).

Neighbour values are symbols "f<v>_<dx>_<dy>_<dz>".  Differences of
neighbours are formed first (symmetric pairs for first derivatives,
neighbours against the centre for second derivatives and dissipation), then
combined, then multiplied by a runtime scale (1/(12h), 1/(12h^2),
1/(144h^2), eps/(64h)).
"""
from . import expr as E

AXES = ((1, 0, 0), (0, 1, 0), (0, 0, 1))

I12H = E.sym("i12h")
I12H2 = E.sym("i12h2")
I144H2 = E.sym("i144h2")
KO_SCALE = E.sym("ko_scale")


def val(v, off=(0, 0, 0)):
    return E.sym("f%d_%d_%d_%d" % (v, off[0], off[1], off[2]))


def _off(base, axis, m):
    o = list(base)
    for q in range(3):
        o[q] += AXES[axis][q] * m
    return tuple(o)


def d1_raw(v, a, base=(0, 0, 0)):
    """12h * D1_a at base: 8 (f+1 - f-1) - (f+2 - f-2)."""
    p1 = E.dif(val(v, _off(base, a, 1)), val(v, _off(base, a, -1)))
    p2 = E.dif(val(v, _off(base, a, 2)), val(v, _off(base, a, -2)))
    return E.box(8 * p1 - p2)


def _centre_diffs(v, a, k):
    f0 = val(v)
    return E.box(E.dif(val(v, _off((0, 0, 0), a, k)), f0) + E.dif(val(v, _off((0, 0, 0), a, -k)), f0))


def d1(v, a):
    return E.box(d1_raw(v, a) * I12H)


def d2_raw(v, a):
    """12h^2 * pure second derivative: 16 d1 - d2, d_k = (f+k - f0) + (f-k - f0)."""
    return E.box(16 * _centre_diffs(v, a, 1) - _centre_diffs(v, a, 2))


def d2(v, a):
    """Pure second derivative: (16 d1 - d2) / (12h^2)."""
    return E.box(d2_raw(v, a) * I12H2)


def d11_raw(v, a, b):
    """144h^2 * mixed derivative D_a D_b: the first-derivative stencil along
    b applied to first-derivative rows along a."""
    r = {m: d1_raw(v, a, _off((0, 0, 0), b, m)) for m in (-2, -1, 1, 2)}
    return E.box(8 * E.dif(r[1], r[-1]) - E.dif(r[2], r[-2]))


def d11(v, a, b):
    """Mixed derivative D_a D_b."""
    return E.box(d11_raw(v, a, b) * I144H2)


def dd(v, a, b):
    return d2(v, a) if a == b else d11(v, min(a, b), max(a, b))


def ko_raw(v, a):
    """64h/eps * KO_a: (d3 - 6 d2 + 15 d1)."""
    return E.box(_centre_diffs(v, a, 3) - 6 * _centre_diffs(v, a, 2) + 15 * _centre_diffs(v, a, 1))


def ko(v):
    """Kreiss-Oliger dissipation summed over the three directions."""
    return E.box(E.box(ko_raw(v, 0) + ko_raw(v, 1) + ko_raw(v, 2)) * KO_SCALE)
