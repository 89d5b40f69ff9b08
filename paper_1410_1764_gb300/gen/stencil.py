"""Finite-difference stencils built as DAG nodes over neighbour values
(Sec. 3.2.2: centred 4th-order operators and 5th-order Kreiss-Oliger
dissipation).

Neighbour values are symbols "f<v>_<dx>_<dy>_<dz>".  Differences of
neighbours are formed first (symmetric pairs for first derivatives,
neighbours against the centre for second derivatives and dissipation), then
combined, then multiplied by a runtime scale (1/(12h), 1/(12h^2),
1/(144h^2), eps/(64h)).
"""
from fractions import Fraction

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


# ---------------------------------------------------------------------------
# x-sharing mode: a warp holds 32 consecutive x points, so differences and
# derivative rows along x come from neighbouring lanes (warp shuffles, no
# arithmetic).  Halo lanes hold 3 first differences / 2 derivative rows on
# each side of the warp.
# ---------------------------------------------------------------------------
_XSHARE = [False]


class xshare:
    """Context manager: build stencils in x-sharing form."""

    def __enter__(self):
        self.prev = _XSHARE[0]
        _XSHARE[0] = True

    def __exit__(self, *exc):
        _XSHARE[0] = self.prev


_YSHARE = [False]
# variables whose z first-derivative rows are shared (those with second
# derivatives in the BSSN system: phi, gt_ij, alpha, beta^i), in smem order
ZROW_VARS = (0, 1, 2, 3, 4, 5, 6, 17, 18, 19, 20)


class yshare:
    """Context manager: y-direction first differences and z-derivative rows
    come from shared memory filled by the kernel's prologue (symbols
    sdy_<v>_<m>: f(y+m+1) - f(y+m); sdz_<v>_<m>: 12h D_z f at y+m)."""

    def __enter__(self):
        self.prev = _YSHARE[0]
        _YSHARE[0] = True

    def __exit__(self, *exc):
        _YSHARE[0] = self.prev


_ZQUEUE = [False]


class zqueue:
    """Context manager: the z-direction pure second derivative comes from a
    register queue of z first differences kept by a thread that marches
    along z (symbols zqa_<v> = e_0 - e_-1 and zqb_<v> = e_1 - e_-2, with
    e_m = f(z+m+1) - f(z+m)); 12h^2 D_zz f = 15 zqa - zqb."""

    def __enter__(self):
        self.prev = _ZQUEUE[0]
        _ZQUEUE[0] = True

    def __exit__(self, *exc):
        _ZQUEUE[0] = self.prev


def _zq(what, v):
    return E.sym("zq%s_%d" % (what, v))


def _dy(v, m):
    return E.sym("sdy_%d_%d" % (v, m))


def _zrow(v, m):
    return E.sym("sdz_%d_%d" % (v, m))


def _dabc(dd):
    a = E.dif(dd(0), dd(-1))
    b = E.dif(dd(1), dd(-2))
    c = E.dif(dd(2), dd(-3))
    return a, b, c


def _dx(v, m):
    """f(x+m+1) - f(x+m), the first difference m lanes away."""
    own = E.dif(val(v, (1, 0, 0)), val(v))
    return E.shx(own, E.ext("dx", v), m, 3)


def _xabc(v):
    """a = d_1, b = d_2 - d_1, c = d_3 - d_2 in first differences (d_k the
    centre-difference sums): a = dx_0 - dx_-1, b = dx_1 - dx_-2,
    c = dx_2 - dx_-3."""
    a = E.dif(_dx(v, 0), _dx(v, -1))
    b = E.dif(_dx(v, 1), _dx(v, -2))
    c = E.dif(_dx(v, 2), _dx(v, -3))
    return a, b, c


def d1_raw(v, a, base=(0, 0, 0)):
    """12h * D1_a at base: 8 (f+1 - f-1) - (f+2 - f-2)."""
    if _YSHARE[0] and base == (0, 0, 0):
        if a == 1:
            s1 = E.box(_dy(v, 0) + _dy(v, -1))
            s2 = E.box(_dy(v, 1) + _dy(v, -2))
            return E.box(7 * s1 - s2)
        if a == 2 and v in ZROW_VARS:
            return _zrow(v, 0)
    if _XSHARE[0] and a == 0 and base == (0, 0, 0):
        # f+1 - f-1 = dx_0 + dx_-1 = s1, f+2 - f-2 = s1 + s2: 7 s1 - s2
        s1 = E.box(_dx(v, 0) + _dx(v, -1))
        s2 = E.box(_dx(v, 1) + _dx(v, -2))
        return E.box(7 * s1 - s2)
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
    if _XSHARE[0] and a == 0:
        xa, xb, _ = _xabc(v)
        return E.box(15 * xa - xb)  # 16 a - (a + b)
    if _YSHARE[0] and a == 1:
        ya, yb, _ = _dabc(lambda m: _dy(v, m))
        return E.box(15 * ya - yb)
    if _ZQUEUE[0] and a == 2:
        return E.box(15 * _zq("a", v) - _zq("b", v))
    return E.box(16 * _centre_diffs(v, a, 1) - _centre_diffs(v, a, 2))


def d2(v, a):
    """Pure second derivative: (16 d1 - d2) / (12h^2)."""
    return E.box(d2_raw(v, a) * I12H2)


def d11_raw(v, a, b):
    """144h^2 * mixed derivative D_a D_b: the first-derivative stencil along
    b applied to first-derivative rows along a."""
    if _YSHARE[0] and a == 1 and b == 2 and v in ZROW_VARS:
        # the y stencil applied to the z-derivative rows of the rows y +- m
        Z = {m: _zrow(v, m) for m in (-2, -1, 1, 2)}
        return E.box(8 * E.dif(Z[1], Z[-1]) - E.dif(Z[2], Z[-2]))
    if _XSHARE[0] and a == 0:
        # the x stencil applied to the neighbours' own D_b rows
        own = d1_raw(v, b)
        Y = {m: E.shx(own, E.ext("d1y" if b == 1 else "d1z", v), m, 2) for m in (-2, -1, 1, 2)}
        return E.box(8 * E.dif(Y[1], Y[-1]) - E.dif(Y[2], Y[-2]))
    r = {m: d1_raw(v, a, _off((0, 0, 0), b, m)) for m in (-2, -1, 1, 2)}
    return E.box(8 * E.dif(r[1], r[-1]) - E.dif(r[2], r[-2]))


def d11(v, a, b):
    """Mixed derivative D_a D_b."""
    return E.box(d11_raw(v, a, b) * I144H2)


def dd(v, a, b):
    return d2(v, a) if a == b else d11(v, min(a, b), max(a, b))


def ko_raw(v, a):
    """64h/eps * KO_a: (d3 - 6 d2 + 15 d1)."""
    if _XSHARE[0] and a == 0:
        xa, xb, xc = _xabc(v)
        return E.box(10 * xa - 5 * xb + xc)  # (a+b+c) - 6 (a+b) + 15 a
    if _YSHARE[0] and a == 1:
        ya, yb, yc = _dabc(lambda m: _dy(v, m))
        return E.box(10 * ya - 5 * yb + yc)
    return E.box(_centre_diffs(v, a, 3) - 6 * _centre_diffs(v, a, 2) + 15 * _centre_diffs(v, a, 1))


def ko(v):
    """Kreiss-Oliger dissipation summed over the three directions."""
    return E.box(E.box(ko_raw(v, 0) + ko_raw(v, 1) + ko_raw(v, 2)) * KO_SCALE)


# ---------------------------------------------------------------------------
# Central differencing of arbitrary even order (Sec. 3.2.2): the weights
# solve the moment conditions exactly in rationals.
# ---------------------------------------------------------------------------
IH = E.sym("ih")
IH2 = E.sym("ih2")


def _solve(A, b):
    """Exact Gaussian elimination over Fractions."""
    n = len(b)
    M = [list(map(Fraction, row)) + [Fraction(bi)] for row, bi in zip(A, b)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def fd_weights(order):
    """(a, b): D1 f = (1/h) sum_k a_k (f_k - f_-k) exact for degree <= order,
    D2 f = (1/h^2) sum_k b_k ((f_k - f_0) + (f_-k - f_0)) exact for degree
    <= order + 1, k = 1..order/2."""
    if order < 2 or order % 2:
        raise ValueError("order must be even and >= 2")
    m = order // 2
    # sum_k a_k (k^j - (-k)^j) = [j == 1] for odd j
    a = _solve([[2 * k ** j for k in range(1, m + 1)] for j in range(1, 2 * m, 2)],
               [1 if j == 1 else 0 for j in range(1, 2 * m, 2)])
    # sum_k b_k (k^j + (-k)^j) = 2 [j == 2] for even j >= 2
    b = _solve([[2 * k ** j for k in range(1, m + 1)] for j in range(2, 2 * m + 1, 2)],
               [2 if j == 2 else 0 for j in range(2, 2 * m + 1, 2)])
    return a, b


def d1o_raw(v, axis, order):
    """h * order-p first derivative."""
    a, _ = fd_weights(order)
    acc = E.const(0)
    for k in range(len(a), 0, -1):
        acc = acc + a[k - 1] * E.dif(val(v, _off((0, 0, 0), axis, k)), val(v, _off((0, 0, 0), axis, -k)))
    return E.box(acc)


def d2o_raw(v, axis, order):
    """h^2 * order-p pure second derivative (differences from the centre)."""
    _, b = fd_weights(order)
    acc = E.const(0)
    for k in range(len(b), 0, -1):
        acc = acc + b[k - 1] * _centre_diffs(v, axis, k)
    return E.box(acc)
