"""Hash-consed expression DAG for the kernel generator.

Every node is interned, so structurally identical subexpressions are one
node: common-subexpression elimination happens by construction (the Kranc
"CSE" transformation of Sec. 3.2.3).  Sums are kept as linear combinations
{term: coefficient} + constant and products as {factor: power}; constants are
folded, (-a)*(-b) becomes a*b, and a*b + c becomes a fused multiply-add when
lowered (the peephole rules of Sec. 3.2.3).

`Dif(a, b)` is an opaque difference a - b that sums never flatten through:
stencils use it so that differences of neighbouring values are formed first
(exact for close values), whatever the surrounding algebra.
"""
from fractions import Fraction
import math

_TABLE = {}
_COUNTER = [0]


class Node:
    __slots__ = ("key", "id", "__weakref__")
    kind = "node"

    def __add__(self, o):
        return add(self, o)

    def __radd__(self, o):
        return add(o, self)

    def __sub__(self, o):
        return add(self, mul(-1, o))

    def __rsub__(self, o):
        return add(o, mul(-1, self))

    def __mul__(self, o):
        return mul(self, o)

    def __rmul__(self, o):
        return mul(o, self)

    def __neg__(self):
        return mul(-1, self)

    def __truediv__(self, o):
        if isinstance(o, (int, float, Fraction)):
            return mul(self, Fraction(1) / Fraction(o) if not isinstance(o, float) else 1.0 / o)
        return mul(self, rcp(o))

    def __pow__(self, n):
        assert isinstance(n, int) and n >= 0
        r = const(1)
        for _ in range(n):
            r = r * self
        return r

    def __repr__(self):
        return "<%s %d>" % (self.kind, self.id)

    def __lt__(self, o):
        return self.id < o.id


def _intern(cls, key, init):
    full = (cls.kind,) + key
    n = _TABLE.get(full)
    if n is None:
        n = cls.__new__(cls)
        n.key = full
        _COUNTER[0] += 1
        n.id = _COUNTER[0]
        init(n)
        _TABLE[full] = n
    return n


class Const(Node):
    __slots__ = ("value",)
    kind = "const"


class Sym(Node):
    """A named input: a loaded grid value or a runtime scalar."""
    __slots__ = ("name",)
    kind = "sym"


class Dif(Node):
    __slots__ = ("a", "b")
    kind = "dif"


class Add(Node):
    __slots__ = ("terms", "c0")   # terms: tuple of (node, coeff); c0 constant
    kind = "add"


class Mul(Node):
    __slots__ = ("factors",)      # tuple of (node, power)
    kind = "mul"


class Fn(Node):
    __slots__ = ("fn", "arg")     # 'exp' or 'rcp'
    kind = "fn"


def _num(x):
    if isinstance(x, Fraction):
        return x
    if isinstance(x, int):
        return Fraction(x)
    if isinstance(x, float):
        f = Fraction(x)
        return f
    raise TypeError(x)


def const(v):
    v = _num(v)

    def init(n):
        n.value = v
    return _intern(Const, (v,), init)


def sym(name):
    def init(n):
        n.name = name
    return _intern(Sym, (name,), init)


def dif(a, b):
    a, b = _wrap(a), _wrap(b)
    if a is b:
        return const(0)

    def init(n):
        n.a, n.b = a, b
    return _intern(Dif, (a.id, b.id), init)


def _wrap(x):
    if isinstance(x, Node):
        return x
    return const(x)


def _lin(x):
    """Linear-combination view: ({node: coeff}, constant)."""
    if isinstance(x, Const):
        return {}, x.value
    if isinstance(x, Add):
        return dict(x.terms), x.c0
    return {x: Fraction(1)}, Fraction(0)


def _make_add(terms, c0):
    terms = {k: v for k, v in terms.items() if v != 0}
    if not terms:
        return const(c0)
    if len(terms) == 1 and c0 == 0:
        (k, v), = terms.items()
        if v == 1:
            return k
    items = tuple(sorted(terms.items(), key=lambda kv: kv[0].id))

    def init(n):
        n.terms = items
        n.c0 = c0
    return _intern(Add, (tuple((k.id, v) for k, v in items), c0), init)


def add(a, b):
    a, b = _wrap(a), _wrap(b)
    ta, ca = _lin(a)
    tb, cb = _lin(b)
    for k, v in tb.items():
        ta[k] = ta.get(k, 0) + v
    return _make_add(ta, ca + cb)


def _mulview(x):
    """(coefficient, {factor: power}) view of a product-like node."""
    if isinstance(x, Const):
        return x.value, {}
    if isinstance(x, Add) and len(x.terms) == 1 and x.c0 == 0:
        (k, v), = x.terms
        c, f = _mulview(k)
        return c * v, f
    if isinstance(x, Mul):
        return Fraction(1), dict(x.factors)
    return Fraction(1), {x: 1}


def _make_mul(factors):
    factors = {k: p for k, p in factors.items() if p != 0}
    if not factors:
        return const(1)
    if len(factors) == 1:
        (k, p), = factors.items()
        if p == 1:
            return k
    items = tuple(sorted(factors.items(), key=lambda kv: kv[0].id))

    def init(n):
        n.factors = items
    return _intern(Mul, tuple((k.id, p) for k, p in items), init)


def mul(a, b):
    a, b = _wrap(a), _wrap(b)
    if isinstance(a, Const) and isinstance(b, Const):
        return const(a.value * b.value)
    if isinstance(a, Const) or isinstance(b, Const):
        c, x = (a, b) if isinstance(a, Const) else (b, a)
        if c.value == 0:
            return const(0)
        t, c0 = _lin(x)
        return _make_add({k: v * c.value for k, v in t.items()}, c0 * c.value)
    ca, fa = _mulview(a)
    cb, fb = _mulview(b)
    for k, p in fb.items():
        fa[k] = fa.get(k, 0) + p
    prod = _make_mul(fa)
    return mul(const(ca * cb), prod) if ca * cb != 1 else prod


def fn(name, x):
    x = _wrap(x)
    if isinstance(x, Const):
        v = float(x.value)
        return const(math.exp(v) if name == "exp" else 1.0 / v)

    def init(n):
        n.fn, n.arg = name, x
    return _intern(Fn, (name, x.id), init)


def exp(x):
    return fn("exp", x)


def rcp(x):
    return fn("rcp", x)


def total(xs):
    r = const(0)
    for x in xs:
        r = r + x
    return r


class Box(Node):
    """An opaque intermediate: sums and products never flatten into it, so
    the order of evaluation written by the author is kept."""
    __slots__ = ("x",)
    kind = "box"


def box(x):
    x = _wrap(x)
    if isinstance(x, (Const, Sym, Box, Dif)):
        return x

    def init(n):
        n.x = x
    return _intern(Box, (x.id,), init)


class Shx(Node):
    """The value `own` takes on the warp lane m places further along x; lanes
    whose source falls outside the warp read `ext` (the halo values, w on
    each side, held by the first 2w lanes).  No arithmetic."""
    __slots__ = ("own", "ext", "m", "w")
    kind = "shx"


def shx(own, ext, m, w):
    if m == 0:
        return own

    def init(n):
        n.own, n.ext, n.m, n.w = own, ext, m, w
    return _intern(Shx, (own.id, ext.id, m, w), init)


class Ext(Node):
    """A lane-dependent halo value computed by the kernel template: 'dx' the
    first difference f(x+1) - f(x) at the halo position of the lane, 'd1y' /
    'd1z' the raw first-derivative stencil (12h D) along y / z there."""
    __slots__ = ("what", "v")
    kind = "ext"


def ext(what, v):
    def init(n):
        n.what, n.v = what, v
    return _intern(Ext, (what, v), init)
