"""Lower an expression DAG to straight-line CUDA and count its operations.

Lowering rules (Sec. 3.2.3 peephole transformations, restated):
  - every DAG node is evaluated once (CSE by hash-consing);
  - a sum c0 + sum_i c_i x_i is an accumulation chain; a term with a
    coefficient other than +-1 becomes fma(c_i, x_i, acc); a product a*b
    used only inside one sum is fused into that sum as fma(+-a, b, acc);
  - a boxed sum or product used only as a +-1 term of one sum is flattened
    into that sum's chain (saves the separate add, lets the product fuse);
  - a term c (a b) with a single-use product takes the constant into the
    factor whose scaled copy c a the most such terms share, so each costs
    one fma (exact for powers of two; otherwise only where the scaled
    factor is shared);
  - negation is free (folded into the consuming instruction);
  - powers are repeated multiplication; rcp(x) is an IEEE 1.0/x; exp(x) is
    the library exp;
  - every add, subtract and multiply is written as an fma whose constant
    operand comes from the run-time constant table sc.k (a + b = fma(b, 1, a),
    a - b = fma(b, -1, a), a b = fma(a, b, -0), c x = fma(c, x, -0)): each is
    exact, so values are those of the plain operations, and numeric
    coefficients are never immediates.  On GB300 FP64 adds, multiplies and
    fmas with an immediate operand issue at 80 % of the rate of an fma whose
    operands are registers or constant-bank values (1.61 vs 1.87-1.91 per
    clock per SM, measured), and a table read from the kernel parameters
    cannot be folded back into immediates by the compiler.

Operation counts: algorithmic flops count fma as 2, add/sub/mul as 1 and
exp/rcp as 1 each; fp64 instructions count every add/sub/mul/fma as 1.
"""
from fractions import Fraction

from . import expr as E


def _lit(c):
    v = float(c)
    if v == int(v) and abs(v) < 1e15:
        return "%d.0" % int(v)
    return repr(v)


def _store(target, expr):
    """An output statement: integer targets go through the output functor
    (out(v, value)), so a kernel can consume each output as soon as it is
    computed; string targets are plain assignments."""
    if isinstance(target, int):
        return "out(%d, %s);" % (target, expr)
    return "%s = %s;" % (target, expr)


def _pow2(n):
    return n > 0 and n & (n - 1) == 0


# Run-time constant table: index -> value, shared by every generated body
# (written to csrc/generated/gen_constants.cuh; the library fills
# Scalars::k from it).  Fixed entries come first, for hand-written code.
K_FIXED = ((1.0, "ONE"), (-0.0, "MZERO"), (2.0, "TWO"), (8.0, "EIGHT"))
# The order of the other entries is pinned (exact decimal images of the
# values): the position of a constant in the kernel parameters changes the
# compiler's register allocation of the large bodies, and this order is the
# one measured fastest for the x/y-sharing BSSN body; constants not listed
# follow in increasing order.
K_PINNED = (16.0, 2.0 / 3.0, 4.0, 0.5, 1.0 / 6.0, 3.0, 1.0 / 3.0, 6.0, 15.0, 1.0 / 12.0, 0.75, 7.0, 10.0,
            5.0, 1.5, 0.15, 1.0 / 90.0, 1.0 / 60.0, 1.6, 0.2, 8.0 / 315.0, 1.0 / 560.0, 0.8, 4.0 / 105.0,
            1.0 / 280.0)
_KTAB = []
_KIDX = {}


def reset_constants(extra=()):
    """Empty the table but for the fixed entries, then the values of extra
    (non-negative) in the given order."""
    _KTAB.clear()
    _KIDX.clear()
    for v in [v for v, _ in K_FIXED] + list(extra):
        if _kkey(v) not in _KIDX:
            _KIDX[_kkey(v)] = len(_KTAB)
            _KTAB.append(v)


def _kkey(v):
    v = float(v)
    return (v, str(v).startswith("-"))


def constants():
    """The table as a list of floats (index order)."""
    return list(_KTAB)


def kref(c):
    """Operand text for the numeric constant c: sc.k[i], negated for c < 0
    (negation is an operand modifier: free)."""
    v = float(c)
    if v == 0.0:
        return "sc.k[%d]" % _KIDX[_kkey(-0.0)]
    a = abs(v)
    key = _kkey(a)
    if key not in _KIDX:
        _KIDX[key] = len(_KTAB)
        _KTAB.append(a)
    return ("-" if v < 0 else "") + "sc.k[%d]" % _KIDX[key]


ONE = "sc.k[0]"
MZERO = "sc.k[1]"


reset_constants()


class Lowering:
    def __init__(self, outputs, sym_expr, prelude=()):
        """outputs: list of (c_name, node); sym_expr: callable mapping a
        symbol name to a C expression (loads and runtime scalars)."""
        self.outputs = outputs
        self.prelude = list(prelude)
        self.sym_expr = sym_expr
        self.uses = {}
        self.names = {}
        self.lines = []
        self.loads = []
        self.flops = 0
        self.dp_ops = 0
        self.special = {"exp": 0, "rcp": 0}
        self._count_uses()
        self._count_scalings()

    # -- use counts --------------------------------------------------------
    def _children(self, n):
        if isinstance(n, E.Add):
            return [k for k, _ in n.terms]
        if isinstance(n, E.Mul):
            return [k for k, _ in n.factors]
        if isinstance(n, E.Dif):
            return [n.a, n.b]
        if isinstance(n, E.Fn):
            return [n.arg]
        if isinstance(n, E.Box):
            return [n.x]
        if isinstance(n, E.Shx):
            return [n.own, n.ext]
        return []

    def _count_uses(self):
        seen = set()
        roots = []
        for _, n in self.outputs:
            roots += [m for _, m in n] if isinstance(n, list) else [n]
        stack = list(roots)
        for n in roots:
            self.uses[n] = self.uses.get(n, 0) + 1
        while stack:
            n = stack.pop()
            if n.id in seen:
                continue
            seen.add(n.id)
            for c in self._children(n):
                self.uses[c] = self.uses.get(c, 0) + 1
                stack.append(c)

    # -- flattening and constant absorption ----------------------------------
    def _single(self, n):
        return self.uses.get(n, 0) == 1 and n not in self.names

    def _unbox_mul(self, x):
        """The product inside a single-use box of a single-use product."""
        if (isinstance(x, E.Box) and isinstance(x.x, E.Mul) and self._single(x)
                and self.uses.get(x.x, 0) == 1 and x.x not in self.names):
            return x.x
        return x

    def _flat_terms(self, n, c, out):
        """Terms of the sum n scaled by c (+-1) into out, single-use boxed sums
        flattened; returns the constant part."""
        c0 = n.c0 * c
        for x, cx in n.terms:
            cc = cx * c
            if (isinstance(x, E.Box) and isinstance(x.x, E.Add) and abs(cc) == 1 and self._single(x)
                    and self.uses.get(x.x, 0) == 1 and x.x not in self.names):
                c0 += self._flat_terms(x.x, cc, out)
            else:
                out.append((self._unbox_mul(x), cc))
        return c0

    @staticmethod
    def _scalable(a):
        return not (isinstance(a, E.Add) and (len(a.terms) != 1 or a.c0 != 0))

    def _count_scalings(self):
        """How many single-use product terms c (a b) could share each scaled
        factor |c| a (absorption candidates)."""
        self.scalings = {}
        for n in list(self.uses):
            if not isinstance(n, E.Add):
                continue
            for x, c in n.terms:
                x = self._unbox_mul(x)
                if abs(c) == 1 or not isinstance(x, E.Mul) or self.uses.get(x, 0) != 1:
                    continue
                for a in {k for k, _ in x.factors}:
                    if self._scalable(a):
                        key = (abs(c), a)
                        self.scalings[key] = self.scalings.get(key, 0) + 1

    # -- emission ----------------------------------------------------------
    def _op(self, flops, text, node=None):
        self.flops += flops
        self.dp_ops += 1
        return text

    def value(self, n):
        """C expression naming the value of node n (emitting it if needed)."""
        if n in self.names:
            return self.names[n]
        if isinstance(n, E.Const):
            return kref(n.value)
        if isinstance(n, E.Sym):
            name = self._sym(n)
            self.names[n] = name
            return name
        expr = self._lower(n)
        name = "t%d" % n.id
        self.lines.append("const double %s = %s;" % (name, expr))
        self.names[n] = name
        return name

    def _sym(self, n):
        ce, is_load = self.sym_expr(n.name)
        if not is_load:
            return ce
        name = "v_" + n.name.replace("-", "m")
        self.loads.append(name)
        self.lines.append("const double %s = %s;" % (name, ce))
        return name

    def _lower(self, n):
        if isinstance(n, E.Box):
            return self._lower_inner(n.x)
        return self._lower_inner(n)

    def _lower_inner(self, n):
        if isinstance(n, (E.Const, E.Sym)):
            return self.value(n)
        if isinstance(n, E.Box):
            return self.value(n)
        if isinstance(n, E.Dif):
            a, b = self.value(n.a), self.value(n.b)
            return self._op(1, "fma(%s, -%s, %s)" % (b, ONE, a))
        if isinstance(n, E.Fn):
            x = self.value(n.arg)
            self.special[n.fn] += 1
            self.flops += 1
            if n.fn == "exp":
                return "exp(%s)" % x
            return "1.0 / %s" % x
        if isinstance(n, E.Mul):
            return self._lower_mul(n.factors)
        if isinstance(n, E.Add):
            return self._lower_add(n)
        if isinstance(n, E.Shx):
            return "chemora_xshfl(%s, %s, %d, %d)" % (self.value(n.own), self.value(n.ext), n.m, n.w)
        if isinstance(n, E.Ext):
            # the halo value costs what its stencil costs: 1 (dx) or 3 (d1) fp64 instructions
            cost = 1 if n.what == "dx" else 3
            self.dp_ops += cost
            self.flops += 1 if n.what == "dx" else 4
            if n.what == "dx":
                return "ld.ext_dx(%d, %s)" % (n.v, ONE)
            return "ld.ext_%s(%d, %s, %s)" % (n.what, n.v, ONE, kref(8))
        raise TypeError(n)

    def _lower_mul(self, factors):
        seq = []
        for k, p in factors:
            seq += [k] * p
        vals = [self.value(k) for k in seq]
        expr = vals[0]
        for v in vals[1:]:
            expr = self._op(1, "fma(%s, %s, %s)" % (expr, v, MZERO))
        return expr

    def _fusable(self, x):
        """A product used only here, split as (rest, last) for an fma."""
        x = self._unbox_mul(x)
        if not isinstance(x, E.Mul) or self.uses.get(x, 0) != 1:
            return None
        seq = []
        for k, p in x.factors:
            seq += [k] * p
        if len(seq) < 2:
            return None
        # keep the existing (shared) partial product when there is one
        best = None
        for i in range(len(seq)):
            rest_f = {}
            for j, k in enumerate(seq):
                if j != i:
                    rest_f[k] = rest_f.get(k, 0) + 1
            rest = E._make_mul(rest_f)
            score = (1 if (rest in self.uses or rest in self.names) else 0, seq[i].id)
            if best is None or score > best[0]:
                best = (score, rest, seq[i])
        return best[1], best[2]

    def _absorb(self, x, c, start=False):
        """For a single-use product x = a * rest and a constant c, the pair
        (|c| a, rest) with the factor a whose scaled copy the most terms
        share, so that a sum of c a b_i costs one fma per term.  Powers of two
        scale exactly and are always absorbed; other constants only into a
        shared scaled factor (one rounding moves from c (a b) to (c a) b).
        As the first term of a chain (start) only a shared scaled factor
        pays (it saves the second multiply)."""
        x = self._unbox_mul(x)
        if not isinstance(x, E.Mul) or self.uses.get(x, 0) != 1:
            return None
        seq = []
        for k, p in x.factors:
            seq += [k] * p
        if len(seq) < 2:
            return None
        ac = abs(c)
        pow2 = _pow2(ac.numerator) and _pow2(ac.denominator) if isinstance(ac, Fraction) else False
        best = None
        for a in sorted(set(seq), key=lambda k: k.id):
            if not self._scalable(a):
                continue
            shared = self.scalings.get((ac, a), 0)
            scaled = E.mul(E.const(ac), a)
            known = scaled in self.names
            score = (known or shared >= 2, shared, -a.id)
            if best is None or score > best[0]:
                best = (score, a, scaled)
        if best is None:
            return None
        if not best[0][0] and (start or not pow2):
            return None
        a = best[1]
        rest_f = {}
        removed = False
        for k in seq:
            if k is a and not removed:
                removed = True
                continue
            rest_f[k] = rest_f.get(k, 0) + 1
        return best[2], E._make_mul(rest_f)

    def _lower_add(self, n):
        flat = []
        c0 = self._flat_terms(n, Fraction(1), flat)
        merged = {}
        for x, c in flat:
            merged[x] = merged.get(x, 0) + c
        terms = [(x, c) for x, c in merged.items() if c != 0]
        # order: plain (+-1) non-fusable terms first so the chain starts free
        def kind(t):
            x, c = t
            if abs(c) == 1 and self._fusable(x) is None:
                return 0
            return 1
        terms.sort(key=lambda t: (kind(t), t[0].id))
        acc = None
        if c0 != 0:
            acc = kref(c0)
        for x, c in terms:
            fz = self._fusable(x) if abs(c) == 1 else None
            sg = "" if c > 0 else "-"
            if acc is None:
                if abs(c) == 1 and fz is None:
                    v = self.value(x)
                    acc = v if c == 1 else "(-%s)" % v
                elif fz is not None:
                    r, l = fz
                    acc = self._op(1, "fma(%s%s, %s, %s)" % (sg, self.value(r), self.value(l), MZERO))
                else:
                    ab = self._absorb(x, c, start=True)
                    if ab is not None:
                        acc = self._op(1, "fma(%s%s, %s, %s)" % (sg, self.value(ab[0]), self.value(ab[1]), MZERO))
                    else:
                        acc = self._op(1, "fma(%s, %s, %s)" % (kref(c), self.value(x), MZERO))
                continue
            if fz is not None:
                r, l = fz
                rv, lv = self.value(r), self.value(l)
                acc = self._op(2, "fma(%s%s, %s, %s)" % (sg, rv, lv, acc))
            elif abs(c) == 1:
                acc = self._op(1, "fma(%s, %s%s, %s)" % (self.value(x), "" if c == 1 else "-", ONE, acc))
            else:
                ab = self._absorb(x, c)
                if ab is not None:
                    # c (a b) -> (|c| a) b with the scaled factor shared
                    acc = self._op(2, "fma(%s%s, %s, %s)" % (sg, self.value(ab[0]), self.value(ab[1]), acc))
                else:
                    acc = self._op(2, "fma(%s, %s, %s)" % (kref(c), self.value(x), acc))
        return acc

    def run(self):
        for n in self.prelude:
            if n in self.uses:
                self.value(n)
        outs = []
        for cname, node in self.outputs:
            if isinstance(node, list):
                vals = [(c, _lit(n.value) if isinstance(n, E.Const) else self.value(n)) for c, n in node]
                expr = vals[-1][1]
                for c, v in reversed(vals[:-1]):
                    expr = "(%s) ? %s : %s" % (c, v, expr)
                outs.append(_store(cname, expr))
            elif isinstance(node, E.Const):
                outs.append(_store(cname, _lit(node.value)))
            else:
                outs.append(_store(cname, self.value(node)))
        return outs


def emit_function(fname, outputs, sym_expr, nout, comment, prelude=()):
    """CUDA device function `fname(ld, sc, out)` computing the outputs.
    prelude: nodes evaluated first, in the given order (controls the
    emission order, e.g. per-variable stencil blocks before the algebra)."""
    L = Lowering(outputs, sym_expr, prelude)
    outs = L.run()
    body = []
    body.append("// %s" % comment)
    body.append("// generated: %d fp64 instructions, %d algorithmic flops, %d exp, %d rcp per point"
                % (L.dp_ops, L.flops, L.special["exp"], L.special["rcp"]))
    body.append("// out(v, value) receives output v (%d outputs) as soon as it is computed" % nout)
    body.append("template <class LD, class SC, class OUT>")
    body.append("__device__ __forceinline__ void %s(const LD& ld, const SC& sc, OUT& out) {" % fname)
    body += ["  " + s for s in L.lines]
    body += ["  " + s for s in outs]
    body.append("}")
    return "\n".join(body) + "\n", L
