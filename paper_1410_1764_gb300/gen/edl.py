"""A small equation-description front end for the generator (the role the
paper's EDL plays in Sec. 3.3: a language with a real parser, so errors are
reported with a line and a column).  The syntax here is this project's own.

    # comment
    system NAME
    order P                      # finite-difference order (even, default 4)
    field NAME                   # a scalar grid function
    field NAME[i]                # a vector: three grid functions (x, y, z)
    rhs NAME = EXPR              # right-hand side of a scalar field
    rhs NAME[i] = EXPR           # of a vector field; i is a free index

Expressions: numbers, + - * /, ^ with an integer exponent, parentheses,
fields (u, v[j], v[0]), and the built-ins
    d(F, i)        first derivative of field F along index i
    dd(F, i, j)    second derivative (pure when i == j, else mixed)
    sum(j, EXPR)   sum of EXPR over j = x, y, z
    delta(i, j)    Kronecker delta
Index slots take a free or summation index name, or a literal 0/1/2 or x/y/z.
Fields are numbered in declaration order (vector components consecutively),
which is the variable order of the generated kernel.

`compile_system(text)` returns (name, order, field names, list of DAG
nodes, one right-hand side per grid function).
"""
from fractions import Fraction

from . import expr as E
from .stencil import IH, IH2, _off, d1o_raw, d2o_raw, fd_weights, val

AXIS = {"x": 0, "y": 1, "z": 2, "0": 0, "1": 1, "2": 2}


class EdlError(ValueError):
    def __init__(self, line, col, msg):
        super().__init__("line %d, col %d: %s" % (line, col, msg))
        self.line, self.col, self.msg = line, col, msg


# ---------------------------------------------------------------------------
# tokens
# ---------------------------------------------------------------------------

def _tokens(text, line_no):
    """Tokens of one line: (kind, value, col); kinds: name, num, op."""
    out, i, n = [], 0, len(text)
    while i < n:
        ch = text[i]
        if ch in " \t":
            i += 1
        elif ch == "#":
            break
        elif ch.isalpha() or ch == "_":
            j = i
            while j < n and (text[j].isalnum() or text[j] == "_"):
                j += 1
            out.append(("name", text[i:j], i + 1))
            i = j
        elif ch.isdigit() or (ch == "." and i + 1 < n and text[i + 1].isdigit()):
            j = i
            while j < n and (text[j].isdigit() or text[j] == "."):
                j += 1
            out.append(("num", text[i:j], i + 1))
            i = j
        elif ch in "+-*/^()[],=":
            out.append(("op", ch, i + 1))
            i += 1
        else:
            raise EdlError(line_no, i + 1, "unexpected character %r" % ch)
    return out


# ---------------------------------------------------------------------------
# expression parser (recursive descent) -> nested tuples
# ---------------------------------------------------------------------------

class _Parser:
    def __init__(self, toks, line_no, end_col):
        self.t, self.k, self.line, self.end = toks, 0, line_no, end_col

    def peek(self):
        return self.t[self.k] if self.k < len(self.t) else ("eol", "", self.end)

    def take(self, kind=None, value=None):
        tok = self.peek()
        if (kind and tok[0] != kind) or (value and tok[1] != value):
            want = value or kind
            raise EdlError(self.line, tok[2], "expected %s, found %s" % (
                want, "end of line" if tok[0] == "eol" else repr(tok[1])))
        self.k += 1
        return tok

    def expr(self):
        node = self.term()
        while self.peek()[1] in ("+", "-") and self.peek()[0] == "op":
            op = self.take()[1]
            node = (op, node, self.term())
        return node

    def term(self):
        node = self.factor()
        while self.peek()[1] in ("*", "/") and self.peek()[0] == "op":
            op = self.take()[1]
            node = (op, node, self.factor())
        return node

    def factor(self):
        if self.peek() == ("op", "-", self.peek()[2]):
            col = self.take()[2]
            return ("neg", self.factor(), col)
        node = self.atom()
        if self.peek()[0] == "op" and self.peek()[1] == "^":
            self.take()
            tok = self.take("num")
            if not tok[1].isdigit():
                raise EdlError(self.line, tok[2], "exponent must be a non-negative integer")
            node = ("pow", node, int(tok[1]))
        return node

    def atom(self):
        tok = self.peek()
        if tok[0] == "num":
            self.take()
            return ("num", Fraction(tok[1]), tok[2])
        if tok[0] == "op" and tok[1] == "(":
            self.take()
            node = self.expr()
            self.take("op", ")")
            return node
        if tok[0] == "name":
            self.take()
            name, col = tok[1], tok[2]
            if self.peek()[1] == "(" and self.peek()[0] == "op":
                self.take()
                args = [self.expr()]
                while self.peek()[1] == ",":
                    self.take()
                    args.append(self.expr())
                self.take("op", ")")
                return ("call", name, args, col)
            idx = []
            if self.peek()[1] == "[" and self.peek()[0] == "op":
                self.take()
                idx.append(self.index_tok())
                while self.peek()[1] == ",":
                    self.take()
                    idx.append(self.index_tok())
                self.take("op", "]")
            return ("ref", name, idx, col)
        raise EdlError(self.line, tok[2], "expected an expression, found %s" % (
            "end of line" if tok[0] == "eol" else repr(tok[1])))

    def index_tok(self):
        tok = self.peek()
        if tok[0] in ("name", "num"):
            self.take()
            return (tok[1], tok[2])
        raise EdlError(self.line, tok[2], "expected an index")


# ---------------------------------------------------------------------------
# compilation to generator DAG nodes
# ---------------------------------------------------------------------------

class _System:
    def __init__(self):
        self.name = None
        self.order = 4
        self.fields = {}   # name -> (first variable number, is_vector, line)
        self.nvars = 0
        self.rhs = {}      # variable number -> node
        self.comp_names = []


def _mixed_raw(var, a, b, order):
    """h^2 * mixed derivative: the order-p first-derivative stencil along b
    applied to first-derivative rows along a."""
    w, _ = fd_weights(order)
    acc = E.const(0)
    for m in range(len(w), 0, -1):
        rows = []
        for sm in (m, -m):
            base = _off((0, 0, 0), b, sm)
            r = E.const(0)
            for k in range(len(w), 0, -1):
                r = r + w[k - 1] * E.dif(val(var, _off(base, a, k)), val(var, _off(base, a, -k)))
            rows.append(E.box(r))
        acc = acc + w[m - 1] * E.dif(rows[0], rows[1])
    return E.box(acc)


class _Compiler:
    def __init__(self, sysm, line_no):
        self.s, self.line = sysm, line_no

    def err(self, col, msg):
        raise EdlError(self.line, col, msg)

    def axis(self, tok, env):
        name, col = tok
        if name in env:
            return env[name]
        if name in AXIS:
            return AXIS[name]
        self.err(col, "unknown index %r" % name)

    def field_var(self, node, env):
        if node[0] != "ref":
            self.err(self._col(node), "expected a field")
        _, name, idx, col = node
        if name not in self.s.fields:
            self.err(col, "unknown field %r" % name)
        base, vec, _ = self.s.fields[name]
        if vec != bool(idx) or len(idx) > 1:
            self.err(col, "field %r takes %s" % (name, "one index" if vec else "no index"))
        return base + (self.axis(idx[0], env) if vec else 0)

    def index_arg(self, node, env):
        if node[0] == "ref" and not node[2] and node[1] not in self.s.fields:
            return self.axis((node[1], node[3]), env)
        if node[0] == "num" and node[1] in (0, 1, 2):
            return int(node[1])
        self.err(self._col(node), "expected an index")

    def _col(self, node):
        return node[-1] if isinstance(node[-1], int) else 1

    def ev(self, node, env):
        kind = node[0]
        if kind == "num":
            return E.const(node[1])
        if kind == "neg":
            return -self.ev(node[1], env)
        if kind == "pow":
            return self.ev(node[1], env) ** node[2]
        if kind in ("+", "-", "*", "/"):
            a, b = self.ev(node[1], env), self.ev(node[2], env)
            if kind == "+":
                return a + b
            if kind == "-":
                return a - b
            if kind == "*":
                return a * b
            if isinstance(b, E.Const) and b.value == 0:
                self.err(self._col(node[2]), "division by zero")
            return a / b
        if kind == "ref":
            return val(self.field_var(node, env))
        if kind == "call":
            _, name, args, col = node
            order = self.s.order
            if name == "d":
                if len(args) != 2:
                    self.err(col, "d(F, i) takes 2 arguments")
                v, a = self.field_var(args[0], env), self.index_arg(args[1], env)
                return d1o_raw(v, a, order) * IH  # unboxed: sums fuse the scale into fmas
            if name == "dd":
                if len(args) != 3:
                    self.err(col, "dd(F, i, j) takes 3 arguments")
                v = self.field_var(args[0], env)
                a, b = self.index_arg(args[1], env), self.index_arg(args[2], env)
                if a == b:
                    return d2o_raw(v, a, order) * IH2
                return _mixed_raw(v, min(a, b), max(a, b), order) * IH2
            if name == "sum":
                if len(args) != 2 or args[0][0] != "ref" or args[0][2]:
                    self.err(col, "sum(j, EXPR) takes an index name and an expression")
                j = args[0][1]
                if j in env or j in self.s.fields or j in AXIS:
                    self.err(args[0][3], "summation index %r is already in use" % j)
                acc = E.const(0)
                for ax in range(3):
                    acc = acc + self.ev(args[1], dict(env, **{j: ax}))
                return acc
            if name == "delta":
                if len(args) != 2:
                    self.err(col, "delta(i, j) takes 2 arguments")
                return E.const(1 if self.index_arg(args[0], env) == self.index_arg(args[1], env) else 0)
            self.err(col, "unknown function %r" % name)
        raise AssertionError(node)


def compile_system(text, order=None):
    """Parse and compile an equation file; returns (name, order, component
    names, [node per grid function]).  `order` overrides the file's order."""
    sysm = _System()
    lines = text.splitlines()
    for ln, raw in enumerate(lines, 1):
        toks = _tokens(raw, ln)
        if not toks:
            continue
        kw = toks[0]
        if kw[0] != "name":
            raise EdlError(ln, kw[2], "expected a statement keyword")
        p = _Parser(toks[1:], ln, len(raw) + 1)
        if kw[1] == "system":
            sysm.name = p.take("name")[1]
        elif kw[1] == "order":
            tok = p.take("num")
            o = int(Fraction(tok[1])) if Fraction(tok[1]).denominator == 1 else -1
            if o < 2 or o % 2 or o > 16:
                raise EdlError(ln, tok[2], "order must be an even integer in [2, 16]")
            if sysm.rhs:
                raise EdlError(ln, kw[2], "order must come before the first rhs")
            sysm.order = o
        elif kw[1] == "field":
            name_tok = p.take("name")
            name = name_tok[1]
            if name in sysm.fields or name in ("d", "dd", "sum", "delta") or name in AXIS:
                raise EdlError(ln, name_tok[2], "field name %r is taken" % name)
            vec = False
            if p.peek()[1] == "[":
                p.take()
                p.take("name")
                p.take("op", "]")
                vec = True
            sysm.fields[name] = (sysm.nvars, vec, ln)
            sysm.comp_names += [name + "_" + c for c in "xyz"] if vec else [name]
            sysm.nvars += 3 if vec else 1
        elif kw[1] == "rhs":
            name_tok = p.take("name")
            if name_tok[1] not in sysm.fields:
                raise EdlError(ln, name_tok[2], "unknown field %r" % name_tok[1])
            base, vec, _ = sysm.fields[name_tok[1]]
            free = None
            if p.peek()[1] == "[":
                p.take()
                free = p.take("name")
                p.take("op", "]")
            if vec != (free is not None):
                raise EdlError(ln, name_tok[2], "field %r takes %s" % (
                    name_tok[1], "one free index" if vec else "no index"))
            p.take("op", "=")
            tree = p.expr()
            if p.peek()[0] != "eol":
                raise EdlError(ln, p.peek()[2], "unexpected %r" % p.peek()[1])
            comp = _Compiler(sysm, ln)
            for ax in (range(3) if vec else [None]):
                var = base + (ax or 0)
                if var in sysm.rhs:
                    raise EdlError(ln, name_tok[2], "second rhs for %r" % sysm.comp_names[var])
                env = {free[1]: ax} if vec else {}
                sysm.rhs[var] = E.box(comp.ev(tree, env))
        else:
            raise EdlError(ln, kw[2], "unknown statement %r" % kw[1])
        if kw[1] in ("system", "order") and p.peek()[0] != "eol":
            raise EdlError(ln, p.peek()[2], "unexpected %r" % p.peek()[1])
        if kw[1] == "order" and order is not None:
            sysm.order = order
    if sysm.name is None:
        raise EdlError(1, 1, "missing 'system NAME'")
    for name, (base, vec, ln) in sysm.fields.items():
        for c in range(3 if vec else 1):
            if base + c not in sysm.rhs:
                raise EdlError(ln, 1, "no rhs for %r" % sysm.comp_names[base + c])
    return sysm.name, sysm.order, sysm.comp_names, [sysm.rhs[v] for v in range(sysm.nvars)]
