"""The equation-file front end of the generator: compiled equations agree
with the hand-written equation lists when evaluated on random neighbour
data, and errors carry a line and a column."""
import re

import numpy as np
import pytest

from paper_1410_1764_gb300.gen import edl, expr as E, stencil, systems


def evaluate(node, env, memo=None):
    """Numeric value of a generator DAG node; env maps symbol names."""
    memo = {} if memo is None else memo
    if node.id in memo:
        return memo[node.id]
    if isinstance(node, E.Const):
        v = float(node.value)
    elif isinstance(node, E.Sym):
        v = env(node.name)
    elif isinstance(node, E.Dif):
        v = evaluate(node.a, env, memo) - evaluate(node.b, env, memo)
    elif isinstance(node, E.Box):
        v = evaluate(node.x, env, memo)
    elif isinstance(node, E.Add):
        v = float(node.c0) + sum(float(c) * evaluate(k, env, memo) for k, c in node.terms)
    elif isinstance(node, E.Mul):
        v = 1.0
        for k, p in node.factors:
            v *= evaluate(k, env, memo) ** p
    elif isinstance(node, E.Fn):
        x = evaluate(node.arg, env, memo)
        v = np.exp(x) if node.fn == "exp" else 1.0 / x
    else:
        raise TypeError(node)
    memo[node.id] = v
    return v


def _env(seed, h=0.1):
    rng = np.random.default_rng(seed)
    vals = {}
    scal = {"ih": 1 / h, "ih2": 1 / h ** 2, "i12h": 1 / (12 * h), "i12h2": 1 / (12 * h * h),
            "i144h2": 1 / (144 * h * h)}

    def env(name):
        if name in scal:
            return scal[name]
        if name not in vals:
            vals[name] = rng.standard_normal()
        return vals[name]
    return env


WAVE1 = open(__import__("os").path.join(__import__("os").path.dirname(edl.__file__), "wave1.eqs")).read()


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_wave1_file_matches_hand_written(order):
    name, o, comps, nodes = edl.compile_system(WAVE1, order=order)
    assert (name, o, comps) == ("wave1", order, ["u", "rho", "v_x", "v_y", "v_z"])
    ref = systems.wave1(order)
    env = _env(order)
    for a, b in zip(nodes, ref):
        assert evaluate(a, env) == pytest.approx(evaluate(b, env), rel=1e-13, abs=1e-12)


def test_second_derivatives_match_stencils():
    text = "system t\nfield u\nfield w[i]\nrhs u = sum(j, dd(u, j, j)) + dd(u, x, y) - 2 * dd(u, z, 1)\n" \
           "rhs w[i] = sum(j, delta(i, j) * d(u, j)) ^ 2 / 3\n"
    _, _, comps, nodes = edl.compile_system(text)
    assert comps == ["u", "w_x", "w_y", "w_z"]
    env = _env(7)
    lap = sum(evaluate(stencil.d2(0, a), env) for a in range(3))
    want = lap + evaluate(stencil.d11(0, 0, 1), env) - 2 * evaluate(stencil.d11(0, 1, 2), env)
    assert evaluate(nodes[0], env) == pytest.approx(want, rel=1e-12)
    for a in range(3):
        assert evaluate(nodes[1 + a], env) == pytest.approx(evaluate(stencil.d1(0, a), env) ** 2 / 3, rel=1e-12)


@pytest.mark.parametrize("text,line,col,msg", [
    ("system s\nfield u\nrhs u = d(w, x)\n", 3, 11, "unknown field"),
    ("system s\nfield u\nrhs u = d(u, q)\n", 3, 14, "unknown index"),
    ("system s\nfield u\nrhs u = (u + 1\n", 3, 15, "expected )"),
    ("system s\nfield u\nfield v\nrhs u = v\n", 3, 1, "no rhs for 'v'"),
    ("system s\nfield u\nrhs u = u\nrhs u = 2 * u\n", 4, 5, "second rhs"),
    ("system s\norder 5\n", 2, 7, "even integer"),
    ("system s\nfield v[i]\nrhs v = 1\n", 3, 5, "one free index"),
    ("system s\nfield u\nrhs u = u $ 2\n", 3, 11, "unexpected character"),
    ("system s\nfield u\nrhs u = sum(x, u)\n", 3, 13, "already in use"),
    ("field u\n", 1, 1, "missing 'system NAME'"),
])
def test_errors_have_line_and_column(text, line, col, msg):
    with pytest.raises(edl.EdlError) as ei:
        edl.compile_system(text)
    assert (ei.value.line, ei.value.col) == (line, col), str(ei.value)
    assert msg in str(ei.value)
    assert re.match(r"line \d+, col \d+: ", str(ei.value))
