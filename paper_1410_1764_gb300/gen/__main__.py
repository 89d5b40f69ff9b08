"""Regenerate the CUDA point bodies under csrc/generated/.

usage: python -m paper_1410_1764_gb300.gen [--check]
  --check  exit 1 if the committed files differ from what would be written
"""
import json
import os
import re
import sys

from . import edl, emit, stencil, systems

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "generated")

HEADER = ("// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in\n"
          "// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen\n"
          "#pragma once\n\n")


def _sym_expr(name):
    m = re.match(r"f(\d+)_(-?\d+)_(-?\d+)_(-?\d+)$", name)
    if m:
        return "ld(%s, %s, %s, %s)" % m.groups(), True
    m = re.match(r"sdy_(\d+)_(-?\d+)$", name)
    if m:
        return "ld.sdy(%s, %s)" % m.groups(), True
    m = re.match(r"zq([ab])_(\d+)$", name)
    if m:
        return "ld.q%s[%s]" % m.groups(), True
    m = re.match(r"sdz_(\d+)_(-?\d+)$", name)
    if m:
        return "ld.sdz(%d, %s)" % (stencil.ZROW_VARS.index(int(m.group(1))), m.group(2)), True
    return "sc." + name, False


# Finite-difference orders compiled for the scalar-wave systems.
ORDERS = (2, 4, 6, 8)

# Output emission order: the BSSN outputs that need the Ricci tensor first
# (measured: fewest register spills of the orders tried).
# The direct body (the batched patches' kernel) starts with Gamma~^i and B^i,
# then K, At_ij, gt_ij, phi, alpha, beta^i (measured on GB300, same-GPU A/B
# of the batched schedule: 9 % faster than the Ricci-first order).
RICCI_FIRST = [8, 9, 10, 11, 12, 13, 7, 14, 15, 16, 21, 22, 23, 1, 2, 3, 4, 5, 6, 0, 17, 18, 19, 20]
EMIT_ORDER = {"bssn": [14, 15, 16, 21, 22, 23, 7, 8, 9, 10, 11, 12, 13, 1, 2, 3, 4, 5, 6, 0, 17, 18, 19, 20]}
EMIT_ORDER["bssn_x"] = RICCI_FIRST
# Emission creates nodes (scaled factors), and node numbers order the terms
# of later bodies' sums; the x/y-sharing body's instruction order, the one
# measured fastest (other orders of the same DAG: up to 3 % slower), arose
# after the direct body was emitted Ricci first.  That emission is repeated
# (and discarded) before the direct body's own, so the later bodies keep it.
NUMBERING_ORDER = {"bssn": RICCI_FIRST}
EMIT_ORDER["bssn_xy"] = RICCI_FIRST


def _varc_numbering():
    """The variable-speed right-hand side in its earlier form, with D_d s
    differenced at every point.  Emitted (and discarded) where the
    variable-speed body used to be emitted: node numbers order the terms of
    later bodies' sums, and the BSSN bodies keep the instruction order they
    were measured with.  The body that is written out (D_d s read from
    precomputed grid functions) is emitted last."""
    U, S = 0, 2
    lap = systems.E.box(systems.E.box(sum((systems._d2raw(U, a) for a in systems.R3), systems.E.const(0)))
                        * stencil.I12H2)
    adv = sum((stencil.d1(S, a) * stencil.d1(U, a) for a in systems.R3), systems.E.const(0))
    return [systems.E.box(stencil.val(1)), systems.E.box(stencil.val(S) * lap + adv)]


def _wave_xz():
    with stencil.xshare(), stencil.zqueue():
        return systems.wave()


def _bssn_xshare():
    with stencil.xshare():
        return systems.bssn()


def _bssn_xyshare():
    with stencil.xshare(), stencil.yshare():
        return systems.bssn()


def _read(name):
    with open(os.path.join(HERE, name)) as f:
        return f.read()


def _constants_header():
    """csrc/generated/gen_constants.cuh: the run-time constant table the
    generated bodies read as sc.k[i] (values exact: hexadecimal literals)."""
    ks = emit.constants()
    out = [HEADER.rstrip("\n") + "\n",
           "// Numeric constants of the generated point bodies, read at run time from\n"
           "// Scalars::k (a kernel parameter) so that every FP64 operation is an fma\n"
           "// with register or constant-bank operands.\n",
           "#define CHEMORA_NK %d\n" % len(ks)]
    for i, (_, name) in enumerate(emit.K_FIXED):
        out.append("#define CHEMORA_K_%s %d\n" % (name, i))
    out.append("#if !defined(__CUDACC_RTC__)\n")
    out.append("static const double kChemoraK[CHEMORA_NK] = {\n")
    for i, v in enumerate(ks):
        out.append("    %s,  // %d: %r\n" % (float(v).hex() if v != 0 or str(v)[0] != "-" else "-0.0", i, float(v)))
    out.append("};\n#endif\n")
    return "".join(out)


def render():
    """All generated files.  The constant table does not depend on the order
    in which bodies and outputs are emitted: a first pass collects the
    constants, the second emits with the fixed entries first, then the
    pinned ones (emit.K_PINNED), then any others in increasing order."""
    emit.reset_constants()
    _render()
    used = set(float(v) for v in emit.constants()[len(emit.K_FIXED):])
    pinned = [v for v in emit.K_PINNED if v in used]
    emit.reset_constants(pinned + sorted(used - set(pinned)))
    return _render()


def _render():
    files = {}
    counts = {}
    specs = [
        ("wave", "chemora_wave_point", systems.wave,
         "scalar wave, Eq. 1 two-variable form: u_t = rho, rho_t = Lap u"),
        ("", "chemora_varc_point", _varc_numbering, ""),
        ("bssn", "chemora_bssn_point", systems.bssn,
         "BSSN phi-form, 1+log/harmonic/frozen slicing, Gamma-driver/frozen shift, KO"),
        ("bssn_x", "chemora_bssn_x_point", _bssn_xshare,
         "BSSN as chemora_bssn_point, x-direction differences and derivative rows shared "
         "across warp lanes (32 consecutive x points per warp)"),
        ("bssn_xy", "chemora_bssn_xy_point", _bssn_xyshare,
         "BSSN as chemora_bssn_x_point, and y-direction first differences and the "
         "z-derivative rows of the yz mixed derivatives read from shared memory"),
        ("bssn_constraints", "chemora_bssn_constraints_point", systems.bssn_constraints,
         "BSSN constraints: Hamiltonian H, momentum M^i, Gamma constraint G^i"),
    ]
    for p in ORDERS:
        if p != 4:
            specs.append(("wave_o%d" % p, "chemora_wave_o%d_point" % p,
                          (lambda p=p: systems.wave_order(p)),
                          "scalar wave, two-variable form, order-%d Laplacian" % p))
        specs.append(("wave1_o%d" % p, "chemora_wave1_o%d_point" % p,
                      (lambda p=p: edl.compile_system(_read("wave1.eqs"), order=p)[3]),
                      "scalar wave, first-order form of Eq. 1 (u, rho, v_i), order-%d D, "
                      "from gen/wave1.eqs" % p))
    # last, so that the constant table of the earlier bodies keeps its order
    specs.append(("wave_xz", "chemora_wave_xz_point", _wave_xz,
                  "scalar wave as chemora_wave_point, x-direction differences shared across warp "
                  "lanes and the z-direction second difference from a register queue of z first "
                  "differences kept by a thread marching along z"))
    specs.append(("wave_varc", "chemora_varc_point", systems.wave_varc,
                  "variable-speed wave: u_t = rho, rho_t = s Lap u + G . grad u, with s = c^2 "
                  "and G = grad s read from grid functions 2 and 3-5"))
    for key, fname, build, comment in specs:
        outs = build()
        nout = len(outs)
        if not key:  # numbering pass only
            emit.emit_function(fname, list(enumerate(outs)), _sym_expr, nout, comment)
            continue
        if key in NUMBERING_ORDER:
            emit.emit_function(fname, [(v, outs[v]) for v in NUMBERING_ORDER[key]], _sym_expr, nout, comment)
        order = EMIT_ORDER.get(key, list(range(nout)))
        src, L = emit.emit_function(fname, [(v, outs[v]) for v in order],
                                    _sym_expr, nout, comment)
        files["gen_%s.cuh" % key] = HEADER + src
        counts[key] = {"fp64_instructions": L.dp_ops, "flops": L.flops, "loads": len(L.loads),
                       "exp": L.special["exp"], "rcp": L.special["rcp"], "nvars": nout}
    files["opcounts.json"] = json.dumps(counts, indent=1, sort_keys=True) + "\n"
    inc = [HEADER.rstrip("\n") + "\n", "// per interior point and RHS evaluation\n"]
    for key, tag in (("wave", "WAVE"), ("wave_varc", "VARC"), ("bssn", "BSSN"), ("wave1_o4", "WAVE1"),
                     ("bssn_x", "BSSN_X"), ("bssn_xy", "BSSN_XY"), ("wave_xz", "WAVE_XZ")):
        inc.append("#define CHEMORA_OPS_%s_INSTR %d\n" % (tag, counts[key]["fp64_instructions"]))
        inc.append("#define CHEMORA_OPS_%s_FLOPS %d\n" % (tag, counts[key]["flops"]))
    files["opcounts.inc"] = "".join(inc)
    files["gen_constants.cuh"] = _constants_header()
    return files


def main(argv):
    check = "--check" in argv
    files = render()
    os.makedirs(OUT, exist_ok=True)
    stale = []
    for name, text in files.items():
        path = os.path.join(OUT, name)
        old = open(path).read() if os.path.exists(path) else None
        if old != text:
            stale.append(name)
            if not check:
                with open(path, "w") as f:
                    f.write(text)
    if check and stale:
        print("stale generated files: %s" % ", ".join(stale))
        return 1
    print(json.dumps(json.loads(files["opcounts.json"])))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
