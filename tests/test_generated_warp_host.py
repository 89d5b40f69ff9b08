"""The lane-sharing point bodies (BSSN x/y-sharing, the bench's body, and the
x-lane / z-queue scalar wave) run on the host: each statement of the
generated straight-line body is evaluated for the 32 lanes of a warp before
the next (temporaries become arrays over lanes), so a warp shuffle reads the
other lanes' values exactly as on the GPU.  The harness supplies what the
kernels supply: neighbour loads, the halo lanes' x differences and derivative
rows, the shared-memory y differences and z-derivative rows of the x/y
prologue, and the z-difference queue; outputs are compared with the oracle.
No GPU: a CPU check of the generated code the GPU kernels compile."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from paper_1410_1764_gb300 import synth
from helpers import scaled_err

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEN = os.path.join(ROOT, "paper_1410_1764_gb300", "csrc", "generated")

DEF = re.compile(r"^  const double (\w+) = (.*);$")
OUT = re.compile(r"^  out\((\d+), (.*)\);$")
SHFL = re.compile(r"chemora_xshfl\((\w+), (\w+), (-?\d+), (\d+)\)")
IDENT = re.compile(r"\b(t\d+|v_\w+)\b")


def _lanewise(header, fn):
    """C++ of the body with every temporary an array over the 32 lanes."""
    body, inside = [], False
    for line in open(os.path.join(GEN, header)):
        line = line.rstrip("\n")
        if line.startswith("__device__ __forceinline__ void %s(" % fn):
            inside = True
            continue
        if not inside:
            continue
        if line == "}":
            break
        m, o = DEF.match(line), OUT.match(line)
        expr = m.group(2) if m else o.group(2)
        calls = []

        def hold(mo):
            calls.append("xshfl(%s, %s, %s, %s, l)" % mo.groups())
            return "@%d@" % (len(calls) - 1)
        expr = SHFL.sub(hold, expr)
        expr = IDENT.sub(lambda mo: "%s[l]" % mo.group(1), expr)
        expr = re.sub(r"@(\d+)@", lambda mo: calls[int(mo.group(1))], expr)
        expr = expr.replace("ld(", "ld.at(l, ").replace("ld.ext_dx(", "ld.ext_dx(l, ")
        expr = expr.replace("ld.ext_d1y(", "ld.ext_d1y(l, ").replace("ld.ext_d1z(", "ld.ext_d1z(l, ")
        expr = expr.replace("ld.sdy(", "ld.sdy(l, ").replace("ld.sdz(", "ld.sdz(l, ")
        expr = re.sub(r"ld\.q([ab])\[(\d+)\]", r"ld.q\1(l, \2)", expr)
        if m:
            body.append("  double %s[32];\n  for (int l = 0; l < 32; ++l) %s[l] = %s;" % (m.group(1), m.group(1), expr))
        else:
            body.append("  for (int l = 0; l < 32; ++l) out(l, %s, %s);" % (o.group(1), expr))
    assert inside and body
    return "\n".join(body)


HARNESS = r"""
#include <cmath>
#include <cstdint>
#define __device__
#define __host__
#define __forceinline__ inline
using std::fma;
using std::exp;
#include "generated/gen_constants.cuh"

struct SC {
  double i12h, i12h2, i144h2, ko_scale, eta;
  int slicing, shift;
  double ih, ih2;
  int order;
  double k[CHEMORA_NK];
};

// one warp: lanes l = 0..31 at x = x0 + l of row y, plane z (interior coordinates)
struct Warp {
  const double* f;
  int64_t sy, sz, sv;
  int g, x0, y, z;
  const int zrow[11] = {0, 1, 2, 3, 4, 5, 6, 17, 18, 19, 20};
  double val(int v, int x, int yy, int zz) const {
    return f[v * sv + (int64_t)(zz + g) * sz + (int64_t)(yy + g) * sy + (x + g)];
  }
  double at(int l, int v, int dx, int dy, int dz) const { return val(v, x0 + l + dx, y + dy, z + dz); }
  double dxd(int v, int x) const { return fma(val(v, x, y, z), -1.0, val(v, x + 1, y, z)); }
  double d1row(int v, int x, int yy, int zz, int ay) const {  // 8 (f+1 - f-1) - (f+2 - f-2) along y or z
    const int a1 = ay ? 1 : 0, b1 = ay ? 0 : 1;
    const double p1 = val(v, x, yy + a1, zz + b1) - val(v, x, yy - a1, zz - b1);
    const double p2 = val(v, x, yy + 2 * a1, zz + 2 * b1) - val(v, x, yy - 2 * a1, zz - 2 * b1);
    return fma(8.0, p1, -p2);
  }
  // halo lanes of the x-sharing loaders (XLoader offsets)
  double ext_dx(int l, int v, double) const {
    const int xo = l < 3 ? -3 : (l < 5 ? 29 : 0);
    return dxd(v, x0 + l + xo);
  }
  double ext_d1y(int l, int v, double, double) const {
    const int xo = l < 2 ? -2 : (l < 4 ? 30 : 0);
    return d1row(v, x0 + l + xo, y, z, 1);
  }
  double ext_d1z(int l, int v, double, double) const {
    const int xo = l < 2 ? -2 : (l < 4 ? 30 : 0);
    return d1row(v, x0 + l + xo, y, z, 0);
  }
  // the x/y prologue's shared memory: y differences and z-derivative rows
  double sdy(int l, int v, int m) const {
    return val(v, x0 + l, y + m + 1, z) - val(v, x0 + l, y + m, z);
  }
  double sdz(int l, int vi, int m) const { return d1row(zrow[vi], x0 + l, y + m, z, 0); }
  // the z queue of the x/z wave body: e_m = u(z+m+1) - u(z+m)
  double e(int l, int m) const { return val(0, x0 + l, y, z + m + 1) - val(0, x0 + l, y, z + m); }
  double qa(int l, int) const { return e(l, 0) - e(l, -1); }
  double qb(int l, int) const { return e(l, 1) - e(l, -2); }
};

static double xshfl(const double* own, const double* ext, int m, int w, int l) {
  const int src = l + m;
  if (src >= 0 && src < 32) return own[src];
  return ext[src < 0 ? src + w : src - 32 + w];
}

struct Out {
  double* o;
  const Warp& W;
  void operator()(int l, int v, double x) const {
    o[v * W.sv + (int64_t)(W.z + W.g) * W.sz + (int64_t)(W.y + W.g) * W.sy + (W.x0 + l + W.g)] = x;
  }
};

static void body(const Warp& ld, const SC& sc, const Out& out) {
%(body)s
}

extern "C" void run(const double* st, double* o, int nx, int ny, int nz, int g, double h) {
  SC sc;
  sc.i12h = 1.0 / (12.0 * h);
  sc.i12h2 = 1.0 / (12.0 * h * h);
  sc.i144h2 = 1.0 / (144.0 * h * h);
  sc.ko_scale = 0.1 / (64.0 * h);
  sc.eta = 2.0;
  sc.slicing = 0;
  sc.shift = 0;
  sc.ih = 1.0 / h;
  sc.ih2 = 1.0 / (h * h);
  sc.order = 4;
  for (int i = 0; i < CHEMORA_NK; ++i) sc.k[i] = kChemoraK[i];
  const int64_t px = nx + 2 * g, py = ny + 2 * g;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x0 = 0; x0 < nx; x0 += 32) {
        Warp W{st, px, px * py, px * py * (nz + 2 * g), g, x0, y, z};
        Out O{o, W};
        body(W, sc, O);
      }
}
"""


def _build(tmp, header, fn):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = os.path.join(str(tmp), fn + ".cpp")
    with open(src, "w") as f:
        f.write(HARNESS % {"body": _lanewise(header, fn)})
    so = os.path.join(str(tmp), fn + ".so")
    r = subprocess.run([cxx, "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I",
                        os.path.dirname(GEN), src, "-o", so], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    lib = ctypes.CDLL(so)
    D = ctypes.POINTER(ctypes.c_double)
    lib.run.argtypes = [D, D] + [ctypes.c_int] * 4 + [ctypes.c_double]
    return lib


def _run(lib, st, g, h):
    out = np.zeros_like(st)
    pz, py, px = st.shape[1:]
    D = ctypes.POINTER(ctypes.c_double)
    lib.run(st.ctypes.data_as(D), out.ctypes.data_as(D), px - 2 * g, py - 2 * g, pz - 2 * g, g, h)
    return out


@pytest.mark.parametrize("amp", [3e-2, 1e-10])
def test_xy_sharing_bssn_body(orc, tmp_path, amp):
    """The bench's body (x lanes, y differences and z rows from the
    prologue) on two warps per row, 24 variables, against the oracle."""
    dims, g, h = (64, 6, 5), 3, 1.0 / 64
    rng = np.random.default_rng(41)
    st = synth.pad(synth.BSSN_FLAT[:, None, None, None] + amp * rng.standard_normal((24, dims[2], dims[1], dims[0])), g)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h)
    got = _run(_build(tmp_path, "gen_bssn_xy.cuh", "chemora_bssn_xy_point"), st, g, h)
    assert scaled_err(got, want, g) <= 1e-12


def test_x_sharing_bssn_body(orc, tmp_path):
    dims, g, h = (32, 5, 4), 3, 1.0 / 32
    rng = np.random.default_rng(42)
    st = synth.pad(synth.BSSN_FLAT[:, None, None, None] + 3e-2 * rng.standard_normal((24, dims[2], dims[1], dims[0])), g)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h)
    got = _run(_build(tmp_path, "gen_bssn_x.cuh", "chemora_bssn_x_point"), st, g, h)
    assert scaled_err(got, want, g) <= 1e-12


def test_xz_wave_body(orc, tmp_path):
    dims, g, h = (64, 7, 9), 2, 1.0 / 64
    st = synth.pad(np.random.default_rng(43).standard_normal((2, dims[2], dims[1], dims[0])), g)
    orc.fill_ghosts(st, g)
    want = orc.wave_rhs(st, g, h)
    got = _run(_build(tmp_path, "gen_wave_xz.cuh", "chemora_wave_xz_point"), st, g, h)
    assert scaled_err(got, want, g) <= 1e-12
