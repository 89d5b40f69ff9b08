"""The generator's point bodies, compiled for the host with g++ (no GPU): the
direct BSSN body, the BSSN constraints, the scalar-wave bodies of every
order, the first-order form and the variable-speed wave, each evaluated at
every interior point of a small grid and compared with the oracle.  A guard
on the generator itself (CSE, flattened chains, absorbed constants, the
constant table and the fma forms) independent of the CUDA kernels; the
lane- and shared-memory-sharing bodies need a warp evaluated in lockstep
(test_generated_warp_host.py) and run on the GPU in the parity tests."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1410_1764_gb300 import synth
from helpers import scaled_err

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_1764_gb300", "csrc")

HARNESS = r"""
#include <cmath>
#include <cstdint>
#define __device__
#define __host__
#define __forceinline__ inline
using std::fma;
using std::exp;
#include "generated/gen_constants.cuh"
#include "generated/%(header)s"

struct SC {
  double i12h, i12h2, i144h2, ko_scale, eta;
  int slicing, shift;
  double ih, ih2;
  int order;
  double k[CHEMORA_NK];
};
struct LD {
  const double* p;
  const double* q;
  int64_t sy, sz, sv;
  double operator()(int v, int dx, int dy, int dz) const {
    const int64_t o = dx + dy * sy + dz * sz;
    return v < %(nv)d ? p[v * sv + o] : q[(v - %(nv)d) * sv + o];  // coefficient fields
  }
};
struct OUT {
  double* o;
  int64_t c, sv;
  void operator()(int v, double x) const { o[v * sv + c] = x; }
};

extern "C" void run(const double* st, const double* coef, double* out, int nx, int ny, int nz, int g,
                    double h, double eps, double eta, int slicing, int shift, int order) {
  SC sc;
  sc.i12h = 1.0 / (12.0 * h);
  sc.i12h2 = 1.0 / (12.0 * h * h);
  sc.i144h2 = 1.0 / (144.0 * h * h);
  sc.ko_scale = eps / (64.0 * h);
  sc.eta = eta;
  sc.slicing = slicing;
  sc.shift = shift;
  sc.ih = 1.0 / h;
  sc.ih2 = 1.0 / (h * h);
  sc.order = order;
  for (int i = 0; i < CHEMORA_NK; ++i) sc.k[i] = kChemoraK[i];
  const int64_t px = nx + 2 * g, py = ny + 2 * g, sy = px, sz = px * py, sv = sz * (nz + 2 * g);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int64_t c = (int64_t)(k + g) * sz + (int64_t)(j + g) * sy + (i + g);
        LD ld{st + c, coef ? coef + c : nullptr, sy, sz, sv};
        OUT o{out, c, sv};
        %(fn)s(ld, sc, o);
      }
}
"""


def _gxx():
    return shutil.which("g++") or shutil.which("c++")


_LIBS = {}


def _body(tmp_root, header, fn, nv):
    key = (header, fn)
    if key in _LIBS:
        return _LIBS[key]
    cxx = _gxx()
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = os.path.join(str(tmp_root), fn)
    os.makedirs(d, exist_ok=True)
    src = os.path.join(d, "h.cpp")
    with open(src, "w") as f:
        f.write(HARNESS % {"header": header, "fn": fn, "nv": nv})
    so = os.path.join(d, "h.so")
    r = subprocess.run([cxx, "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC, src,
                        "-o", so], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    lib = ctypes.CDLL(so)
    D = ctypes.POINTER(ctypes.c_double)
    lib.run.argtypes = [D, D, D] + [ctypes.c_int] * 4 + [ctypes.c_double] * 3 + [ctypes.c_int] * 3
    _LIBS[key] = lib
    return lib


def _run(lib, st, g, h, coef=None, nout=None, eps=0.1, eta=2.0, slicing=0, shift=0, order=4):
    nv = st.shape[0] if nout is None else nout
    out = np.zeros((nv,) + st.shape[1:])
    pz, py, px = st.shape[1:]
    D = ctypes.POINTER(ctypes.c_double)
    cp = coef.ctypes.data_as(D) if coef is not None else D()
    lib.run(st.ctypes.data_as(D), cp, out.ctypes.data_as(D), px - 2 * g, py - 2 * g, pz - 2 * g, g, h,
            eps, eta, slicing, shift, order)
    return out


@pytest.fixture(scope="module")
def tmp_root(tmp_path_factory):
    return tmp_path_factory.mktemp("genhost")


def _bssn_state(dims, amp, seed, g=3):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    return synth.pad(synth.BSSN_FLAT[:, None, None, None] + amp * rng.standard_normal((24, nz, ny, nx)), g)


@pytest.mark.parametrize("slicing,shift", [(0, 0), (1, 1), (2, 0)])
def test_direct_bssn_body(orc, tmp_root, slicing, shift):
    dims, g, h = (9, 8, 7), 3, 1.0 / 9
    st = _bssn_state(dims, 3e-2, seed=21)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h, orc.Params(0.1, 2.0, slicing, shift))
    lib = _body(tmp_root, "gen_bssn.cuh", "chemora_bssn_point", 24)
    got = _run(lib, st, g, h, slicing=slicing, shift=shift)
    assert scaled_err(got, want, g) <= 1e-12


def test_direct_bssn_body_noise(orc, tmp_root):
    """Flat space with 1e-10 noise: the conditioning of the bench workload."""
    dims, g, h = (10, 9, 8), 3, 1.0 / 10
    st = _bssn_state(dims, 1e-10, seed=22)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h)
    got = _run(_body(tmp_root, "gen_bssn.cuh", "chemora_bssn_point", 24), st, g, h)
    assert scaled_err(got, want, g) <= 1e-12


def test_constraints_body(orc, tmp_root):
    dims, g, h = (9, 8, 7), 3, 1.0 / 9
    st = _bssn_state(dims, 3e-2, seed=23)
    orc.fill_ghosts(st, g)
    want = orc.bssn_constraints(st, g, h)
    lib = _body(tmp_root, "gen_bssn_constraints.cuh", "chemora_bssn_constraints_point", 24)
    got = _run(lib, st, g, h, nout=7)
    assert scaled_err(got, want, g) <= 1e-12


@pytest.mark.parametrize("order,header,fn", [(4, "gen_wave.cuh", "chemora_wave_point"),
                                             (2, "gen_wave_o2.cuh", "chemora_wave_o2_point"),
                                             (6, "gen_wave_o6.cuh", "chemora_wave_o6_point"),
                                             (8, "gen_wave_o8.cuh", "chemora_wave_o8_point")])
def test_wave_bodies(orc, tmp_root, order, header, fn):
    dims, g = (11, 9, 8), max(2, order // 2)
    h = 1.0 / 11
    st = synth.pad(np.random.default_rng(order).standard_normal((2, dims[2], dims[1], dims[0])), g)
    orc.fill_ghosts(st, g)
    want = orc.rhs(orc.WAVE, st, g, h, params=orc.default_params(order))
    got = _run(_body(tmp_root, header, fn, 2), st, g, h, order=order)
    assert scaled_err(got, want, g) <= 1e-12


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_first_order_bodies(orc, tmp_root, order):
    dims, g = (10, 9, 7), max(2, order // 2)
    h = 1.0 / 10
    st = synth.pad(np.random.default_rng(10 + order).standard_normal((5, dims[2], dims[1], dims[0])), g)
    orc.fill_ghosts(st, g)
    want = orc.wave1_rhs(st, g, h, order)
    got = _run(_body(tmp_root, "gen_wave1_o%d.cuh" % order, "chemora_wave1_o%d_point" % order, 5),
               st, g, h, order=order)
    assert scaled_err(got, want, g) <= 1e-12


def test_variable_speed_body(orc, tmp_root):
    dims, g, h = (10, 9, 8), 2, 1.0 / 10
    rng = np.random.default_rng(31)
    st = synth.pad(rng.standard_normal((2, dims[2], dims[1], dims[0])), g)
    orc.fill_ghosts(st, g)
    c = synth.pad(1.0 + 0.2 * rng.uniform(-1, 1, (dims[2], dims[1], dims[0])), g)[0]
    s = (c * c).copy()
    orc.fill_ghosts(s, g)
    want = orc.varc_rhs(st, s, g, h)
    # the body reads s and its centred first derivatives (taken once per speed)
    coef = np.stack([s] + [orc.deriv(s, g, h, 0, a) for a in range(3)])
    got = _run(_body(tmp_root, "gen_wave_varc.cuh", "chemora_varc_point", 2), st, g, h, coef=coef)
    assert scaled_err(got, want, g) <= 1e-12
