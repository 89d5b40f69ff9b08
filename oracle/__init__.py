"""FP64 CPU oracle for the Chemora hot path (arXiv 1410.1764).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The CUDA library never imports, links or
calls anything here, and this package imports nothing from the CUDA side.

Arrays are numpy float64, C-contiguous, shaped (nvars, nz+2g, ny+2g, nx+2g)
(x fastest) with ghost zones included; a single grid function may also be
passed as (nz+2g, ny+2g, nx+2g).

What is computed (each routine cites the passage it follows):
  fill_ghosts        periodic ghost zones (Sec. 2, driver ghost zones)
  deriv              4th-order centred D1, D2, mixed D2 and the 5th-order
                     Kreiss-Oliger operator (Sec. 3.2.2)
  wave_rhs           Eq. 1 in two-variable form u_t = rho, rho_t = Lap u
  varc_rhs           u_t = rho, rho_t = s Lap u + grad s . grad u, s = c^2
  bssn_rhs           Einstein equations in BSSN phi-form with 1+log slicing,
                     Gamma-driver shift and KO dissipation (Sec. 3.4, Sec. 5:
                     the paper names the system but prints no formulas; the
                     standard phi-form is written out in oracle.c)
  bssn_constraints   Hamiltonian, momentum and Gamma constraints
  rk4                classic RK4 method of lines (Sec. 2, time integrator)
  varc_tlm_rk4       tangent-linear RK4 of the variable-speed wave
  varc_adj_rhs       exact discrete transpose of the variable-speed RHS
  varc_vjp           stage-wise reverse RK4 with checkpoint recomputation
  varc_adjoint       misfit loss at receivers and its gradient
  amr_*              two-level refinement of the scalar wave with one box,
                     Berger-Oliger subcycling (Sec. 4, Carpet's AMR)
  amrn_*             the same with several boxes, for the wave or BSSN
"""
import ctypes
import os

import numpy as np

from . import build as _build

WAVE, WAVE_VARC, BSSN, WAVE1 = 1, 2, 3, 4
NVARS = {WAVE: 2, WAVE_VARC: 2, BSSN: 24, WAVE1: 5}


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("g", ctypes.c_int), ("h", ctypes.c_double)]


class Params(ctypes.Structure):
    """BSSN parameters: KO strength, Gamma-driver eta, slicing
    (0 = 1+log, 1 = harmonic, 2 = frozen lapse), shift (0 = Gamma-driver,
    1 = frozen shift and B); finite-difference order of the wave systems
    (0 = 4)."""
    _fields_ = [("eps_diss", ctypes.c_double), ("eta", ctypes.c_double),
                ("slicing", ctypes.c_int), ("shift", ctypes.c_int), ("order", ctypes.c_int)]


def default_params(order=0):
    return Params(0.1, 2.0, 0, 0, order)


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(ctypes.c_double)
        G = ctypes.POINTER(_Grid)
        L.orc_fill_ghosts.argtypes = [P, ctypes.c_int, G]
        L.orc_deriv.argtypes = [P, P, G, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_wave_rhs.argtypes = [P, P, G]
        L.orc_varc_rhs.argtypes = [P, P, P, G]
        L.orc_varc_tlm_rhs.argtypes = [P, P, P, P, P, G]
        L.orc_varc_adj_rhs.argtypes = [P, P, P, P, P, G]
        L.orc_bssn_rhs.argtypes = [P, P, G, ctypes.POINTER(Params)]
        L.orc_bssn_constraints.argtypes = [P, P, G]
        L.orc_rk4.argtypes = [ctypes.c_int, P, P, G, ctypes.POINTER(Params),
                              ctypes.c_double, ctypes.c_int]
        L.orc_rk4.restype = ctypes.c_int
        L.orc_varc_tlm_rk4.argtypes = [P, P, P, P, G, ctypes.c_double, ctypes.c_int]
        L.orc_varc_tlm_rk4.restype = ctypes.c_int
        L.orc_varc_vjp.argtypes = [P, P, G, ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P]
        L.orc_varc_vjp.restype = ctypes.c_int
        L.orc_varc_adjoint.argtypes = [P, P, G, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.c_int, P, P, P, P]
        L.orc_varc_adjoint.restype = ctypes.c_int
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc_set_num_threads.restype = None
        L.orc_fd_weights.argtypes = [ctypes.c_int, P, P]
        L.orc_fd_weights.restype = ctypes.c_int
        L.orc_deriv_order.argtypes = [P, P, G, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_deriv_order.restype = ctypes.c_int
        L.orc_wave_rhs_order.argtypes = [P, P, G, ctypes.c_int]
        L.orc_wave_rhs_order.restype = ctypes.c_int
        L.orc_wave1_rhs.argtypes = [P, P, G, ctypes.c_int]
        L.orc_wave1_rhs.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def grid(nx, ny, nz, g, h):
    return _Grid(nx, ny, nz, g, h)


def grid_of(a, g, h):
    """Grid description of a padded array (..., nz+2g, ny+2g, nx+2g)."""
    pz, py, px = a.shape[-3:]
    return _Grid(px - 2 * g, py - 2 * g, pz - 2 * g, g, h)


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    """Threads of the following calls (timing only: results do not depend
    on the thread count)."""
    lib().orc_set_num_threads(int(n))


def fill_ghosts(f, g):
    """Periodic ghost zones, in place (Sec. 2, driver ghost zones)."""
    G = grid_of(f, g, 1.0)
    nv = 1 if f.ndim == 3 else f.shape[0]
    lib().orc_fill_ghosts(_p(f), nv, ctypes.byref(G))
    return f


def deriv(f, g, h, kind, a, b=0):
    """Derivative of one grid function on the interior (Sec. 3.2.2).
    kind 0: D1 along a; 1: pure D2 along a; 2: mixed D_a D_b; 3: KO along a
    with eps = 1.  Ghost entries of the result are zero."""
    G = grid_of(f, g, h)
    out = np.zeros_like(f)
    lib().orc_deriv(_p(f), _p(out), ctypes.byref(G), kind, a, b)
    return out


def wave_rhs(st, g, h):
    out = np.zeros_like(st)
    lib().orc_wave_rhs(_p(st), _p(out), ctypes.byref(grid_of(st, g, h)))
    return out


def varc_rhs(st, s, g, h):
    out = np.zeros_like(st)
    lib().orc_varc_rhs(_p(st), _p(s), _p(out), ctypes.byref(grid_of(st, g, h)))
    return out


def varc_tlm_rhs(st, s, dst, ds, g, h):
    out = np.zeros_like(st)
    lib().orc_varc_tlm_rhs(_p(st), _p(s), _p(dst), _p(ds), _p(out),
                           ctypes.byref(grid_of(st, g, h)))
    return out


def varc_adj_rhs(st, s, kb, g, h):
    """(yhat, sbar) with yhat = J^T kb and sbar the s-cotangent."""
    yhat = np.zeros_like(st)
    sbar = np.zeros_like(s)
    lib().orc_varc_adj_rhs(_p(st), _p(s), _p(kb), _p(yhat), _p(sbar),
                           ctypes.byref(grid_of(st, g, h)))
    return yhat, sbar


def bssn_rhs(st, g, h, params=None):
    params = params or default_params()
    out = np.zeros_like(st)
    lib().orc_bssn_rhs(_p(st), _p(out), ctypes.byref(grid_of(st, g, h)), ctypes.byref(params))
    return out


def bssn_constraints(st, g, h):
    out = np.zeros((7,) + st.shape[1:])
    lib().orc_bssn_constraints(_p(st), _p(out), ctypes.byref(grid_of(st, g, h)))
    return out


def fd_weights(order):
    """Central weights (a_k, b_k), k = 1..order/2, of the order-p first and
    second derivatives on (f_k - f_-k) and (f_k - f_0) + (f_-k - f_0)."""
    a = np.zeros(8)
    b = np.zeros(8)
    if lib().orc_fd_weights(order, _p(a), _p(b)) != 0:
        raise ValueError("order must be even, 2..16")
    return a[:order // 2], b[:order // 2]


def deriv_order(f, g, h, order, kind, a):
    """Order-p derivative (kind 0: D1, 1: D2) along axis a on the interior."""
    out = np.zeros_like(f)
    if lib().orc_deriv_order(_p(f), _p(out), ctypes.byref(grid_of(f, g, h)), order, kind, a) != 0:
        raise ValueError("bad order or too few ghosts")
    return out


def wave_rhs_order(st, g, h, order):
    out = np.zeros_like(st)
    if lib().orc_wave_rhs_order(_p(st), _p(out), ctypes.byref(grid_of(st, g, h)), order) != 0:
        raise ValueError("bad order or too few ghosts")
    return out


def wave1_rhs(st, g, h, order=4):
    """First-order form of Eq. 1: (u, rho, v_x, v_y, v_z)."""
    out = np.zeros_like(st)
    if lib().orc_wave1_rhs(_p(st), _p(out), ctypes.byref(grid_of(st, g, h)), order) != 0:
        raise ValueError("bad order or too few ghosts")
    return out


def rhs(kind, st, g, h, s=None, params=None):
    if kind == WAVE1:
        return wave1_rhs(st, g, h, (params.order if params is not None and params.order else 4))
    if kind == WAVE and params is not None and params.order not in (0, 4):
        return wave_rhs_order(st, g, h, params.order)
    if kind == WAVE:
        return wave_rhs(st, g, h)
    if kind == WAVE_VARC:
        return varc_rhs(st, s, g, h)
    return bssn_rhs(st, g, h, params)


def rk4(kind, y, g, h, dt, nsteps, s=None, params=None):
    """nsteps classic RK4 steps on a copy of y; returns the new state with
    periodic ghosts filled."""
    y = np.ascontiguousarray(y, dtype=np.float64).copy()
    params = params or default_params()
    sp = _p(s) if s is not None else ctypes.POINTER(ctypes.c_double)()
    rc = lib().orc_rk4(kind, _p(y), sp, ctypes.byref(grid_of(y, g, h)), ctypes.byref(params),
                       dt, nsteps)
    if rc != 0:
        raise RuntimeError("orc_rk4 failed: %d" % rc)
    return y


def varc_tlm_rk4(y, dy, s, ds, g, h, dt, nsteps):
    y = y.copy()
    dy = dy.copy()
    rc = lib().orc_varc_tlm_rk4(_p(y), _p(dy), _p(s), _p(ds), ctypes.byref(grid_of(y, g, h)),
                                dt, nsteps)
    if rc != 0:
        raise RuntimeError("orc_varc_tlm_rk4 failed: %d" % rc)
    return y, dy


def varc_adjoint(y0, s, g, h, dt, nsteps, ckpt_every, recv, data):
    """(loss, grad_y0, grad_s) of J = 1/2 sum (u_N(recv) - data)^2.
    recv: padded linear indices into one grid function."""
    recv = np.ascontiguousarray(recv, dtype=np.int64)
    data = np.ascontiguousarray(data, dtype=np.float64)
    gy = np.zeros_like(y0)
    gs = np.zeros_like(s)
    loss = np.zeros(1)
    rc = lib().orc_varc_adjoint(_p(y0), _p(s), ctypes.byref(grid_of(y0, g, h)), dt, nsteps,
                                ckpt_every, recv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                len(recv), _p(data), _p(loss), _p(gy), _p(gs))
    if rc != 0:
        raise RuntimeError("orc_varc_adjoint failed: %d" % rc)
    return float(loss[0]), gy, gs


def varc_vjp(y0, s, g, h, dt, nsteps, ckpt_every, ybar_N):
    """Cotangents (ybar_0, sbar) of the initial state and of s for the final
    cotangent ybar_N of the nsteps-step RK4 map."""
    ybar = np.ascontiguousarray(ybar_N, dtype=np.float64).copy()
    sbar = np.zeros_like(s)
    rc = lib().orc_varc_vjp(_p(y0), _p(s), ctypes.byref(grid_of(y0, g, h)), dt, nsteps,
                            ckpt_every, _p(ybar), _p(sbar))
    if rc != 0:
        raise RuntimeError("orc_varc_vjp failed: %d" % rc)
    return ybar, sbar


class _Amr(ctypes.Structure):
    _fields_ = [("nc", ctypes.c_int), ("gc", ctypes.c_int), ("lo", ctypes.c_int * 3),
                ("hi", ctypes.c_int * 3), ("gf", ctypes.c_int), ("H", ctypes.c_double)]


def amr(nc, lo, hi, H, gc=2, gf=8):
    """Two-level configuration: periodic coarse grid of nc^3 points, fine box
    of coarse points [lo, hi) refined by 2."""
    return _Amr(nc, gc, (ctypes.c_int * 3)(*lo), (ctypes.c_int * 3)(*hi), gf, H)


def _amr_lib():
    L = lib()
    if not getattr(L, "_amr_ready", False):
        PP = ctypes.POINTER(ctypes.POINTER(ctypes.c_double))
        P = ctypes.POINTER(ctypes.c_double)
        A = ctypes.POINTER(_Amr)
        L.orc_amr_prolong.argtypes = [A, ctypes.c_int, PP, P, ctypes.c_int, P]
        L.orc_amr_restrict.argtypes = [A, ctypes.c_int, P, P]
        L.orc_amr_step.argtypes = [A, P, P, ctypes.c_double, ctypes.c_int]
        L.orc_amr_step.restype = ctypes.c_int
        L._amr_ready = True
    return L


def amr_prolong(cfg, levels, tw, fine):
    """Fill the ghosts of `fine` (nv, ...) from coarse time levels (each
    (nv, ...)) with time weights tw, in place."""
    nv = fine.shape[0]
    arr = (ctypes.POINTER(ctypes.c_double) * len(levels))(*[_p(c) for c in levels])
    w = np.ascontiguousarray(tw, dtype=np.float64)
    _amr_lib().orc_amr_prolong(ctypes.byref(cfg), nv, arr, _p(w), len(levels), _p(fine))
    return fine


def amr_restrict(cfg, fine, coarse):
    _amr_lib().orc_amr_restrict(ctypes.byref(cfg), fine.shape[0], _p(fine), _p(coarse))
    return coarse


def amr_step(cfg, coarse, fine, dt, nsteps):
    """nsteps Berger-Oliger steps (scalar wave); arrays updated in place."""
    rc = _amr_lib().orc_amr_step(ctypes.byref(cfg), _p(coarse), _p(fine), dt, nsteps)
    if rc != 0:
        raise RuntimeError("orc_amr_step failed: %d" % rc)


class _AmrN(ctypes.Structure):
    _fields_ = [("nc", ctypes.c_int * 3), ("gc", ctypes.c_int), ("nbox", ctypes.c_int),
                ("lo", ctypes.POINTER(ctypes.c_int)), ("hi", ctypes.POINTER(ctypes.c_int)),
                ("gf", ctypes.c_int), ("H", ctypes.c_double)]


def amrn(nc, boxes, H, gc, gf):
    """Two-level configuration with several boxes: periodic coarse grid of
    nc = (nx, ny, nz) points (spacing H, ghosts gc); each box (lo, hi)
    refines the coarse points [lo, hi) per axis by 2 (buffer width gf)."""
    nb = len(boxes)
    lo = (ctypes.c_int * (3 * nb))(*[int(v) for b in boxes for v in b[0]])
    hi = (ctypes.c_int * (3 * nb))(*[int(v) for b in boxes for v in b[1]])
    cfg = _AmrN((ctypes.c_int * 3)(*[int(v) for v in nc]), gc, nb,
                ctypes.cast(lo, ctypes.POINTER(ctypes.c_int)), ctypes.cast(hi, ctypes.POINTER(ctypes.c_int)),
                gf, H)
    cfg._keep = (lo, hi)
    cfg.boxes = [(tuple(b[0]), tuple(b[1])) for b in boxes]
    return cfg


def _amrn_lib():
    L = lib()
    if not getattr(L, "_amrn_ready", False):
        PP = ctypes.POINTER(ctypes.POINTER(ctypes.c_double))
        P = ctypes.POINTER(ctypes.c_double)
        A = ctypes.POINTER(_AmrN)
        L.orc_amrn_prolong.argtypes = [A, ctypes.c_int, ctypes.c_int, PP, P, ctypes.c_int, P]
        L.orc_amrn_prolong.restype = ctypes.c_int
        L.orc_amrn_restrict.argtypes = [A, ctypes.c_int, ctypes.c_int, P, P]
        L.orc_amrn_restrict.restype = ctypes.c_int
        L.orc_amrn_step.argtypes = [A, ctypes.c_int, ctypes.POINTER(Params), P, PP, ctypes.c_double,
                                    ctypes.c_int]
        L.orc_amrn_step.restype = ctypes.c_int
        L._amrn_ready = True
    return L


def amrn_prolong(cfg, b, levels, tw, fine):
    """Fill the buffer of box b's state `fine` (nv, ...) from coarse time
    levels with time weights tw, in place."""
    nv = fine.shape[0]
    arr = (ctypes.POINTER(ctypes.c_double) * len(levels))(*[_p(c) for c in levels])
    w = np.ascontiguousarray(tw, dtype=np.float64)
    if _amrn_lib().orc_amrn_prolong(ctypes.byref(cfg), b, nv, arr, _p(w), len(levels), _p(fine)):
        raise ValueError("orc_amrn_prolong: invalid configuration or box")
    return fine


def amrn_restrict(cfg, b, fine, coarse):
    if _amrn_lib().orc_amrn_restrict(ctypes.byref(cfg), b, fine.shape[0], _p(fine), _p(coarse)):
        raise ValueError("orc_amrn_restrict: invalid configuration or box")
    return coarse


def amrn_step(cfg, kind, coarse, fines, dt, nsteps, params=None):
    """nsteps Berger-Oliger steps of the two-level system `kind` (WAVE or
    BSSN) with every box; arrays updated in place."""
    prm = params if params is not None else default_params()
    arr = (ctypes.POINTER(ctypes.c_double) * len(fines))(*[_p(f) for f in fines])
    rc = _amrn_lib().orc_amrn_step(ctypes.byref(cfg), kind, ctypes.byref(prm), _p(coarse), arr, dt, nsteps)
    if rc != 0:
        raise RuntimeError("orc_amrn_step failed: %d" % rc)


def patches_rk4(states, g, h, dt, nsteps, params=None):
    """Batched patches: each periodic patch advanced on its own."""
    return [rk4(BSSN, y, g, h, dt, nsteps, params=params) for y in states]
