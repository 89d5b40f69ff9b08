"""Python API over the C ABI: grids, systems, batched patches and the
discrete-adjoint autograd Function.

PyTorch provides device memory and streams only; every computation runs in
libchemora's kernels.  State tensors are float64 CUDA tensors shaped
(nvars, nz+2g, ny+2g, nx+2g), contiguous.
"""
import ctypes

import torch

from . import _native as N
from ._native import BSSN, WAVE, WAVE1, WAVE_VARC, Params, check, lib

NVARS = {WAVE: 2, WAVE_VARC: 2, BSSN: 24, WAVE1: 5}
NGHOST = {WAVE: 2, WAVE_VARC: 2, BSSN: 3, WAVE1: 2}


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def default_params(eps_diss=0.1, eta=2.0, slicing=0, shift=0, fd_order=0):
    return Params(eps_diss, eta, slicing, shift, fd_order)


class Grid:
    """Uniform periodic grid with ghost zones (chemora_grid_create)."""

    def __init__(self, nx, ny, nz, nvars, nghost, dx):
        h = ctypes.c_void_p()
        check(lib().chemora_grid_create(nx, ny, nz, nvars, nghost, dx, ctypes.byref(h)),
              "chemora_grid_create")
        self.handle = h
        self.nx, self.ny, self.nz, self.nvars, self.nghost, self.dx = nx, ny, nz, nvars, nghost, dx

    @property
    def shape(self):
        g = self.nghost
        return (self.nvars, self.nz + 2 * g, self.ny + 2 * g, self.nx + 2 * g)

    def layout(self):
        sy, sz, sv = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().chemora_grid_layout(self.handle, ctypes.byref(sy), ctypes.byref(sz),
                                        ctypes.byref(sv)), "chemora_grid_layout")
        return sy.value, sz.value, sv.value

    def __del__(self):
        if getattr(self, "handle", None) and N._lib is not None:
            N._lib.chemora_destroy(self.handle)
            self.handle = None


class System:
    """A PDE system on a grid (chemora_system_create)."""

    def __init__(self, grid, kind, params=None):
        self.grid = grid
        self.kind = kind
        h = ctypes.c_void_p()
        p = ctypes.byref(params) if params is not None else None
        check(lib().chemora_system_create(grid.handle, kind, p, ctypes.byref(h)),
              "chemora_system_create")
        self.handle = h

    def set_speed(self, c, stream=None):
        check(lib().chemora_system_set_speed(self.handle, _ptr(c), _stream(stream)),
              "chemora_system_set_speed")

    def fill_ghosts(self, state, stream=None):
        check(lib().chemora_fill_ghosts(self.handle, _ptr(state), _stream(stream)),
              "chemora_fill_ghosts")
        return state

    def fill_ghosts_axes(self, state, axes, stream=None):
        """Periodic ghosts along the axes of the bit mask (1 x, 2 y, 4 z)."""
        check(lib().chemora_fill_ghosts_axes(self.handle, _ptr(state), int(axes), _stream(stream)),
              "chemora_fill_ghosts_axes")
        return state

    def stage(self, mode, src, yn, acc, dst, c1=0.0, c2=0.0, stream=None):
        """One fused stage kernel (chemora_stage)."""
        nul = ctypes.c_void_p()
        check(lib().chemora_stage(self.handle, int(mode), _ptr(src), _ptr(yn) if yn is not None else nul,
                                  _ptr(acc) if acc is not None else nul, _ptr(dst), float(c1), float(c2),
                                  _stream(stream)), "chemora_stage")
        return dst

    def rhs(self, state, out=None, stream=None):
        if out is None:
            out = torch.zeros_like(state)
        check(lib().chemora_rhs(self.handle, _ptr(state), _ptr(out), _stream(stream)),
              "chemora_rhs")
        return out

    def rk4_step(self, state, dt, nsteps=1, stream=None):
        check(lib().chemora_rk4_step(self.handle, _ptr(state), float(dt), int(nsteps),
                                     _stream(stream)), "chemora_rk4_step")
        return state

    def rk4_step_host(self, state, dt, nsteps=1, stream=None):
        """RK4 steps of a float64 CPU tensor (pinned recommended), in place."""
        if state.is_cuda or state.dtype != torch.float64 or not state.is_contiguous():
            raise ValueError("expected a contiguous float64 CPU tensor")
        check(lib().chemora_rk4_step_host(self.handle, ctypes.c_void_p(state.data_ptr()), float(dt),
                                          int(nsteps), _stream(stream)), "chemora_rk4_step_host")
        return state

    def set_chain(self, mode):
        """Order-4 scalar wave: 0 per-stage kernels, 1 launch-chained stage
        kernels (programmatic dependent launches), -1 query; returns the
        mode in force."""
        a = ctypes.c_int()
        check(lib().chemora_system_set_chain(self.handle, int(mode), ctypes.byref(a)), "chemora_system_set_chain")
        return a.value

    def autotune(self, state, stream=None):
        """Pick the fastest launch shape on `state` (fills its ghosts);
        returns (variant, (tx, ty), rhs_ms)."""
        v, ms = ctypes.c_int(), ctypes.c_double()
        check(lib().chemora_autotune(self.handle, _ptr(state), ctypes.byref(v), ctypes.byref(ms),
                                     _stream(stream)), "chemora_autotune")
        return v.value, self.variant()[1], ms.value

    def specialize(self, enable=True, cache_dir=None):
        """Compile (NVRTC) and use stage kernels specialised to this system's
        grid, scalars and current launch shape (enable=False returns to the
        ahead-of-time kernels).  cache_dir: cubin cache directory (None: the
        library default, "": none).  Returns the compile time in seconds (0
        when nothing was compiled)."""
        secs = ctypes.c_double()
        cd = None if cache_dir is None else str(cache_dir).encode()
        check(lib().chemora_system_specialize(self.handle, 1 if enable else 0, cd, ctypes.byref(secs)),
              "chemora_system_specialize")
        return secs.value

    def variant(self, set_to=None):
        v, tx, ty = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().chemora_system_variant(self.handle, -1 if set_to is None else int(set_to),
                                           ctypes.byref(v), ctypes.byref(tx), ctypes.byref(ty)),
              "chemora_system_variant")
        return v.value, (tx.value, ty.value)

    def constraints(self, state, out=None, stream=None):
        """BSSN constraints (H, M^x, M^y, M^z, G^x, G^y, G^z); ghosts of state valid."""
        if out is None:
            out = torch.zeros((7,) + tuple(state.shape[1:]), dtype=torch.float64, device=state.device)
        check(lib().chemora_constraints(self.handle, _ptr(state), _ptr(out), _stream(stream)),
              "chemora_constraints")
        return out

    def energy(self, state, stream=None):
        """Discrete wave energy 1/2 sum (rho^2 - u Lap u) h^3 (ghosts valid)."""
        e = ctypes.c_double()
        check(lib().chemora_energy(self.handle, _ptr(state), ctypes.byref(e), _stream(stream)),
              "chemora_energy")
        return e.value

    def nonfinite(self, state, stream=None):
        """Number of NaN/Inf interior values (0 when the state is finite)."""
        n = ctypes.c_int64()
        code = lib().chemora_check_finite(self.handle, _ptr(state), ctypes.byref(n), _stream(stream))
        if code not in (N.OK, N.ENONFINITE):
            check(code, "chemora_check_finite")
        return n.value

    def opcount(self):
        """(fp64 instructions, flops) per point per RHS of the body this
        system launches."""
        i, f = ctypes.c_int64(), ctypes.c_int64()
        check(lib().chemora_system_opcount(self.handle, ctypes.byref(i), ctypes.byref(f)),
              "chemora_system_opcount")
        return i.value, f.value

    def profile(self, on=True):
        check(lib().chemora_profile_enable(self.handle, 1 if on else 0), "chemora_profile_enable")

    def profile_read(self, reset=True):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        check(lib().chemora_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(n),
                                         1 if reset else 0), "chemora_profile_read")
        return ms.value, n.value

    def __del__(self):
        if getattr(self, "handle", None) and N._lib is not None:
            N._lib.chemora_destroy(self.handle)
            self.handle = None


def make_system(kind, nx, ny, nz, dx, params=None, nghost=None):
    order = (params.fd_order if params is not None else 0) or 4
    g = Grid(nx, ny, nz, NVARS[kind], nghost or max(NGHOST[kind], order // 2), dx)
    return System(g, kind, params)


def save_checkpoint(path, state, t=0.0, step=0, **meta):
    """Write a state (any float64 tensor, e.g. the padded grid state, copied
    to the host) with its time, step count and caller metadata to `path`
    (torch.save): the simulation's checkpoint, restored by load_checkpoint."""
    torch.save({"state": state.detach().to("cpu"), "t": float(t), "step": int(step), "meta": dict(meta)}, path)


def load_checkpoint(path, device=None):
    """(state, t, step, meta) written by save_checkpoint; the state is moved
    to `device` when one is given."""
    ck = torch.load(path, map_location="cpu", weights_only=True)
    st = ck["state"] if device is None else ck["state"].to(device)
    return st, ck["t"], ck["step"], ck["meta"]


def launch_count():
    return lib().chemora_launch_count()


def opcount(kind):
    i, f = ctypes.c_int64(), ctypes.c_int64()
    check(lib().chemora_opcount(kind, ctypes.byref(i), ctypes.byref(f)), "chemora_opcount")
    return i.value, f.value


def variant_info(kind, variant):
    """(tx, ty, min_blocks, sharing) of a compiled launch shape; sharing 0 =
    direct body, 1 = x lanes, 2 = x lanes + y through shared memory."""
    o = [ctypes.c_int() for _ in range(4)]
    check(lib().chemora_variant_info(int(kind), int(variant), *[ctypes.byref(x) for x in o]),
          "chemora_variant_info")
    return tuple(x.value for x in o)


def fp64_peak(stream=None):
    v = ctypes.c_double()
    check(lib().chemora_fp64_peak(ctypes.byref(v), _stream(stream)), "chemora_fp64_peak")
    return v.value


class _DeviceArray:
    """A view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, shape, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


class Batch:
    """Many independent periodic patches advanced together
    (chemora_patches_create / chemora_patches_step)."""

    def __init__(self, dims, nghost, dx, kind=BSSN, params=None):
        dims = [tuple(int(v) for v in d) for d in dims]
        arr = (ctypes.c_int * (3 * len(dims)))(*[v for d in dims for v in d])
        h = ctypes.c_void_p()
        p = ctypes.byref(params) if params is not None else None
        check(lib().chemora_patches_create(len(dims), arr, nghost, float(dx), kind, p, ctypes.byref(h)),
              "chemora_patches_create")
        self.handle = h
        self.dims = dims
        self.nghost = nghost
        self.kind = kind
        self.nvars = NVARS[kind]

    def shape(self, p):
        nx, ny, nz = self.dims[p]
        g = self.nghost
        return (self.nvars, nz + 2 * g, ny + 2 * g, nx + 2 * g)

    def state(self, p):
        """A torch view (no copy) of patch p's state inside the batch storage."""
        ptr = ctypes.c_void_p()
        check(lib().chemora_patches_state(self.handle, p, ctypes.byref(ptr)), "chemora_patches_state")
        return torch.as_tensor(_DeviceArray(ptr.value, self.shape(p), self), device="cuda")

    def step(self, dt, nsteps=1, mode=0, stream=None):
        check(lib().chemora_patches_step(self.handle, float(dt), int(nsteps), int(mode), _stream(stream)),
              "chemora_patches_step")

    def set_time_limit(self, seconds):
        """Time limit of each persistent stage launch (0: none); a step that
        passes it raises ChemoraError with CHEMORA_ETIMEOUT."""
        check(lib().chemora_patches_set_time_limit(self.handle, float(seconds)),
              "chemora_patches_set_time_limit")

    def __del__(self):
        if getattr(self, "handle", None) and N._lib is not None:
            N._lib.chemora_destroy(self.handle)
            self.handle = None


def adjoint_rk4(system, state0, c, dt, nsteps, ckpt_every, recv, data, stream=None):
    """Loss J = 1/2 sum (u_N[recv] - data)^2 of the variable-speed wave
    equation after nsteps RK4 steps and its gradients with respect to the
    initial state and the wave speed c (chemora_adjoint_rk4).
    recv: padded linear indices (int64, host); data: float64 (host).
    Returns (loss: float, grad_state0: tensor, grad_c: tensor)."""
    import numpy as np
    recv = np.ascontiguousarray(np.asarray(recv, dtype=np.int64))
    data = np.ascontiguousarray(np.asarray(data, dtype=np.float64))
    gs = torch.empty_like(state0)
    gc = torch.empty_like(c)
    loss = ctypes.c_double()
    check(lib().chemora_adjoint_rk4(system.handle, _ptr(state0), _ptr(c), float(dt), int(nsteps),
                                    int(ckpt_every), recv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    len(recv), data.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    ctypes.byref(loss), _ptr(gs), _ptr(gc), _stream(stream)),
          "chemora_adjoint_rk4")
    return loss.value, gs, gc


class WaveAdjoint(torch.autograd.Function):
    """J(state0, c) of the variable-speed wave equation with the discrete
    adjoint as its backward.  The library computes J and both gradients in one
    call (forward pass with checkpoints, then the reverse sweep), so forward
    keeps the gradients and backward scales them by the incoming gradient.

        loss = WaveAdjoint.apply(state0, c, system, recv, data, dt, nsteps, ckpt_every)
    """

    @staticmethod
    def forward(ctx, state0, c, system, recv, data, dt, nsteps, ckpt_every):
        loss, gs, gc = adjoint_rk4(system, state0.detach().contiguous(), c.detach().contiguous(),
                                   dt, nsteps, ckpt_every, recv, data)
        ctx.save_for_backward(gs, gc)
        return torch.tensor(loss, dtype=torch.float64, device=state0.device)

    @staticmethod
    def backward(ctx, grad_loss):
        gs, gc = ctx.saved_tensors
        return grad_loss * gs, grad_loss * gc, None, None, None, None, None, None


class AmrBoxes:
    """Two-level mesh refinement with Berger-Oliger subcycling, several
    boxes, scalar wave or BSSN (chemora_amr_create_boxes /
    chemora_amr_step_mode).  nc = (nx, ny, nz) coarse points; boxes = list of
    (lo, hi) coarse point ranges refined by 2."""

    def __init__(self, kind, nc, boxes, dx, params=None):
        nb = len(boxes)
        lo = (ctypes.c_int * (3 * nb))(*[int(v) for b in boxes for v in b[0]])
        hi = (ctypes.c_int * (3 * nb))(*[int(v) for b in boxes for v in b[1]])
        h = ctypes.c_void_p()
        prm = ctypes.byref(params) if params is not None else None
        check(lib().chemora_amr_create_boxes(int(kind), (ctypes.c_int * 3)(*[int(v) for v in nc]), nb, lo, hi,
                                             float(dx), prm, ctypes.byref(h)), "chemora_amr_create_boxes")
        self.handle = h
        self.kind, self.nv = kind, NVARS[kind]
        self.nc, self.boxes = tuple(nc), [(tuple(b[0]), tuple(b[1])) for b in boxes]

    def state(self, level):
        """A torch view (no copy) of level 0 (coarse) or 1 + b (box b, with
        its buffer) of the state, shaped (nvars, pz, py, px)."""
        ptr, sy, sz, sv = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().chemora_amr_state(self.handle, int(level), ctypes.byref(ptr), ctypes.byref(sy),
                                      ctypes.byref(sz), ctypes.byref(sv)), "chemora_amr_state")
        px, py, pz = sy.value, sz.value // sy.value, sv.value // sz.value
        return torch.as_tensor(_DeviceArray(ptr.value, (self.nv, pz, py, px), self), device="cuda")

    def autotune(self, stream=None):
        """Pick the coarse stage kernel's launch shape by timing; returns it."""
        v = ctypes.c_int()
        check(lib().chemora_amr_autotune(self.handle, ctypes.byref(v), _stream(stream)), "chemora_amr_autotune")
        return v.value

    def step(self, dt, nsteps=1, mode=0, stream=None):
        """mode 0: one batched launch per fine RK stage over every box;
        mode 1: box by box."""
        check(lib().chemora_amr_step_mode(self.handle, float(dt), int(nsteps), int(mode), _stream(stream)),
              "chemora_amr_step_mode")

    def __del__(self):
        if getattr(self, "handle", None) and N._lib is not None:
            N._lib.chemora_destroy(self.handle)
            self.handle = None


class Amr:
    """Two-level mesh refinement with Berger-Oliger subcycling for the
    scalar wave with one box (chemora_amr_create / chemora_amr_step)."""

    def __init__(self, nc, lo, hi, dx):
        h = ctypes.c_void_p()
        check(lib().chemora_amr_create(int(nc), (ctypes.c_int * 3)(*lo), (ctypes.c_int * 3)(*hi), float(dx),
                                       ctypes.byref(h)), "chemora_amr_create")
        self.handle = h
        self.nc, self.lo, self.hi = nc, tuple(lo), tuple(hi)

    def state(self, level):
        """A torch view (no copy) of level 0 (coarse) or 1 (fine, with its
        8-point buffer) of the 2-variable state."""
        ptr, sy, sz, sv = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().chemora_amr_state(self.handle, level, ctypes.byref(ptr), ctypes.byref(sy), ctypes.byref(sz),
                                      ctypes.byref(sv)), "chemora_amr_state")
        px, py, pz = sy.value, sz.value // sy.value, sv.value // sz.value
        return torch.as_tensor(_DeviceArray(ptr.value, (2, pz, py, px), self), device="cuda")

    def step(self, dt, nsteps=1, stream=None):
        check(lib().chemora_amr_step(self.handle, float(dt), int(nsteps), _stream(stream)), "chemora_amr_step")

    def __del__(self):
        if getattr(self, "handle", None) and N._lib is not None:
            N._lib.chemora_destroy(self.handle)
            self.handle = None
