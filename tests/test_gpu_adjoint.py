"""GPU discrete adjoint (chemora_adjoint_rk4) against the oracle's adjoint,
a central finite difference of the GPU's own loss, and the autograd
Function."""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth
from helpers import scaled_err, to_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1764_gb300 import api as A
    A.lib()
    return A


def _problem(orc, n, g, seed, nrecv, nsteps):
    y0, h = synth.gaussian_pulses(n, g, seed=seed, width=0.1)
    c = synth.wave_speed(n, g, seed)
    ctrue = synth.wave_speed(n, g, seed + 1)
    recv = synth.receivers(n, g, seed, nrecv)
    st = (ctrue * ctrue).copy()
    orc.fill_ghosts(st, g)
    yt = orc.rk4(orc.WAVE_VARC, y0, g, h, 0.25 * h, nsteps, s=st)
    data = yt[0].reshape(-1)[recv]
    return y0, c, recv, data, h


@pytest.mark.parametrize("n,nsteps,ckpt", [(16, 12, 4), (20, 7, 3), (12, 5, 10)])
def test_adjoint_matches_oracle(api, orc, n, nsteps, ckpt):
    g = 2
    y0, c, recv, data, h = _problem(orc, n, g, seed=3, nrecv=40, nsteps=nsteps)
    dt = 0.25 * h
    s = (c * c).copy()
    orc.fill_ghosts(s, g)
    J, gy, gs = orc.varc_adjoint(y0, s, g, h, dt, nsteps, ckpt, recv, data)
    gc = 2 * c * gs
    sysm = api.make_system(api.WAVE_VARC, n, n, n, h)
    Jg, gyg, gcg = api.adjoint_rk4(sysm, to_gpu(y0), to_gpu(c), dt, nsteps, ckpt, recv, data)
    assert Jg == pytest.approx(J, rel=1e-11)
    assert scaled_err(to_np(gyg), gy, g) <= 1e-10
    assert scaled_err(to_np(gcg)[None], gc[None], g) <= 1e-10
    # ghosts of the gradients are zero
    assert np.all(to_np(gcg)[:g] == 0) and np.all(to_np(gyg)[:, :, :g] == 0)


def test_checkpoint_interval_changes_no_value(api, orc):
    """Checkpointing only trades memory for recomputation: every interval
    (each step, ragged segments, one segment written by the forward pass
    alone) gives the same loss and gradients, bit for bit."""
    n, g, nsteps = 16, 2, 9
    y0, c, recv, data, h = _problem(orc, n, g, seed=5, nrecv=24, nsteps=nsteps)
    sysm = api.make_system(api.WAVE_VARC, n, n, n, h)
    Y0, C = to_gpu(y0), to_gpu(c)
    runs = [api.adjoint_rk4(sysm, Y0, C, 0.25 * h, nsteps, ck, recv, data) for ck in (1, 2, 4, 9, 50)]
    J0, gy0, gc0 = runs[0][0], to_np(runs[0][1]), to_np(runs[0][2])
    for J, gy, gc in runs[1:]:
        assert J == J0
        assert np.array_equal(to_np(gy), gy0) and np.array_equal(to_np(gc), gc0)


def test_adjoint_fd_full_size(api):
    """The 128^3, 50-step, 512-receiver workload: the gradient in c matches a
    central difference of the GPU's own loss along a smooth direction."""
    import torch
    n, g, nsteps = 128, 2, 50
    y0, c, recv, h, seed_true = synth.adjoint_problem(n=n, g=g)
    dt = 0.25 * h
    sysm = api.make_system(api.WAVE_VARC, n, n, n, h)
    # data from the 'true' speed: forward run through the library
    ctrue = to_gpu(synth.wave_speed(n, g, seed_true))
    sysm.set_speed(ctrue)
    yt = to_gpu(y0)
    sysm.rk4_step(yt, dt, nsteps)
    data = to_np(yt)[0].reshape(-1)[recv]
    Y0, C = to_gpu(y0), to_gpu(c)
    J, gy, gc = api.adjoint_rk4(sysm, Y0, C, dt, nsteps, 10, recv, data)
    assert J > 0
    dc = to_gpu(synth.pad(synth.smooth_field(n, 77, sigma_cells=8.0), g)[0])
    eps = 1e-5 * float(C.abs().max())
    Jp = api.adjoint_rk4(sysm, Y0, C + eps * dc, dt, nsteps, 10, recv, data)[0]
    Jm = api.adjoint_rk4(sysm, Y0, C - eps * dc, dt, nsteps, 10, recv, data)[0]
    fd = (Jp - Jm) / (2 * eps)
    an = float((gc * dc).sum())
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
    torch.cuda.synchronize()


def test_autograd_function(api, orc):
    import torch
    n, g, nsteps = 12, 2, 6
    y0, c, recv, data, h = _problem(orc, n, g, seed=5, nrecv=30, nsteps=nsteps)
    sysm = api.make_system(api.WAVE_VARC, n, n, n, h)
    Y0 = to_gpu(y0).requires_grad_(True)
    C = to_gpu(c).requires_grad_(True)
    loss = api.WaveAdjoint.apply(Y0, C, sysm, recv, data, 0.25 * h, nsteps, 2)
    (3.0 * loss).backward()
    J, gy, gc = api.adjoint_rk4(sysm, to_gpu(y0), to_gpu(c), 0.25 * h, nsteps, 2, recv, data)
    assert float(loss.detach()) == J
    assert torch.equal(Y0.grad, 3.0 * gy) and torch.equal(C.grad, 3.0 * gc)


def test_adjoint_rejects_bad_receivers(api):
    import torch
    from paper_1410_1764_gb300._native import ChemoraError
    n, g = 8, 2
    sysm = api.make_system(api.WAVE_VARC, n, n, n, 1.0 / n)
    y0 = torch.zeros(sysm.grid.shape, dtype=torch.float64, device="cuda")
    c = torch.ones(sysm.grid.shape[1:], dtype=torch.float64, device="cuda")
    with pytest.raises(ChemoraError):
        api.adjoint_rk4(sysm, y0, c, 0.01, 2, 1, [0], [0.0])  # a ghost point


def _dot_inputs(nx, ny, nz, g, seed, nrecv):
    """Random state pair x (u and rho white noise), a smooth speed c and
    receiver weights y at nrecv distinct interior points of an nx x ny x nz
    grid (padded linear indices)."""
    r = synth.rng(seed)
    x = synth.pad(r.standard_normal((2, nz, ny, nx)), g)
    m = max(nx, ny, nz)
    c = synth.pad(1.0 + 0.2 * synth.smooth_field(m, seed + 1, sigma_cells=2.0)[:nz, :ny, :nx], g)[0]
    flat = r.choice(nx * ny * nz, size=nrecv, replace=False)
    k, rem = np.divmod(flat, nx * ny)
    j, i = np.divmod(rem, nx)
    recv = ((k + g) * (ny + 2 * g) + (j + g)) * (nx + 2 * g) + (i + g)
    y = r.standard_normal(nrecv)
    return x, c, recv, y


DOT_CASES = [(128, 128, 128, 50, 10, 512), (21, 13, 17, 9, 4, 300)]


@pytest.mark.parametrize("nx,ny,nz,nsteps,ckpt,nrecv", DOT_CASES)
def test_adjoint_dot_product_quadratic(api, nx, ny, nz, nsteps, ckpt, nrecv):
    """With data = 0 the loss is J = 1/2 |R M x|^2 for the linear RK4 map M
    (fixed c) and receiver restriction R, so <x, grad_x J> = <x, M^T R^T R M x>
    must equal 2 J: the reverse sweep is the transpose of the forward pass
    along x (dot-product identity, 1e-12)."""
    g = 2
    x, c, recv, _ = _dot_inputs(nx, ny, nz, g, seed=11, nrecv=nrecv)
    h = 1.0 / max(nx, ny, nz)
    sysm = api.make_system(api.WAVE_VARC, nx, ny, nz, h)
    X = to_gpu(x)
    J, gx, _ = api.adjoint_rk4(sysm, X, to_gpu(c), 0.25 * h, nsteps, ckpt, recv, np.zeros(nrecv))
    assert J > 0
    lhs = float((X * gx).sum())
    assert abs(lhs - 2 * J) <= 1e-12 * (2 * J), (lhs, 2 * J)


@pytest.mark.parametrize("nx,ny,nz,nsteps,ckpt,nrecv", DOT_CASES)
def test_adjoint_dot_product_two_vectors(api, nx, ny, nz, nsteps, ckpt, nrecv):
    """<R M x, y> = <x, M^T R^T y> with x and y independent.  M x is the
    library's RK4 forward (chemora_rk4_step after chemora_system_set_speed);
    M^T R^T y is the gradient of the adjoint call started from the zero
    state with data = -y (then u_N = 0 and the misfit seed is y)."""
    g = 2
    x, c, recv, y = _dot_inputs(nx, ny, nz, g, seed=12, nrecv=nrecv)
    h = 1.0 / max(nx, ny, nz)
    dt = 0.25 * h
    sysm = api.make_system(api.WAVE_VARC, nx, ny, nz, h)
    C = to_gpu(c)
    Z = to_gpu(np.zeros_like(x))
    J, mty, _ = api.adjoint_rk4(sysm, Z, C, dt, nsteps, ckpt, recv, -y)
    assert J == pytest.approx(0.5 * float(np.sum(y * y)), rel=1e-14)
    sysm.set_speed(C)
    X = to_gpu(x)
    sysm.rk4_step(X, dt, nsteps)
    mx = to_np(X)[0].reshape(-1)[recv]
    lhs = float(np.sum(mx * y))
    rhs = float((to_gpu(x) * mty).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)
