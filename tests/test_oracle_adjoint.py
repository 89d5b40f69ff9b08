"""Pins of the oracle's differentiation of the variable-speed wave RK4 map.

- the tangent-linear map matches central finite differences of the forward
  map (the map is linear in the state, quadratic-plus in s);
- dot-product identity <M x, y> = <x, M^T y> for the one-step and the
  many-step maps, with respect to the state and to s = c^2;
- the gradient of the receiver misfit matches central differences;
- for constant c the spatial operator is self-adjoint;
- checkpointing changes no value.
"""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth

G = 2


def _setup(n=12, seed=0):
    rng = np.random.default_rng(seed)
    y0 = synth.pad(rng.standard_normal((2, n, n, n)), G)
    c = synth.pad(1.0 + 0.2 * synth.smooth_field(n, seed + 10, sigma_cells=1.5), G)[0]
    h = 1.0 / n
    return y0, c, h, rng


def _filled(a, orc):
    a = a.copy()
    orc.fill_ghosts(a, G)
    return a


def _ip(a, b):
    return float(np.sum(synth.interior(a, G) * synth.interior(b, G)))


def test_tlm_matches_fd(orc):
    y0, c, h, rng = _setup()
    s = _filled(c * c, orc)
    dt = 0.25 * h
    dy = synth.pad(rng.standard_normal((2, 12, 12, 12)), G)
    ds = _filled(synth.pad(rng.standard_normal((12, 12, 12)), G)[0], orc)
    _, tl = orc.varc_tlm_rk4(y0, dy, s, ds, G, h, dt, 3)
    eps = 1e-4
    fp = orc.rk4(orc.WAVE_VARC, y0 + eps * dy, G, h, dt, 3, s=s + eps * ds)
    fm = orc.rk4(orc.WAVE_VARC, y0 - eps * dy, G, h, dt, 3, s=s - eps * ds)
    fd = (fp - fm) / (2 * eps)
    a, b = synth.interior(tl, G), synth.interior(fd, G)
    assert np.abs(a - b).max() < 1e-7 * np.abs(b).max()


@pytest.mark.parametrize("nsteps,ckpt", [(1, 1), (7, 3)])
def test_dot_product(orc, nsteps, ckpt):
    y0, c, h, rng = _setup(seed=1)
    s = _filled(c * c, orc)
    dt = 0.25 * h
    dy = synth.pad(rng.standard_normal((2, 12, 12, 12)), G)
    ds = _filled(synth.pad(rng.standard_normal((12, 12, 12)), G)[0], orc)
    ybar = synth.pad(rng.standard_normal((2, 12, 12, 12)), G)
    _, tl = orc.varc_tlm_rk4(y0, dy, s, ds, G, h, dt, nsteps)
    yb0, sb = orc.varc_vjp(y0, s, G, h, dt, nsteps, ckpt, ybar)
    lhs = _ip(tl, ybar)
    rhs = _ip(dy, yb0) + _ip(ds[None], sb[None])
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_constant_c_self_adjoint(orc):
    """With s constant, L(s)^T = L(s): J^T (kb_u, kb_rho) = (L kb_rho, kb_u)."""
    y0, _, h, rng = _setup(seed=2)
    s = np.full_like(y0[0], 1.44)
    kb = _filled(synth.pad(rng.standard_normal((2, 12, 12, 12)), G), orc)
    yhat, _ = orc.varc_adj_rhs(_filled(y0, orc), s, kb, G, h)
    fwd = orc.varc_rhs(np.stack([kb[1], kb[0]]), s, G, h)
    np.testing.assert_allclose(synth.interior(yhat[0], G), synth.interior(fwd[1], G),
                               rtol=0, atol=1e-9 * np.abs(fwd[1]).max())
    np.testing.assert_array_equal(synth.interior(yhat[1], G), synth.interior(kb[0], G))


def _loss(orc, y0, c, h, dt, nsteps, recv, data):
    y = orc.rk4(orc.WAVE_VARC, y0, G, h, dt, nsteps, s=_filled(c * c, orc))
    m = y[0].reshape(-1)[recv] - data
    return 0.5 * float(np.sum(m * m))


def test_gradient_fd(orc):
    """Directional central difference of J with respect to c (smooth
    direction, eps = 1e-5 |c|_inf) and 16 single-point checks on u0."""
    n = 16
    y0, h = synth.gaussian_pulses(n, G, seed=3, width=0.1)
    c = synth.wave_speed(n, G, seed=3)
    recv = synth.receivers(n, G, seed=3, nrecv=64)
    dt, nsteps = 0.25 * h, 12
    ctrue = synth.wave_speed(n, G, seed=4)
    ytrue = orc.rk4(orc.WAVE_VARC, y0, G, h, dt, nsteps, s=_filled(ctrue * ctrue, orc))
    data = ytrue[0].reshape(-1)[recv]
    s = _filled(c * c, orc)
    J, gy, gs = orc.varc_adjoint(y0, s, G, h, dt, nsteps, 4, recv, data)
    assert J > 0
    assert J == pytest.approx(_loss(orc, y0, c, h, dt, nsteps, recv, data), rel=1e-14)
    gc = 2 * c * gs
    dc = synth.pad(synth.smooth_field(n, 99, sigma_cells=2.0), G)[0]
    eps = 1e-5 * np.abs(c).max()
    fd = (_loss(orc, y0, c + eps * dc, h, dt, nsteps, recv, data)
          - _loss(orc, y0, c - eps * dc, h, dt, nsteps, recv, data)) / (2 * eps)
    an = _ip(gc[None], dc[None])
    assert abs(fd - an) <= 1e-6 * abs(an)
    rng = np.random.default_rng(5)
    pts = rng.choice(n ** 3, 16, replace=False)
    for q in pts:
        k, r = divmod(int(q), n * n)
        j, i = divmod(r, n)
        e = np.zeros_like(y0)
        e[0, k + G, j + G, i + G] = 1.0
        d = 1e-3
        fd = (_loss(orc, y0 + d * e, c, h, dt, nsteps, recv, data)
              - _loss(orc, y0 - d * e, c, h, dt, nsteps, recv, data)) / (2 * d)
        an = gy[0, k + G, j + G, i + G]
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-8 * np.abs(gy).max()), (fd, an)


def test_checkpointing_changes_nothing(orc):
    n = 10
    y0, h = synth.gaussian_pulses(n, G, seed=6, width=0.15)
    c = synth.wave_speed(n, G, seed=6)
    s = _filled(c * c, orc)
    recv = synth.receivers(n, G, seed=6, nrecv=20)
    data = np.zeros(20)
    ref = orc.varc_adjoint(y0, s, G, h, 0.25 * h, 9, 1, recv, data)
    for ck in (2, 4, 9, 50):
        got = orc.varc_adjoint(y0, s, G, h, 0.25 * h, 9, ck, recv, data)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
