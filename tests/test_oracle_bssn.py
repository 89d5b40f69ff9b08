"""Pins of the oracle's BSSN right-hand side and constraints.

The paper (Sec. 3.4, Sec. 5) names the Einstein equations but prints no
formulas; the oracle writes out the standard BSSN phi-form.  These tests pin
it against what the mathematics fixes:
  - flat space is an exact static solution (RHS == 0 exactly);
  - spatially homogeneous data reduce the system to ODEs (closed form for
    harmonic slicing and the Gamma-driver, an independent DOP853 solution for
    1+log), reached by RK4 at 4th order in dt;
  - the RHS commutes with permutations of the coordinate axes;
  - the gauge wave (harmonic slicing, zero shift) is an exact solution: state
    and constraints converge at 4th order;
  - Kerr-Schild Schwarzschild with frozen gauge is stationary: the RHS of
    every non-gauge variable and the constraints vanish at 4th order (exact
    data from an independent sympy computation);
  - flat space plus 1e-10 noise stays at round-off over 100 steps.
"""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth

G = 3
SYM = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]
NONGAUGE = list(range(17))


def _params(orc, eps=0.1, eta=2.0, slicing=0, shift=0):
    return orc.Params(eps, eta, slicing, shift)


def _const_state(n, vals):
    st = np.empty((24, n + 2 * G, n + 2 * G, n + 2 * G))
    st[:] = np.asarray(vals)[:, None, None, None]
    return st


def test_flat_rhs_is_zero(orc):
    st = _const_state(6, synth.BSSN_FLAT)
    r = orc.bssn_rhs(st, G, 1.0 / 6)
    assert np.array_equal(synth.interior(r, G), np.zeros((24, 6, 6, 6)))


def _homog_state(phi0, K0, al0, be0, B0):
    v = synth.BSSN_FLAT.copy()
    v[0] = phi0
    v[7] = K0
    v[17] = al0
    v[18:21] = be0
    v[21:24] = B0
    return v


def _reduced_ode_1log(phi0, K0, a0, T):
    """Homogeneous reduction with 1+log slicing, solved by an independent
    high-order integrator: alpha' = -2 alpha K, K' = alpha K^2 / 3,
    phi' = -alpha K / 6."""
    integrate = pytest.importorskip("scipy.integrate")
    f = lambda t, y: [-2 * y[0] * y[1], y[0] * y[1] ** 2 / 3, -y[0] * y[1] / 6]
    sol = integrate.solve_ivp(f, (0, T), [a0, K0, phi0], method="DOP853", rtol=1e-13, atol=1e-15)
    return sol.y[:, -1]


@pytest.mark.parametrize("slicing", [0, 1])
def test_homogeneous_ode_closed_form(orc, slicing):
    """Homogeneous data with flat conformal metric and At = 0 reduce the
    system to ODEs.  Harmonic slicing has the closed form
      alpha = a0 (K0/K)^3,  K^2 = K0^2 + 2/3 a0 K0^3 t,  phi = phi0 - ln(K/K0)/2;
    1+log slicing is checked against an independent DOP853 solution.  For
    both, B = B0 e^{-eta t} and beta = beta0 + 3/4 B0 (1 - e^{-eta t}) / eta."""
    phi0, K0, a0, eta, T = 0.1, 0.3, 0.8, 2.0, 1.0
    be0 = np.array([0.1, -0.2, 0.05])
    B0 = np.array([0.3, 0.1, -0.2])
    if slicing == 0:
        al, K, phi = _reduced_ode_1log(phi0, K0, a0, T)
    else:
        K = np.sqrt(K0 ** 2 + 2.0 / 3.0 * a0 * K0 ** 3 * T)
        al = a0 * (K0 / K) ** 3
        phi = phi0 - 0.5 * np.log(K / K0)
    exact = _homog_state(phi, K, al, be0 + 0.75 * B0 * (1 - np.exp(-eta * T)) / eta,
                         B0 * np.exp(-eta * T))
    errs = []
    for nsteps in (8, 16):
        st = _const_state(4, _homog_state(phi0, K0, a0, be0, B0))
        y = orc.rk4(orc.BSSN, st, G, 0.25, T / nsteps, nsteps,
                    params=_params(orc, slicing=slicing, eta=eta))
        got = y[:, G, G, G]
        errs.append(np.abs(got - exact).max())
        # the conformal metric, At and Xt stay flat
        assert np.array_equal(y[1:7, G, G, G], synth.BSSN_FLAT[1:7])
        assert np.array_equal(y[8:17, G, G, G], synth.BSSN_FLAT[8:17])
    assert errs[1] < 1e-6
    assert 12.0 < errs[0] / errs[1] < 20.0, errs


def _permute(st, sigma):
    """Relabel coordinate axes: new axis i is old axis sigma[i]."""
    out = np.empty_like(st)
    order = (3 - sigma[2], 3 - sigma[1], 3 - sigma[0])
    sp = lambda a: np.transpose(a, (order[0] - 1, order[1] - 1, order[2] - 1))
    out[0] = sp(st[0])
    out[7] = sp(st[7])
    out[17] = sp(st[17])
    for i in range(3):
        for j in range(i, 3):
            out[1 + SYM[i][j]] = sp(st[1 + SYM[sigma[i]][sigma[j]]])
            out[8 + SYM[i][j]] = sp(st[8 + SYM[sigma[i]][sigma[j]]])
        for base in (14, 18, 21):
            out[base + i] = sp(st[base + sigma[i]])
    return out


@pytest.mark.parametrize("sigma", [(1, 0, 2), (0, 2, 1), (2, 0, 1)])
def test_axis_permutation(orc, sigma):
    n = 10
    rng = np.random.default_rng(11)
    st = synth.pad(synth.BSSN_FLAT[:, None, None, None] + 1e-2 * rng.standard_normal((24, n, n, n)), G)
    orc.fill_ghosts(st, G)
    h = 1.0 / n
    r = orc.bssn_rhs(st, G, h)
    rp = orc.bssn_rhs(_permute(st, sigma), G, h)
    want = _permute(r, sigma)
    a, b = synth.interior(rp, G), synth.interior(want, G)
    scale = np.abs(b).max(axis=(1, 2, 3), keepdims=True)
    err = np.abs(a - b) / np.maximum(np.abs(b), scale)
    assert err.max() < 1e-13


def gauge_wave_state(nx, ny, nz, t, A=0.1):
    """Exact gauge-wave data in BSSN variables (harmonic slicing, zero shift):
    ds^2 = -H dt^2 + H dx^2 + dy^2 + dz^2, H = 1 - A sin(2 pi (x - t))."""
    h = 1.0 / nx
    p = lambda n: (np.arange(n + 2 * G) - G) * h
    Z, Y, X = np.meshgrid(p(nz), p(ny), p(nx), indexing="ij")
    ph = 2 * np.pi * (X - t)
    H = 1 - A * np.sin(ph)
    dH = -2 * np.pi * A * np.cos(ph)
    Kxx = -(np.pi * A) * np.cos(ph) / np.sqrt(H)
    st = np.zeros((24,) + X.shape)
    st[0] = np.log(H) / 12
    st[1] = H ** (2.0 / 3)
    st[4] = H ** (-1.0 / 3)
    st[6] = H ** (-1.0 / 3)
    st[7] = Kxx / H
    st[8] = 2.0 / 3 * H ** (-1.0 / 3) * Kxx
    st[11] = -1.0 / 3 * H ** (-4.0 / 3) * Kxx
    st[13] = -1.0 / 3 * H ** (-4.0 / 3) * Kxx
    st[14] = 2.0 / 3 * H ** (-5.0 / 3) * dH
    st[17] = np.sqrt(H)
    return st, h


def test_gauge_wave_convergence(orc):
    T = 0.25
    prm = _params(orc, slicing=1, shift=1)
    errs, cons0 = [], []
    for nx in (32, 64, 128):
        st, h = gauge_wave_state(nx, 6, 6, 0.0)
        c = orc.bssn_constraints(st, G, h)
        cons0.append(np.abs(synth.interior(c, G)).max())
        dt = 0.25 * h
        nsteps = int(round(T / dt))
        y = orc.rk4(orc.BSSN, st, G, h, dt, nsteps, params=prm)
        ex, _ = gauge_wave_state(nx, 6, 6, nsteps * dt)
        errs.append(np.abs(synth.interior(y - ex, G)).max())
    for e in (errs, cons0):
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert 13.0 < r1 < 19.5 and 14.0 < r2 < 18.0, e


def test_noise_stays_roundoff(orc):
    """Flat space plus 1e-10 noise: the perturbation stays within the linear
    scale (amplitude times Nyquist wavenumber, ~1e-8) and decays under KO
    dissipation between step 50 and step 150: no growth."""
    n = 16
    st, h = synth.bssn_noise(n, n, n, G, seed=2)
    flat = synth.BSSN_FLAT[:, None, None, None]
    y50 = orc.rk4(orc.BSSN, st, G, h, 0.25 * h, 50)
    y150 = orc.rk4(orc.BSSN, y50, G, h, 0.25 * h, 100)
    d50 = np.abs(synth.interior(y50, G) - flat).max()
    d150 = np.abs(synth.interior(y150, G) - flat).max()
    assert d50 < 1e-8 and d150 < d50


# ---------------------------------------------------------------------------
# Kerr-Schild Schwarzschild (M = 1) with frozen gauge
# ---------------------------------------------------------------------------

def _kerr_schild_funcs():
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    X = [x, y, z]
    r = sp.sqrt(x * x + y * y + z * z)
    Hs = 1 / r
    l = [xi / r for xi in X]
    gam = sp.Matrix(3, 3, lambda i, j: (1 if i == j else 0) + 2 * Hs * l[i] * l[j])
    gi = sp.Matrix(3, 3, lambda i, j: (1 if i == j else 0) - 2 * Hs * l[i] * l[j] / (1 + 2 * Hs))
    alpha = 1 / sp.sqrt(1 + 2 * Hs)
    beta_d = [2 * Hs * l[i] for i in range(3)]
    beta_u = [sum(gi[i, j] * beta_d[j] for j in range(3)) for i in range(3)]
    dg = [[[sp.diff(gam[i, j], X[k]) for k in range(3)] for j in range(3)] for i in range(3)]
    Chr = [[[sum(gi[k, m] * (dg[m][i][j] + dg[m][j][i] - dg[i][j][m]) for m in range(3)) / 2
             for j in range(3)] for i in range(3)] for k in range(3)]
    Db = [[sp.diff(beta_d[j], X[i]) - sum(Chr[k][i][j] * beta_d[k] for k in range(3))
           for j in range(3)] for i in range(3)]
    Kij = sp.Matrix(3, 3, lambda i, j: (Db[i][j] + Db[j][i]) / (2 * alpha))
    detg = 1 + 2 * Hs
    psi4m = detg ** sp.Rational(-1, 3)  # e^{-4 phi}
    gt = gam * psi4m
    gtu = gi / psi4m
    trK = sum(gi[i, j] * Kij[i, j] for i in range(3) for j in range(3))
    At = (Kij - gam * trK / 3) * psi4m
    Xt = [-sum(sp.diff(gtu[i, j], X[j]) for j in range(3)) for i in range(3)]
    exprs = [sp.log(detg) / 12]
    exprs += [gt[i, j] for i, j in ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))]
    exprs += [trK]
    exprs += [At[i, j] for i, j in ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))]
    exprs += Xt + [alpha] + beta_u + [0, 0, 0]
    f = sp.lambdify((x, y, z), exprs, "numpy")
    return f


@pytest.fixture(scope="module")
def kerr_schild():
    return _kerr_schild_funcs()


def _ks_state(f, centre, n, h):
    c = (np.arange(n + 2 * G) - G - (n - 1) / 2) * h
    Z, Y, X = np.meshgrid(c + centre[2], c + centre[1], c + centre[0], indexing="ij")
    vals = f(X, Y, Z)
    return np.stack([np.broadcast_to(np.asarray(v, dtype=float), X.shape) for v in vals])


def test_kerr_schild_stationary(orc, kerr_schild):
    centre = (2.0, 1.5, 1.2)
    prm = _params(orc, eps=0.0, slicing=2, shift=1)
    n = 5
    mid, rhs_err, cons_err = [], [], []
    for h in (0.08, 0.04, 0.02):
        st = np.ascontiguousarray(_ks_state(kerr_schild, centre, n, h))
        r = synth.interior(orc.bssn_rhs(st, G, h, prm), G)
        c = synth.interior(orc.bssn_constraints(st, G, h), G)
        mid.append(np.abs(r[NONGAUGE, 2, 2, 2]).max())
        rhs_err.append(np.abs(r[NONGAUGE]).max())
        cons_err.append(np.abs(c[:, 2, 2, 2]).max())
        # frozen gauge: RHS of lapse, shift and B exactly zero
        assert np.array_equal(r[17:], np.zeros_like(r[17:]))
    # at the fixed centre point the residual falls by 2^4 per halving of h
    for e in (mid, cons_err):
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert 14.5 < r1 < 17.5 and 15.0 < r2 < 17.0, e
    # over the (shrinking) patch interior it falls at least as fast
    assert rhs_err[0] / rhs_err[1] > 14.5 and rhs_err[1] / rhs_err[2] > 14.5, rhs_err
    assert mid[-1] < 1e-8


# ---------------------------------------------------------------------------
# Constant shift over polynomial lapse, Gamma^i and B^i
# ---------------------------------------------------------------------------

def _poly(rng, deg=4):
    terms = [(a, b, c) for a in range(deg + 1) for b in range(deg + 1) for c in range(deg + 1)
             if a + b + c <= deg]
    return {t: rng.uniform(-1, 1) for t in terms}


def _peval(coef, X, Y, Z, d=(0, 0, 0)):
    out = np.zeros_like(X)
    for (a, b, c), v in coef.items():
        e = [a, b, c]
        f = v
        for ax, m in enumerate(d):
            for _ in range(m):
                f *= e[ax]
                e[ax] -= 1
        if f != 0 and min(e) >= 0:
            out += f * X ** e[0] * Y ** e[1] * Z ** e[2]
    return out


def test_constant_shift_polynomial_reduction(orc):
    """Flat conformal metric, phi = K = At = 0, constant shift b, lapse,
    Gamma^i and B^i polynomials of degree 4 (4th-order stencils exact on
    them).  The system reduces to
      phi_t = gt_t = 0,  K_t = -Lap alpha,  alpha_t = b.grad alpha,
      At_t = [-d_i d_j alpha + alpha (d_i Gamma_j + d_j Gamma_i)/2]^TF,
      Gamma_t = b.grad Gamma,  beta_t = 3/4 B,  B_t = b.grad B - eta B,
    evaluated here with the polynomials' exact derivatives."""
    rng = np.random.default_rng(21)
    n, h, eta = 6, 0.05, 2.0
    c = (np.arange(n + 2 * G) - G) * h + 0.1
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    b = np.array([0.3, -0.2, 0.4])
    pa = _poly(rng)
    pg = [_poly(rng) for _ in range(3)]
    pb = [_poly(rng) for _ in range(3)]
    st = np.zeros((24,) + X.shape)
    st[:] = synth.BSSN_FLAT[:, None, None, None]
    st[17] = 1.0 + 0.1 * _peval(pa, X, Y, Z)
    for i in range(3):
        st[14 + i] = 0.1 * _peval(pg[i], X, Y, Z)
        st[18 + i] = b[i]
        st[21 + i] = 0.1 * _peval(pb[i], X, Y, Z)
    prm = _params(orc, eps=0.0, eta=eta)
    r = synth.interior(orc.bssn_rhs(st, G, h, prm), G)
    I = lambda a: synth.interior(a, G)
    unit = np.eye(3, dtype=int)
    grad = lambda p, s=0.1: [s * I(_peval(p, X, Y, Z, tuple(unit[k]))) for k in range(3)]
    dal = grad(pa)
    ddal = [[0.1 * I(_peval(pa, X, Y, Z, tuple(unit[i] + unit[j]))) for j in range(3)] for i in range(3)]
    lap = ddal[0][0] + ddal[1][1] + ddal[2][2]
    want = np.zeros_like(r)
    want[7] = -lap
    want[17] = sum(b[k] * dal[k] for k in range(3))
    dG = [grad(pg[i]) for i in range(3)]
    al = I(st[17])
    M = [[-ddal[i][j] + al * 0.5 * (dG[i][j] + dG[j][i]) for j in range(3)] for i in range(3)]
    tr = M[0][0] + M[1][1] + M[2][2]
    for i in range(3):
        for j in range(i, 3):
            want[8 + SYM[i][j]] = M[i][j] - (tr / 3 if i == j else 0)
    for i in range(3):
        want[14 + i] = sum(b[k] * dG[i][k] for k in range(3))
        want[18 + i] = 0.75 * I(st[21 + i])
        dB = grad(pb[i])
        want[21 + i] = sum(b[k] * dB[k] for k in range(3)) - eta * I(st[21 + i])
    np.testing.assert_allclose(r, want, rtol=0, atol=1e-9)


def test_thread_count_changes_no_value(orc):
    """The oracle's OpenMP loops give every point to one thread: one thread
    and all threads give the same RHS and RK4 step, bit for bit (the CPU
    baseline times it both ways)."""
    st, h = synth.bssn_noise(12, 10, 9, G, seed=11, amp=1e-2)
    orc.fill_ghosts(st, G)
    n = orc.num_threads()
    want_rhs = orc.bssn_rhs(st, G, h)
    want_step = orc.rk4(orc.BSSN, st, G, h, 0.25 * h, 1)
    orc.set_num_threads(1)
    try:
        got_rhs = orc.bssn_rhs(st, G, h)
        got_step = orc.rk4(orc.BSSN, st, G, h, 0.25 * h, 1)
    finally:
        orc.set_num_threads(n)
    assert orc.num_threads() == n
    assert np.array_equal(got_rhs, want_rhs) and np.array_equal(got_step, want_step)
