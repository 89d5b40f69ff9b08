"""Equation lists of the systems the generator turns into CUDA.

Each system is written once, symbolically, with tensor indices expanded by
Python loops (the Kranc tensor expansion of Sec. 3.2.3, restated): symmetric
tensors are stored as 6 components and index symmetry is respected because
identical components are the same DAG node.

  wave        Sec. 3 Eq. 1 in two-variable form: u_t = rho, rho_t = Lap u
  wave_varc   u_t = rho, rho_t = s Lap u + sum_d G_d D_d u (s = c^2 and
              G_d = D_d s, computed once when the speed is set, as read-only
              grid functions 2 and 3-5)
  bssn        Einstein equations, BSSN phi-form with 1+log (or harmonic, or
              frozen) slicing, Gamma-driver (or frozen) shift and
              Kreiss-Oliger dissipation on every evolved variable
"""
from fractions import Fraction

from . import expr as E
from .stencil import (val, d1, dd, ko, d1_raw, d2_raw, d11_raw, d1o_raw, d2o_raw, _centre_diffs, I12H,
                      I12H2, IH, IH2,
                      KO_SCALE)

SYM = ((0, 1, 2), (1, 3, 4), (2, 4, 5))
R3 = range(3)

# BSSN variable indices
PHI, GT, TRK, AT, XT, ALPHA, BETA, BB = 0, 1, 7, 8, 14, 17, 18, 21
NVARS = {"wave": 2, "wave_varc": 2, "bssn": 24}
GHOSTS = {"wave": 2, "wave_varc": 2, "bssn": 3}


def wave():
    """u_t = rho; rho_t = (sum_d (16 d1_d - d2_d)) / (12 h^2)."""
    lap_raw = E.box(sum((d2_raw(0, a) for a in R3), E.const(0)))
    return [E.box(val(1)), E.box(lap_raw * I12H2)]


def _d2raw(v, a):
    return E.box(16 * _centre_diffs(v, a, 1) - _centre_diffs(v, a, 2))


def wave_varc():
    """u_t = rho; rho_t = s Lap u + sum_d G_d D_d u, with s grid function 2
    and its centred first derivatives G_d = D_d s grid functions 3, 4, 5
    (the speed is constant in time, so D_d s is taken once, not per stage)."""
    U, S, G = 0, 2, 3
    lap = E.box(E.box(sum((_d2raw(U, a) for a in R3), E.const(0))) * I12H2)
    adv = sum((val(G + a) * d1(U, a) for a in R3), E.const(0))
    return [E.box(val(1)), E.box(val(S) * lap + adv)]


def _bssn_geometry():
    """Derivatives and geometric intermediates of the BSSN variables at a
    point, shared by the right-hand side and the constraints."""
    V = val
    phi = V(PHI)
    K = V(TRK)
    al = V(ALPHA)
    gt = [[V(GT + SYM[i][j]) for j in R3] for i in R3]
    At = [[V(AT + SYM[i][j]) for j in R3] for i in R3]
    Xt = [V(XT + i) for i in R3]
    be = [V(BETA + i) for i in R3]
    B = [V(BB + i) for i in R3]

    # first and second derivatives
    dphi = [d1(PHI, k) for k in R3]
    dK = [d1(TRK, k) for k in R3]
    dal = [d1(ALPHA, k) for k in R3]
    dgt = [[[d1(GT + SYM[i][j], k) for k in R3] for j in R3] for i in R3]
    dAt = [[[d1(AT + SYM[i][j], k) for k in R3] for j in R3] for i in R3]
    dXt = [[d1(XT + i, k) for k in R3] for i in R3]   # dXt[i][k] = d_k Xt^i
    dbe = [[d1(BETA + i, k) for k in R3] for i in R3]  # dbe[i][k] = d_k beta^i
    dB = [[d1(BB + i, k) for k in R3] for i in R3]
    ddphi = [[dd(PHI, a, b) for b in R3] for a in R3]
    ddal = [[dd(ALPHA, a, b) for b in R3] for a in R3]
    ddgt = [[[[dd(GT + SYM[i][j], a, b) for b in R3] for a in R3] for j in R3] for i in R3]
    ddbe = [[[dd(BETA + i, a, b) for b in R3] for a in R3] for i in R3]

    # advection beta^k D_k f with the stencil scale folded into the shift:
    # sum_k (beta^k / 12h) (12h D_k f)
    bs = [E.box(be[k] * I12H) for k in R3]

    def advect(df, v=None):
        if v is not None:
            return E.box(sum((bs[k] * d1_raw(v, k) for k in R3), E.const(0)))
        return E.box(sum((be[k] * df[k] for k in R3), E.const(0)))

    # gt^lm d_l d_m f from raw stencils, one scaling: pure terms carry
    # 1/(12h^2), mixed ones 1/(144h^2) = 1/(12h^2) / 12
    gtu6 = [[None] * 3 for _ in R3]

    def gtu_dd(v):
        acc = E.const(0)
        for l in R3:
            for m in R3:
                if l == m:
                    acc = acc + gtu[l][l] * d2_raw(v, l)
                elif l < m:
                    if gtu6[l][m] is None:
                        gtu6[l][m] = E.box(gtu[l][m] * E.const(Fraction(1, 6)))
                    acc = acc + gtu6[l][m] * d11_raw(v, l, m)
        return E.box(E.box(acc) * I12H2)

    # inverse conformal metric (adjugate / determinant, one reciprocal)
    c00 = E.box(gt[1][1] * gt[2][2] - gt[1][2] * gt[1][2])
    c01 = E.box(gt[1][2] * gt[0][2] - gt[0][1] * gt[2][2])
    c02 = E.box(gt[0][1] * gt[1][2] - gt[1][1] * gt[0][2])
    c11 = E.box(gt[0][0] * gt[2][2] - gt[0][2] * gt[0][2])
    c12 = E.box(gt[0][2] * gt[0][1] - gt[0][0] * gt[1][2])
    c22 = E.box(gt[0][0] * gt[1][1] - gt[0][1] * gt[0][1])
    det = E.box(gt[0][0] * c00 + gt[0][1] * c01 + gt[0][2] * c02)
    idet = E.rcp(det)
    cof = [[c00, c01, c02], [c01, c11, c12], [c02, c12, c22]]
    gtu = [[E.box(cof[i][j] * idet) for j in R3] for i in R3]

    # Christoffel symbols: first kind Gl[k][i][j], second kind Gu[k][i][j]
    Gl = [[[E.box(E.const(0.5) * (dgt[j][k][i] + dgt[i][k][j] - dgt[i][j][k]))
            for j in R3] for i in R3] for k in R3]
    Gu = [[[E.box(sum((gtu[k][l] * Gl[l][i][j] for l in R3), E.const(0)))
            for j in R3] for i in R3] for k in R3]
    Xtn = [E.box(sum((gtu[i][j] * Gu[k][i][j] for i in R3 for j in R3), E.const(0))) for k in R3]
    e4 = E.exp(-4 * phi)

    # raised traceless curvature
    Atm = [[E.box(sum((gtu[i][k] * At[k][j] for k in R3), E.const(0))) for j in R3] for i in R3]
    Atu = [[None] * 3 for _ in R3]
    for i in R3:
        for j in range(i, 3):  # symmetric: evaluate once
            Atu[i][j] = Atu[j][i] = E.box(sum((Atm[i][k] * gtu[k][j] for k in R3), E.const(0)))
    AA = E.box(sum((At[i][j] * Atu[i][j] for i in R3 for j in R3), E.const(0)))

    # Ricci tensor
    DDphi = [[E.box(ddphi[i][j] - sum((Gu[k][i][j] * dphi[k] for k in R3), E.const(0)))
              for j in R3] for i in R3]
    tr_DDphi = E.box(sum((gtu[l][m] * DDphi[l][m] for l in R3 for m in R3), E.const(0)))
    dphi2 = E.box(sum((gtu[l][m] * dphi[l] * dphi[m] for l in R3 for m in R3), E.const(0)))
    # Christoffels of the first kind with the last index raised:
    # C[j][k][l] = gt^{lm} Gamma~_{jkm}.  The quadratic Ricci terms
    #   gt^lm (G^k_li G_jkm + G^k_lj G_ikm + G^k_im G_klj)
    # become sum_kl (G^k_li C_jk^l + G^k_lj C_ik^l + G^k_il C_kj^l)
    # (the third uses the symmetry G_klj = G_kjl).
    C = [[[E.box(sum((gtu[l][m] * Gl[j][k][m] for m in R3), E.const(0))) for l in R3]
          for k in R3] for j in R3]
    R = [[None] * 3 for _ in R3]
    for i in R3:
        for j in range(i, 3):
            t1 = gtu_dd(GT + SYM[i][j])
            t2 = sum((gt[k][i] * dXt[k][j] + gt[k][j] * dXt[k][i] for k in R3), E.const(0))
            t3 = sum((Xtn[k] * (Gl[i][j][k] + Gl[j][i][k]) for k in R3), E.const(0))
            t4 = sum((Gu[k][l][i] * C[j][k][l] + Gu[k][l][j] * C[i][k][l] + Gu[k][i][l] * C[k][j][l]
                      for k in R3 for l in R3), E.const(0))
            Rt = -0.5 * t1 + 0.5 * t2 + 0.5 * t3 + t4
            Rp = (-2 * DDphi[i][j] - 2 * gt[i][j] * tr_DDphi + 4 * dphi[i] * dphi[j]
                  - 4 * gt[i][j] * dphi2)
            R[i][j] = R[j][i] = E.box(Rt + Rp)

    # lapse Hessian (conformal decomposition) and its physical trace
    dphidal = E.box(sum((gtu[k][l] * dphi[k] * dal[l] for k in R3 for l in R3), E.const(0)))
    DDal = [[None] * 3 for _ in R3]
    for i in R3:
        for j in range(i, 3):
            DDal[i][j] = DDal[j][i] = E.box(
                ddal[i][j] - sum((Gu[k][i][j] * dal[k] for k in R3), E.const(0))
                - 2 * (dphi[i] * dal[j] + dphi[j] * dal[i]) + 2 * gt[i][j] * dphidal)
    tr_ddal = sum((gtu[i][j] * ddal[i][j] for i in R3 for j in R3), E.const(0))
    Xdal = sum((Xtn[k] * dal[k] for k in R3), E.const(0))
    trDDal = E.box(e4 * E.box(tr_ddal - Xdal + 2 * dphidal))

    return dict(locals())


def bssn(eta_sym="eta"):
    """BSSN right-hand side, all 24 variables, KO included on every evolved
    variable.  The gauge is chosen at run time: sc.slicing 0 1+log,
    1 harmonic, 2 frozen lapse; sc.shift 0 Gamma-driver, 1 frozen shift and B
    (frozen variables have a zero right-hand side and no dissipation).
    An output is a node or a list of (condition, node) alternatives."""
    eta = E.sym(eta_sym)
    G = _bssn_geometry()
    (phi, K, al, gt, At, Xt, be, B) = (G["phi"], G["K"], G["al"], G["gt"], G["At"], G["Xt"], G["be"], G["B"])
    (dphi, dK, dal, dgt, dAt, dXt, dbe, dB) = (G["dphi"], G["dK"], G["dal"], G["dgt"], G["dAt"], G["dXt"],
                                               G["dbe"], G["dB"])
    (ddbe, gtu, Gl, Gu, Xtn, e4, Atm, Atu, AA, R, DDal, trDDal, advect, gtu_dd) = (
        G["ddbe"], G["gtu"], G["Gl"], G["Gu"], G["Xtn"], G["e4"], G["Atm"], G["Atu"], G["AA"], G["R"],
        G["DDal"], G["trDDal"], G["advect"], G["gtu_dd"])
    divbe = E.box(dbe[0][0] + dbe[1][1] + dbe[2][2])
    out = [None] * 24
    out[PHI] = advect(dphi, PHI) + E.const(1) / 6 * (divbe - al * K)
    for i in R3:
        for j in range(i, 3):
            s = advect(dgt[i][j], GT + SYM[i][j])
            s = s + sum((gt[i][k] * dbe[k][j] + gt[j][k] * dbe[k][i] for k in R3), E.const(0))
            s = s - E.const(2) / 3 * gt[i][j] * divbe - 2 * al * At[i][j]
            out[GT + SYM[i][j]] = s
    out[TRK] = advect(dK, TRK) - trDDal + al * (AA + E.const(1) / 3 * K * K)
    X = [[E.box(-DDal[i][j] + al * R[i][j]) for j in R3] for i in R3]
    trX = E.box(sum((gtu[k][l] * X[k][l] for k in R3 for l in R3), E.const(0)))
    for i in R3:
        for j in range(i, 3):
            s = advect(dAt[i][j], AT + SYM[i][j])
            s = s + sum((At[i][k] * dbe[k][j] + At[j][k] * dbe[k][i] for k in R3), E.const(0))
            s = s - E.const(2) / 3 * At[i][j] * divbe
            s = s + e4 * E.box(X[i][j] - E.const(1) / 3 * gt[i][j] * trX)
            AtAt = sum((At[i][k] * Atm[k][j] for k in R3), E.const(0))
            s = s + al * E.box(K * At[i][j] - 2 * AtAt)
            out[AT + SYM[i][j]] = s
    # sum_k d_j d_k beta^k from raw stencils, one scaling (mixed / 12)
    ddbe_div = [E.box(E.box(d2_raw(BETA + j, j)
                            + sum((E.const(Fraction(1, 12)) * d11_raw(BETA + k, min(j, k), max(j, k))
                                   for k in R3 if k != j), E.const(0))) * I12H2) for j in R3]
    rXt = [None] * 3
    for i in R3:
        s = advect(dXt[i], XT + i)
        s = s - sum((Xtn[j] * dbe[i][j] for j in R3), E.const(0))
        s = s + E.const(2) / 3 * Xtn[i] * divbe
        s = s + gtu_dd(BETA + i)
        s = s + E.const(1) / 3 * sum((gtu[i][j] * ddbe_div[j] for j in R3), E.const(0))
        s = s - 2 * sum((Atu[i][j] * dal[j] for j in R3), E.const(0))
        t = (sum((Gu[i][j][k] * Atu[j][k] for j in R3 for k in R3), E.const(0))
             + 6 * sum((Atu[i][j] * dphi[j] for j in R3), E.const(0))
             - E.const(2) / 3 * sum((gtu[i][j] * dK[j] for j in R3), E.const(0)))
        s = s + 2 * al * E.box(t)
        rXt[i] = E.box(s)
        out[XT + i] = rXt[i]
    # gauge: alternatives selected at run time by the uniform flags
    kov = {v: ko(v) for v in (ALPHA,) + tuple(range(BETA, BB + 3))}
    out[ALPHA] = [("sc.slicing == 0", E.box(advect(dal, ALPHA) - 2 * al * K) + kov[ALPHA]),
                  ("sc.slicing == 1", E.box(advect(dal, ALPHA) - al * al * K) + kov[ALPHA]),
                  (None, E.const(0))]
    for i in R3:
        out[BETA + i] = [("sc.shift == 0", E.box(advect(dbe[i], BETA + i) + E.const(3) / 4 * B[i]) + kov[BETA + i]),
                         (None, E.const(0))]
        out[BB + i] = [("sc.shift == 0", E.box(advect(dB[i], BB + i) + (rXt[i] - advect(dXt[i], XT + i)) - eta * B[i])
                        + kov[BB + i]), (None, E.const(0))]
    return [out[v] if isinstance(out[v], list) else E.box(out[v]) + ko(v) for v in range(24)]


def bssn_constraints():
    """BSSN constraints at a point (7 outputs):
      H   = R + 2/3 K^2 - At_ij At^ij,  R = e^{-4 phi} gt^ij R_ij
      M^i = d_j At^ij + Gamma~^i_jk At^jk + 6 At^ij d_j phi - 2/3 gt^ij d_j K,
            d_j At^ij by the product rule with d_k gt^ij = -gt^ia gt^jb d_k gt_ab
      G^i = Xt^i - Gamma~^i_(d)."""
    G = _bssn_geometry()
    gtu, R, e4, K, AA = G["gtu"], G["R"], G["e4"], G["K"], G["AA"]
    At, Atu, Gu, dgt, dAt, dphi, dK, Xt, Xtn = (G["At"], G["Atu"], G["Gu"], G["dgt"], G["dAt"],
                                                G["dphi"], G["dK"], G["Xt"], G["Xtn"])
    trR = E.box(sum((gtu[i][j] * R[i][j] for i in R3 for j in R3), E.const(0)))
    H = E.box(e4 * trR + E.const(2) / 3 * K * K - AA)
    dgtu = [[[E.box(-sum((gtu[i][a] * gtu[j][b] * dgt[a][b][k] for a in R3 for b in R3), E.const(0)))
              for k in R3] for j in R3] for i in R3]
    out = [H]
    for i in R3:
        div = sum((dgtu[i][a][j] * gtu[j][b] * At[a][b] + gtu[i][a] * dgtu[j][b][j] * At[a][b]
                   + gtu[i][a] * gtu[j][b] * dAt[a][b][j] for j in R3 for a in R3 for b in R3), E.const(0))
        m = (div + sum((Gu[i][j][k] * Atu[j][k] for j in R3 for k in R3), E.const(0))
             + 6 * sum((Atu[i][j] * dphi[j] for j in R3), E.const(0))
             - E.const(2) / 3 * sum((gtu[i][j] * dK[j] for j in R3), E.const(0)))
        out.append(E.box(m))
    for i in R3:
        out.append(E.box(Xt[i] - Xtn[i]))
    return out


def wave_order(order):
    """Two-variable scalar wave with an order-p Laplacian:
    u_t = rho, rho_t = (1/h^2) sum_d sum_k b_k d_k,d."""
    lap = E.box(sum((d2o_raw(0, a, order) for a in R3), E.const(0)))
    return [E.box(val(1)), E.box(lap * IH2)]


def wave1(order):
    """First-order form of Eq. 1, variables (u, rho, v_x, v_y, v_z):
    u_t = rho, rho_t = sum_i D_i v_i, (v_i)_t = D_i rho (order-p D)."""
    div = E.box(sum((d1o_raw(2 + a, a, order) for a in R3), E.const(0)))
    return ([E.box(val(1)), E.box(div * IH)]
            + [E.box(d1o_raw(1, a, order) * IH) for a in R3])
