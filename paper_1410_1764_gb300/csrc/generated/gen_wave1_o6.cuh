// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// scalar wave, first-order form of Eq. 1 (u, rho, v_i), order-6 D, from gen/wave1.eqs
// generated: 42 fp64 instructions, 56 algorithmic flops, 0 exp, 0 rcp per point
// out(v, value) receives output v (5 outputs) as soon as it is computed
template <class LD, class SC, class OUT>
__device__ __forceinline__ void chemora_wave1_o6_point(const LD& ld, const SC& sc, OUT& out) {
  const double v_f1_0_0_0 = ld(1, 0, 0, 0);
  const double v_f2_1_0_0 = ld(2, 1, 0, 0);
  const double v_f2_m1_0_0 = ld(2, -1, 0, 0);
  const double t67 = fma(v_f2_m1_0_0, -sc.k[0], v_f2_1_0_0);
  const double v_f2_2_0_0 = ld(2, 2, 0, 0);
  const double v_f2_m2_0_0 = ld(2, -2, 0, 0);
  const double t70 = fma(v_f2_m2_0_0, -sc.k[0], v_f2_2_0_0);
  const double v_f2_3_0_0 = ld(2, 3, 0, 0);
  const double v_f2_m3_0_0 = ld(2, -3, 0, 0);
  const double t13737 = fma(v_f2_m3_0_0, -sc.k[0], v_f2_3_0_0);
  const double t13744 = fma(sc.k[21], t13737, fma(-sc.k[19], t70, fma(sc.k[14], t67, sc.k[1])));
  const double v_f3_0_1_0 = ld(3, 0, 1, 0);
  const double v_f3_0_m1_0 = ld(3, 0, -1, 0);
  const double t279 = fma(v_f3_0_m1_0, -sc.k[0], v_f3_0_1_0);
  const double v_f3_0_2_0 = ld(3, 0, 2, 0);
  const double v_f3_0_m2_0 = ld(3, 0, -2, 0);
  const double t282 = fma(v_f3_0_m2_0, -sc.k[0], v_f3_0_2_0);
  const double v_f3_0_3_0 = ld(3, 0, 3, 0);
  const double v_f3_0_m3_0 = ld(3, 0, -3, 0);
  const double t13746 = fma(v_f3_0_m3_0, -sc.k[0], v_f3_0_3_0);
  const double t13752 = fma(sc.k[21], t13746, fma(-sc.k[19], t282, fma(sc.k[14], t279, sc.k[1])));
  const double v_f4_0_0_1 = ld(4, 0, 0, 1);
  const double v_f4_0_0_m1 = ld(4, 0, 0, -1);
  const double t327 = fma(v_f4_0_0_m1, -sc.k[0], v_f4_0_0_1);
  const double v_f4_0_0_2 = ld(4, 0, 0, 2);
  const double v_f4_0_0_m2 = ld(4, 0, 0, -2);
  const double t330 = fma(v_f4_0_0_m2, -sc.k[0], v_f4_0_0_2);
  const double v_f4_0_0_3 = ld(4, 0, 0, 3);
  const double v_f4_0_0_m3 = ld(4, 0, 0, -3);
  const double t13755 = fma(v_f4_0_0_m3, -sc.k[0], v_f4_0_0_3);
  const double t13761 = fma(sc.k[21], t13755, fma(-sc.k[19], t330, fma(sc.k[14], t327, sc.k[1])));
  const double t13764 = fma(sc.ih, t13761, fma(sc.ih, t13752, fma(sc.ih, t13744, sc.k[1])));
  const double v_f1_1_0_0 = ld(1, 1, 0, 0);
  const double v_f1_m1_0_0 = ld(1, -1, 0, 0);
  const double t231 = fma(v_f1_m1_0_0, -sc.k[0], v_f1_1_0_0);
  const double v_f1_2_0_0 = ld(1, 2, 0, 0);
  const double v_f1_m2_0_0 = ld(1, -2, 0, 0);
  const double t234 = fma(v_f1_m2_0_0, -sc.k[0], v_f1_2_0_0);
  const double v_f1_3_0_0 = ld(1, 3, 0, 0);
  const double v_f1_m3_0_0 = ld(1, -3, 0, 0);
  const double t13765 = fma(v_f1_m3_0_0, -sc.k[0], v_f1_3_0_0);
  const double t13771 = fma(sc.k[21], t13765, fma(-sc.k[19], t234, fma(sc.k[14], t231, sc.k[1])));
  const double t13773 = fma(sc.ih, t13771, sc.k[1]);
  const double v_f1_0_1_0 = ld(1, 0, 1, 0);
  const double v_f1_0_m1_0 = ld(1, 0, -1, 0);
  const double t243 = fma(v_f1_0_m1_0, -sc.k[0], v_f1_0_1_0);
  const double v_f1_0_2_0 = ld(1, 0, 2, 0);
  const double v_f1_0_m2_0 = ld(1, 0, -2, 0);
  const double t246 = fma(v_f1_0_m2_0, -sc.k[0], v_f1_0_2_0);
  const double v_f1_0_3_0 = ld(1, 0, 3, 0);
  const double v_f1_0_m3_0 = ld(1, 0, -3, 0);
  const double t13774 = fma(v_f1_0_m3_0, -sc.k[0], v_f1_0_3_0);
  const double t13780 = fma(sc.k[21], t13774, fma(-sc.k[19], t246, fma(sc.k[14], t243, sc.k[1])));
  const double t13782 = fma(sc.ih, t13780, sc.k[1]);
  const double v_f1_0_0_1 = ld(1, 0, 0, 1);
  const double v_f1_0_0_m1 = ld(1, 0, 0, -1);
  const double t255 = fma(v_f1_0_0_m1, -sc.k[0], v_f1_0_0_1);
  const double v_f1_0_0_2 = ld(1, 0, 0, 2);
  const double v_f1_0_0_m2 = ld(1, 0, 0, -2);
  const double t258 = fma(v_f1_0_0_m2, -sc.k[0], v_f1_0_0_2);
  const double v_f1_0_0_3 = ld(1, 0, 0, 3);
  const double v_f1_0_0_m3 = ld(1, 0, 0, -3);
  const double t13783 = fma(v_f1_0_0_m3, -sc.k[0], v_f1_0_0_3);
  const double t13789 = fma(sc.k[21], t13783, fma(-sc.k[19], t258, fma(sc.k[14], t255, sc.k[1])));
  const double t13791 = fma(sc.ih, t13789, sc.k[1]);
  out(0, v_f1_0_0_0);
  out(1, t13764);
  out(2, t13773);
  out(3, t13782);
  out(4, t13791);
}
