// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// scalar wave, first-order form of Eq. 1 (u, rho, v_i), order-8 D, from gen/wave1.eqs
// generated: 54 fp64 instructions, 74 algorithmic flops, 0 exp, 0 rcp per point
// out(v, value) receives output v (5 outputs) as soon as it is computed
template <class LD, class SC, class OUT>
__device__ __forceinline__ void chemora_wave1_o8_point(const LD& ld, const SC& sc, OUT& out) {
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
  const double v_f2_4_0_0 = ld(2, 4, 0, 0);
  const double v_f2_m4_0_0 = ld(2, -4, 0, 0);
  const double t13845 = fma(v_f2_m4_0_0, -sc.k[0], v_f2_4_0_0);
  const double t13856 = fma(-sc.k[28], t13845, fma(sc.k[27], t13737, fma(-sc.k[23], t70, fma(sc.k[26], t67, sc.k[1]))));
  const double v_f3_0_1_0 = ld(3, 0, 1, 0);
  const double v_f3_0_m1_0 = ld(3, 0, -1, 0);
  const double t279 = fma(v_f3_0_m1_0, -sc.k[0], v_f3_0_1_0);
  const double v_f3_0_2_0 = ld(3, 0, 2, 0);
  const double v_f3_0_m2_0 = ld(3, 0, -2, 0);
  const double t282 = fma(v_f3_0_m2_0, -sc.k[0], v_f3_0_2_0);
  const double v_f3_0_3_0 = ld(3, 0, 3, 0);
  const double v_f3_0_m3_0 = ld(3, 0, -3, 0);
  const double t13746 = fma(v_f3_0_m3_0, -sc.k[0], v_f3_0_3_0);
  const double v_f3_0_4_0 = ld(3, 0, 4, 0);
  const double v_f3_0_m4_0 = ld(3, 0, -4, 0);
  const double t13860 = fma(v_f3_0_m4_0, -sc.k[0], v_f3_0_4_0);
  const double t13868 = fma(-sc.k[28], t13860, fma(sc.k[27], t13746, fma(-sc.k[23], t282, fma(sc.k[26], t279, sc.k[1]))));
  const double v_f4_0_0_1 = ld(4, 0, 0, 1);
  const double v_f4_0_0_m1 = ld(4, 0, 0, -1);
  const double t327 = fma(v_f4_0_0_m1, -sc.k[0], v_f4_0_0_1);
  const double v_f4_0_0_2 = ld(4, 0, 0, 2);
  const double v_f4_0_0_m2 = ld(4, 0, 0, -2);
  const double t330 = fma(v_f4_0_0_m2, -sc.k[0], v_f4_0_0_2);
  const double v_f4_0_0_3 = ld(4, 0, 0, 3);
  const double v_f4_0_0_m3 = ld(4, 0, 0, -3);
  const double t13755 = fma(v_f4_0_0_m3, -sc.k[0], v_f4_0_0_3);
  const double v_f4_0_0_4 = ld(4, 0, 0, 4);
  const double v_f4_0_0_m4 = ld(4, 0, 0, -4);
  const double t13873 = fma(v_f4_0_0_m4, -sc.k[0], v_f4_0_0_4);
  const double t13881 = fma(-sc.k[28], t13873, fma(sc.k[27], t13755, fma(-sc.k[23], t330, fma(sc.k[26], t327, sc.k[1]))));
  const double t13884 = fma(sc.ih, t13881, fma(sc.ih, t13868, fma(sc.ih, t13856, sc.k[1])));
  const double v_f1_1_0_0 = ld(1, 1, 0, 0);
  const double v_f1_m1_0_0 = ld(1, -1, 0, 0);
  const double t231 = fma(v_f1_m1_0_0, -sc.k[0], v_f1_1_0_0);
  const double v_f1_2_0_0 = ld(1, 2, 0, 0);
  const double v_f1_m2_0_0 = ld(1, -2, 0, 0);
  const double t234 = fma(v_f1_m2_0_0, -sc.k[0], v_f1_2_0_0);
  const double v_f1_3_0_0 = ld(1, 3, 0, 0);
  const double v_f1_m3_0_0 = ld(1, -3, 0, 0);
  const double t13765 = fma(v_f1_m3_0_0, -sc.k[0], v_f1_3_0_0);
  const double v_f1_4_0_0 = ld(1, 4, 0, 0);
  const double v_f1_m4_0_0 = ld(1, -4, 0, 0);
  const double t13887 = fma(v_f1_m4_0_0, -sc.k[0], v_f1_4_0_0);
  const double t13895 = fma(-sc.k[28], t13887, fma(sc.k[27], t13765, fma(-sc.k[23], t234, fma(sc.k[26], t231, sc.k[1]))));
  const double t13897 = fma(sc.ih, t13895, sc.k[1]);
  const double v_f1_0_1_0 = ld(1, 0, 1, 0);
  const double v_f1_0_m1_0 = ld(1, 0, -1, 0);
  const double t243 = fma(v_f1_0_m1_0, -sc.k[0], v_f1_0_1_0);
  const double v_f1_0_2_0 = ld(1, 0, 2, 0);
  const double v_f1_0_m2_0 = ld(1, 0, -2, 0);
  const double t246 = fma(v_f1_0_m2_0, -sc.k[0], v_f1_0_2_0);
  const double v_f1_0_3_0 = ld(1, 0, 3, 0);
  const double v_f1_0_m3_0 = ld(1, 0, -3, 0);
  const double t13774 = fma(v_f1_0_m3_0, -sc.k[0], v_f1_0_3_0);
  const double v_f1_0_4_0 = ld(1, 0, 4, 0);
  const double v_f1_0_m4_0 = ld(1, 0, -4, 0);
  const double t13900 = fma(v_f1_0_m4_0, -sc.k[0], v_f1_0_4_0);
  const double t13908 = fma(-sc.k[28], t13900, fma(sc.k[27], t13774, fma(-sc.k[23], t246, fma(sc.k[26], t243, sc.k[1]))));
  const double t13910 = fma(sc.ih, t13908, sc.k[1]);
  const double v_f1_0_0_1 = ld(1, 0, 0, 1);
  const double v_f1_0_0_m1 = ld(1, 0, 0, -1);
  const double t255 = fma(v_f1_0_0_m1, -sc.k[0], v_f1_0_0_1);
  const double v_f1_0_0_2 = ld(1, 0, 0, 2);
  const double v_f1_0_0_m2 = ld(1, 0, 0, -2);
  const double t258 = fma(v_f1_0_0_m2, -sc.k[0], v_f1_0_0_2);
  const double v_f1_0_0_3 = ld(1, 0, 0, 3);
  const double v_f1_0_0_m3 = ld(1, 0, 0, -3);
  const double t13783 = fma(v_f1_0_0_m3, -sc.k[0], v_f1_0_0_3);
  const double v_f1_0_0_4 = ld(1, 0, 0, 4);
  const double v_f1_0_0_m4 = ld(1, 0, 0, -4);
  const double t13913 = fma(v_f1_0_0_m4, -sc.k[0], v_f1_0_0_4);
  const double t13921 = fma(-sc.k[28], t13913, fma(sc.k[27], t13783, fma(-sc.k[23], t258, fma(sc.k[26], t255, sc.k[1]))));
  const double t13923 = fma(sc.ih, t13921, sc.k[1]);
  out(0, v_f1_0_0_0);
  out(1, t13884);
  out(2, t13897);
  out(3, t13910);
  out(4, t13923);
}
