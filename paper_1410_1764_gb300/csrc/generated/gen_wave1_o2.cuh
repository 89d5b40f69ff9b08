// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// scalar wave, first-order form of Eq. 1 (u, rho, v_i), order-2 D, from gen/wave1.eqs
// generated: 18 fp64 instructions, 20 algorithmic flops, 0 exp, 0 rcp per point
// out(v, value) receives output v (5 outputs) as soon as it is computed
template <class LD, class SC, class OUT>
__device__ __forceinline__ void chemora_wave1_o2_point(const LD& ld, const SC& sc, OUT& out) {
  const double v_f1_0_0_0 = ld(1, 0, 0, 0);
  const double v_f2_1_0_0 = ld(2, 1, 0, 0);
  const double v_f2_m1_0_0 = ld(2, -1, 0, 0);
  const double t67 = v_f2_1_0_0 - v_f2_m1_0_0;
  const double t13390 = 0.5 * t67;
  const double v_f3_0_1_0 = ld(3, 0, 1, 0);
  const double v_f3_0_m1_0 = ld(3, 0, -1, 0);
  const double t279 = v_f3_0_1_0 - v_f3_0_m1_0;
  const double t13393 = 0.5 * t279;
  const double v_f4_0_0_1 = ld(4, 0, 0, 1);
  const double v_f4_0_0_m1 = ld(4, 0, 0, -1);
  const double t327 = v_f4_0_0_1 - v_f4_0_0_m1;
  const double t13397 = 0.5 * t327;
  const double t13400 = fma(sc.ih, t13397, fma(sc.ih, t13393, sc.ih * t13390));
  const double v_f1_1_0_0 = ld(1, 1, 0, 0);
  const double v_f1_m1_0_0 = ld(1, -1, 0, 0);
  const double t231 = v_f1_1_0_0 - v_f1_m1_0_0;
  const double t13402 = 0.5 * t231;
  const double t13404 = sc.ih * t13402;
  const double v_f1_0_1_0 = ld(1, 0, 1, 0);
  const double v_f1_0_m1_0 = ld(1, 0, -1, 0);
  const double t243 = v_f1_0_1_0 - v_f1_0_m1_0;
  const double t13406 = 0.5 * t243;
  const double t13408 = sc.ih * t13406;
  const double v_f1_0_0_1 = ld(1, 0, 0, 1);
  const double v_f1_0_0_m1 = ld(1, 0, 0, -1);
  const double t255 = v_f1_0_0_1 - v_f1_0_0_m1;
  const double t13410 = 0.5 * t255;
  const double t13412 = sc.ih * t13410;
  out(0, v_f1_0_0_0);
  out(1, t13400);
  out(2, t13404);
  out(3, t13408);
  out(4, t13412);
}
