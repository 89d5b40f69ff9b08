// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// variable-speed wave: u_t = rho, rho_t = s Lap u + grad s . grad u
// generated: 52 fp64 instructions, 64 algorithmic flops, 0 exp, 0 rcp per point
// out(v, value) receives output v (2 outputs) as soon as it is computed
template <class LD, class SC, class OUT>
__device__ __forceinline__ void chemora_varc_point(const LD& ld, const SC& sc, OUT& out) {
  const double v_f1_0_0_0 = ld(1, 0, 0, 0);
  const double v_f2_2_0_0 = ld(2, 2, 0, 0);
  const double v_f2_m2_0_0 = ld(2, -2, 0, 0);
  const double t70 = v_f2_2_0_0 - v_f2_m2_0_0;
  const double v_f2_1_0_0 = ld(2, 1, 0, 0);
  const double v_f2_m1_0_0 = ld(2, -1, 0, 0);
  const double t67 = v_f2_1_0_0 - v_f2_m1_0_0;
  const double t75 = fma(8.0, t67, (-t70));
  const double t77 = sc.i12h * t75;
  const double v_f0_2_0_0 = ld(0, 2, 0, 0);
  const double v_f0_m2_0_0 = ld(0, -2, 0, 0);
  const double t79 = v_f0_2_0_0 - v_f0_m2_0_0;
  const double v_f0_1_0_0 = ld(0, 1, 0, 0);
  const double v_f0_m1_0_0 = ld(0, -1, 0, 0);
  const double t78 = v_f0_1_0_0 - v_f0_m1_0_0;
  const double t83 = fma(8.0, t78, (-t79));
  const double t85 = sc.i12h * t83;
  const double v_f2_0_2_0 = ld(2, 0, 2, 0);
  const double v_f2_0_m2_0 = ld(2, 0, -2, 0);
  const double t92 = v_f2_0_2_0 - v_f2_0_m2_0;
  const double v_f2_0_1_0 = ld(2, 0, 1, 0);
  const double v_f2_0_m1_0 = ld(2, 0, -1, 0);
  const double t89 = v_f2_0_1_0 - v_f2_0_m1_0;
  const double t96 = fma(8.0, t89, (-t92));
  const double t98 = sc.i12h * t96;
  const double v_f0_0_2_0 = ld(0, 0, 2, 0);
  const double v_f0_0_m2_0 = ld(0, 0, -2, 0);
  const double t100 = v_f0_0_2_0 - v_f0_0_m2_0;
  const double v_f0_0_1_0 = ld(0, 0, 1, 0);
  const double v_f0_0_m1_0 = ld(0, 0, -1, 0);
  const double t99 = v_f0_0_1_0 - v_f0_0_m1_0;
  const double t104 = fma(8.0, t99, (-t100));
  const double t106 = sc.i12h * t104;
  const double v_f2_0_0_2 = ld(2, 0, 0, 2);
  const double v_f2_0_0_m2 = ld(2, 0, 0, -2);
  const double t114 = v_f2_0_0_2 - v_f2_0_0_m2;
  const double v_f2_0_0_1 = ld(2, 0, 0, 1);
  const double v_f2_0_0_m1 = ld(2, 0, 0, -1);
  const double t111 = v_f2_0_0_1 - v_f2_0_0_m1;
  const double t118 = fma(8.0, t111, (-t114));
  const double t120 = sc.i12h * t118;
  const double v_f0_0_0_2 = ld(0, 0, 0, 2);
  const double v_f0_0_0_m2 = ld(0, 0, 0, -2);
  const double t122 = v_f0_0_0_2 - v_f0_0_0_m2;
  const double v_f0_0_0_1 = ld(0, 0, 0, 1);
  const double v_f0_0_0_m1 = ld(0, 0, 0, -1);
  const double t121 = v_f0_0_0_1 - v_f0_0_0_m1;
  const double t126 = fma(8.0, t121, (-t122));
  const double t128 = sc.i12h * t126;
  const double v_f0_0_0_0 = ld(0, 0, 0, 0);
  const double t18 = v_f0_2_0_0 - v_f0_0_0_0;
  const double t20 = v_f0_m2_0_0 - v_f0_0_0_0;
  const double t35 = v_f0_0_2_0 - v_f0_0_0_0;
  const double t37 = v_f0_0_m2_0 - v_f0_0_0_0;
  const double t52 = v_f0_0_0_2 - v_f0_0_0_0;
  const double t54 = v_f0_0_0_m2 - v_f0_0_0_0;
  const double t10 = v_f0_1_0_0 - v_f0_0_0_0;
  const double t12 = v_f0_m1_0_0 - v_f0_0_0_0;
  const double t14 = t10 + t12;
  const double t28 = v_f0_0_1_0 - v_f0_0_0_0;
  const double t30 = v_f0_0_m1_0 - v_f0_0_0_0;
  const double t32 = t28 + t30;
  const double t45 = v_f0_0_0_1 - v_f0_0_0_0;
  const double t47 = v_f0_0_0_m1 - v_f0_0_0_0;
  const double t49 = t45 + t47;
  const double t61 = fma(16.0, t49, fma(16.0, t32, fma(16.0, t14, (-t18) - t20 - t35 - t37 - t52 - t54)));
  const double t64 = sc.i12h2 * t61;
  const double v_f2_0_0_0 = ld(2, 0, 0, 0);
  const double t134 = fma(t64, v_f2_0_0_0, fma(t120, t128, fma(t98, t106, t77 * t85)));
  out(0, v_f1_0_0_0);
  out(1, t134);
}
